// Solve-phase kernels of the AMS-preconditioned CG (one GPU, sm_103a).
//
// One CG iteration (Section 3.1 preconditioner inside CG) is five kernels:
//   k_dir_update      p = z + beta p_old
//   k_spmv_dot        q = A p and p.q                          (SELL-32 SpMV)
//   k_local_solve     z_f = sum_i R_i^T A_i^{-1} R_i r'  and  r_c = R_0 r',
//   (k_local_tma*)    r' = r - alpha q formed on the fly       (alpha = rho/pq)
//   k_coarse_*        y = L_c^{-1} r_c  (k_coarse.cu)          (A_0 = L_c L_c^T)
//   k_prolong_update  e_c = L_c^{-T} y, z = z_f + R_0^T e_c, r = r',
//                     x += alpha p, r.z, r.r, z.q, convergence test, beta
#include <cstdint>
#include <cstdio>
#include <type_traits>

#include "ams_internal.h"
#include "kernels.cuh"
#include "launch.h"
#include "mma_tf32.cuh"

namespace ams {

// ===========================================================================
// a1: SpMV q = A p and the dot p.q per (system, rhs) (SELL-32: slice s =
// rows 32s..32s+31, entry j of lane l at sell_ptr[s] + 32 j + l; padded
// entries have value 0 and a valid column).  One element (row, rhs) per
// thread per step; the first JU entries of the row are loaded before any
// product, so their loads and then their gathers are in flight together.
// FP64 arithmetic is scarce on this GPU (about 1/64 of the FP32 rate), so
// the direction update p = z + beta p_old runs as its own streaming pass
// (k_dir_update) rather than being recomputed for every gathered entry.
// with_dot = 0: plain product (no dot, no solve state).
// ===========================================================================
template <int LD, int JU>
__global__ void __launch_bounds__(kRedThreads)
k_spmv_dot(const int64_t* __restrict__ sell_ptr, const int32_t* __restrict__ sell_col,
           const double* __restrict__ sell_val, const double* __restrict__ p, double* __restrict__ q,
           RedLayout R, CgScalars* sc, SolveState* st, int with_dot) {
    __shared__ double s_out[kRedMaxNV * kMaxLd];
    __shared__ double s_scr[kRedThreads];
    const int rhs = threadIdx.x % LD;                // kRedThreads is a multiple of LD
    const int64_t lo = R.blk_lo[blockIdx.x], hi = R.blk_lo[blockIdx.x + 1];
    int64_t b0 = 0;
    int w = 0, lane = 0;
    int col[JU];
    double val[JU];
    // matrix entries of one element (setup data: may be read before pdl_wait)
    auto load_row = [&](int64_t e) {
        const int64_t row = e / LD;
        const int64_t sl = row >> 5;
        lane = (int)(row & 31);
        b0 = __ldg(sell_ptr + sl);
        w = (int)((__ldg(sell_ptr + sl + 1) - b0) >> 5);
#pragma unroll
        for (int j = 0; j < JU; ++j) {
            col[j] = 0;
            val[j] = 0.0;
            if (j < w) {
                col[j] = __ldg(sell_col + b0 + 32 * j + lane);
                val[j] = __ldg(sell_val + b0 + 32 * j + lane);
            }
        }
    };
    int64_t e = lo + threadIdx.x;
    if (e < hi) load_row(e);
    pdl_wait();
    if (st != nullptr && st->done) return;
    double dot[1] = {0.0};
    while (e < hi) {
        double xv[JU];
#pragma unroll
        for (int j = 0; j < JU; ++j) {
            xv[j] = 0.0;
            if (j < w && AMS_ROW_OK(col[j], 1)) xv[j] = __ldg(p + (int64_t)col[j] * LD + rhs);
        }
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < JU; ++j)
            if (j < w) acc = fma(val[j], xv[j], acc);
        for (int j = JU; j < w; ++j) {
            const int64_t o = b0 + 32 * j + lane;
            const int cj = __ldg(sell_col + o);
            if (AMS_ROW_OK(cj, 1)) acc = fma(__ldg(sell_val + o), __ldg(p + (int64_t)cj * LD + rhs), acc);
        }
        q[e] = acc;
        if (with_dot) dot[0] = fma(__ldg(p + e), acc, dot[0]);
        e += kRedThreads;
        if (e < hi) load_row(e);
    }
    pdl_trigger();
    if (!with_dot) return;
    int seg;
    if (!seg_reduce<1>(dot, LD, R, s_out, s_scr, seg)) return;
    if (threadIdx.x < LD) {
        CgScalars& c = sc[seg * LD + threadIdx.x];
        c.pq = s_out[threadIdx.x];
        if (c.active && !(c.pq > 0.0 && isfinite(c.pq))) {
            st->status = AMS_ERR_BREAKDOWN;
            st->done = 1;
        }
    }
}

// a7: p_new = z + beta p_old per (system, rhs); p_old and p_new are
// different buffers (successive iterations alternate them).  XUPD: this
// launch also applies the previous iteration's x += alpha p_old (from 8
// right-hand sides, where the prolongation leaves it); without it the
// kernel is the bare direction update.
template <int LD, typename ZT, bool XUPD>
__global__ void __launch_bounds__(kRedThreads)
k_dir_update(const ZT* __restrict__ z, const double* __restrict__ p_old, double* __restrict__ p_new,
             double* __restrict__ x, RedLayout R, const CgScalars* sc, SolveState* st) {
    pdl_wait();
    if (st->done) return;
    pdl_trigger();
    const CgScalars& c = sc[R.blk_seg[blockIdx.x] * LD + threadIdx.x % LD];
    const int64_t lo = R.blk_lo[blockIdx.x], hi = R.blk_lo[blockIdx.x + 1];
    if constexpr (!XUPD) {
        const double beta = c.beta;
#pragma unroll 4
        for (int64_t e = lo + threadIdx.x; e < hi; e += kRedThreads) p_new[e] = fma(beta, p_old[e], widen(z[e]));
    } else {
        if (blockIdx.x == 0 && threadIdx.x == 0) st->xdone_it = st->it;
        const double beta = c.beta, alpha = c.alpha;
        const bool xupd = c.xpend != 0;
#pragma unroll 4
        for (int64_t e = lo + threadIdx.x; e < hi; e += kRedThreads) {
            const double po = p_old[e];
            p_new[e] = fma(beta, po, widen(z[e]));
            if (xupd) x[e] = fma(alpha, po, x[e]);   // the previous iteration's x += alpha p
        }
    }
}

// After the loop: the last iteration's x += alpha p, unless a direction
// update ran after it (a breakdown found by the next SpMV ends the loop
// after that update).  Its direction is the one that iteration computed:
// iteration k writes p2 when k is even, p when it is odd.
template <int LD>
__global__ void __launch_bounds__(kRedThreads)
k_x_flush(const double* __restrict__ p, const double* __restrict__ p2, double* __restrict__ x, RedLayout R,
          const CgScalars* sc, const SolveState* st) {
    const int it = st->it;
    if (it == 0 || st->xdone_it == it) return;
    const CgScalars& c = sc[R.blk_seg[blockIdx.x] * LD + threadIdx.x % LD];
    if (!c.xpend) return;
    const double alpha = c.alpha;
    const double* pl = ((it - 1) % 2 == 0) ? p2 : p;
    const int64_t lo = R.blk_lo[blockIdx.x], hi = R.blk_lo[blockIdx.x + 1];
    for (int64_t e = lo + threadIdx.x; e < hi; e += kRedThreads) x[e] = fma(alpha, pl[e], x[e]);
}

// ===========================================================================
// a3+a4: local solves z_f = A_i^{-1} r_i for every subdomain (one thread
// block per subdomain, warps split the right-hand sides, NR per warp), with
// the restriction r_c = Psi_i^T r_i accumulated on the way.
//
// Forward sweep over block rows K = 0..nb-1 (lane = row of the block):
//   t   = r_K - sum_{d<c} L_{K,K-c+d} y_{K-c+d}
//   y_K = L_KK^{-1} t
// Backward sweep K = nb-1..0 (lane = column of the block):
//   w   = y_K - sum_{d=1..c} L_{K+d,K}^T x_{K+d}
//   x_K = L_KK^{-T} w
// Factor block rows are staged through shared memory with cp.async in a
// ring of c+D+1 buffers, D block rows ahead of the sweep (one commit group
// per block row); y is kept in z_f between the sweeps.
// ===========================================================================
template <typename TF, typename TP, int NR, int MM>
__global__ void k_local_solve(const SubInfo* __restrict__ subs, const TF* __restrict__ fac,
                              const double* __restrict__ rin, const double* __restrict__ qin,
                              const CgScalars* __restrict__ csc, const double* __restrict__ rowscale,
                              TF* __restrict__ zf, const TP* __restrict__ psi, TF* __restrict__ rc,
                              int ld, int cmax, int depth, const SolveState* st) {
    pdl_wait();
    if (st != nullptr && st->done) return;
    using A = typename Acc<TF>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SubInfo S = subs[blockIdx.x];
    const int c = S.c, nb = S.nb, n = S.n;
    const int D = depth;                                       // block rows in flight
    const int nbuf = c + D + 1;
    const int64_t brs = blockrow_elems(c);
    const int64_t brs_max = blockrow_elems(cmax);
    TF* bufs = (TF*)smem_raw;                                  // (cmax+D+1) * brs_max
    TF* ring = bufs + (int64_t)(cmax + D + 1) * brs_max;       // (cmax+1) * 32 * ld
    TF* tmp = ring + (int64_t)(cmax + 1) * 32 * ld;            // 32 * ld
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int rhs0 = warp * NR;
    const TF* F = fac + S.fac_off;
    const int m = S.m;

    A racc[MM][NR];
#pragma unroll
    for (int k = 0; k < MM; ++k)
#pragma unroll
        for (int j = 0; j < NR; ++j) racc[k][j] = A(0);

    // r' = r - alpha q for (system, rhs) pairs still iterating (see ResidIn)
    double al[NR];
    bool upd[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        al[j] = 0.0;
        upd[j] = false;
        if (qin != nullptr) {
            const CgScalars cj = csc[(int64_t)S.seg * ld + rhs0 + j];
            upd[j] = cj.active != 0;
            if (upd[j]) al[j] = cj.rho / cj.pq;
        }
    }
    // Inputs of block row K (r and q rows, basis rows, row scale) are
    // loaded two block rows ahead into alternating register buffers and
    // kept in their loaded type until the step that uses them, so their
    // global-memory latency overlaps the substitution of earlier rows.
    auto load_fwd = [&](int K, double (&rv)[NR], double (&qv)[NR], TP (&pv)[MM], double& scv) {
        const int row = K * 32 + lane;
        const bool valid = K < nb && row < n;
        const int64_t grow = S.row0 + row;
        scv = 1.0;
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            rv[j] = 0.0;
            qv[j] = 0.0;
        }
#pragma unroll
        for (int k = 0; k < MM; ++k) pv[k] = TP(0.f);
        if (valid) {
            if (rowscale != nullptr) scv = rowscale[grow];
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                rv[j] = rin[grow * ld + rhs0 + j];
                if (upd[j]) qv[j] = qin[grow * ld + rhs0 + j];
            }
            if (rc != nullptr) {
#pragma unroll
                for (int k = 0; k < MM; ++k)
                    if (k < m) pv[k] = psi[S.psi_off + (int64_t)row * m + k];
            }
        }
    };
    double rb[2][NR], qb[2][NR], sb[2];
    TP pb[2][MM];
    load_fwd(0, rb[0], qb[0], pb[0], sb[0]);
    load_fwd(1, rb[1], qb[1], pb[1], sb[1]);

    // ---------------- forward ----------------
    // one commit group per block row; row K+D is requested at step K
    for (int j = 0; j < D; ++j) {
        if (j < nb) block_copy_async(bufs + (int64_t)(j % nbuf) * brs_max, F + (int64_t)j * brs, brs * sizeof(TF));
        cp_async_commit();
    }
    auto fwd_step = [&](int K, double (&rv)[NR], double (&qv)[NR], TP (&pb_)[MM], double& scv) {
        if (K + D < nb)
            block_copy_async(bufs + (int64_t)((K + D) % nbuf) * brs_max, F + (int64_t)(K + D) * brs,
                             brs * sizeof(TF));
        cp_async_commit();
        A t[NR], pv[MM];
#pragma unroll
        for (int j = 0; j < NR; ++j) t[j] = (A)((upd[j] ? fma(-al[j], qv[j], rv[j]) : rv[j]) * scv);
#pragma unroll
        for (int k = 0; k < MM; ++k) pv[k] = (A)to_d(pb_[k]);
        load_fwd(K + 2, rv, qv, pb_, scv);
        cp_async_wait_n(D);
        __syncthreads();
        const TF* B = bufs + (int64_t)(K % nbuf) * brs_max;
        const int row = K * 32 + lane;
        const bool valid = row < n;
        const int64_t grow = S.row0 + row;
        if (rc != nullptr) {
#pragma unroll
            for (int k = 0; k < MM; ++k)
#pragma unroll
                for (int j = 0; j < NR; ++j) racc[k][j] += pv[k] * t[j];
        }
        for (int d = 0; d < c; ++d) {
            const int src = K - c + d;
            if (src < 0) continue;
            const TF* T = B + d * 1024;
            const TF* ys = ring + (int64_t)(src % (c + 1)) * 32 * ld + rhs0;
#pragma unroll 8
            for (int q = 0; q < 32; ++q) {
                A coef = (A)T[tile_idx(lane, q)];
                if (d == 0 && q < lane) coef = A(0);
#pragma unroll
                for (int j = 0; j < NR; ++j) t[j] -= coef * (A)ys[q * ld + j];
            }
        }
#pragma unroll
        for (int j = 0; j < NR; ++j) tmp[lane * ld + rhs0 + j] = (TF)t[j];
        __syncwarp();
        const A piv = (A)B[c * 1024 + lane];
        A y[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) y[j] = piv * t[j];
#pragma unroll 8
        for (int q = 0; q < 32; ++q) {
            const A coef = q < lane ? (A)B[tile_idx(lane, q)] : A(0);
#pragma unroll
            for (int j = 0; j < NR; ++j) y[j] += coef * (A)tmp[q * ld + rhs0 + j];
        }
        TF* yr = ring + (int64_t)(K % (c + 1)) * 32 * ld + rhs0;
#pragma unroll
        for (int j = 0; j < NR; ++j) yr[lane * ld + j] = (TF)y[j];
        if (valid) {
#pragma unroll
            for (int j = 0; j < NR; ++j) zf[grow * ld + rhs0 + j] = (TF)y[j];
        }
        __syncthreads();
    };
#pragma unroll 1
    for (int K = 0; K < nb; K += 2) {
        fwd_step(K, rb[0], qb[0], pb[0], sb[0]);
        if (K + 1 < nb) fwd_step(K + 1, rb[1], qb[1], pb[1], sb[1]);
    }
    pdl_trigger();
    // restriction: reduce over lanes, lane 0 writes r_c rows of this subdomain
    if (rc != nullptr) {
#pragma unroll
        for (int k = 0; k < MM; ++k) {
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                A v = racc[k][j];
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if (lane == 0 && k < m) rc[(S.coff + k) * ld + rhs0 + j] = (TF)v;
            }
        }
    }
    // ---------------- backward ----------------
    // step K needs block rows K..K+c; row K-D is requested at step K
    cp_async_wait_all();
    __syncthreads();
    for (int j = 0; j < D; ++j) {
        const int r = nb - 1 - j;
        if (r >= 0) block_copy_async(bufs + (int64_t)(r % nbuf) * brs_max, F + (int64_t)r * brs, brs * sizeof(TF));
        cp_async_commit();
    }
    auto load_bwd = [&](int K, TF (&wv)[NR]) {
        const int row = K * 32 + lane;
        const bool valid = K >= 0 && row < n;
        const int64_t grow = S.row0 + row;
#pragma unroll
        for (int j = 0; j < NR; ++j) wv[j] = TF(0);
        if (valid) {
#pragma unroll
            for (int j = 0; j < NR; ++j) wv[j] = zf[grow * ld + rhs0 + j];
        }
    };
    TF wb[2][NR];
    load_bwd(nb - 1, wb[0]);
    load_bwd(nb - 2, wb[1]);
    auto bwd_step = [&](int K, TF (&wv)[NR]) {
        if (K - D >= 0)
            block_copy_async(bufs + (int64_t)((K - D) % nbuf) * brs_max, F + (int64_t)(K - D) * brs,
                             brs * sizeof(TF));
        cp_async_commit();
        A w[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) w[j] = (A)wv[j];
        load_bwd(K - 2, wv);
        cp_async_wait_n(D);
        __syncthreads();
        const int row = K * 32 + lane;
        const bool valid = row < n;
        const int64_t grow = S.row0 + row;
        for (int d = 1; d <= c; ++d) {
            const int src = K + d;
            if (src >= nb) break;
            const TF* Bs = bufs + (int64_t)(src % nbuf) * brs_max;
            const TF* T = (d < c) ? Bs + (c - d) * 1024 : Bs;
            const TF* xs = ring + (int64_t)(src % (c + 1)) * 32 * ld + rhs0;
#pragma unroll 8
            for (int r = 0; r < 32; ++r) {
                A coef = (A)T[tile_idx(r, lane)];
                if (d == c && r > lane) coef = A(0);
#pragma unroll
                for (int j = 0; j < NR; ++j) w[j] -= coef * (A)xs[r * ld + j];
            }
        }
#pragma unroll
        for (int j = 0; j < NR; ++j) tmp[lane * ld + rhs0 + j] = (TF)w[j];
        __syncwarp();
        const TF* B = bufs + (int64_t)(K % nbuf) * brs_max;
        const A piv = (A)B[c * 1024 + lane];
        A x[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) x[j] = piv * w[j];
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
            const A coef = r > lane ? (A)B[tile_idx(r, lane)] : A(0);
#pragma unroll
            for (int j = 0; j < NR; ++j) x[j] += coef * (A)tmp[r * ld + rhs0 + j];
        }
        TF* xr = ring + (int64_t)(K % (c + 1)) * 32 * ld + rhs0;
#pragma unroll
        for (int j = 0; j < NR; ++j) xr[lane * ld + j] = (TF)x[j];
        if (valid) {
#pragma unroll
            for (int j = 0; j < NR; ++j) zf[grow * ld + rhs0 + j] = (TF)x[j];
        }
        __syncthreads();
    };
#pragma unroll 1
    for (int K = nb - 1; K >= 0; K -= 2) {
        bwd_step(K, wb[0]);
        if (K - 1 >= 0) bwd_step(K - 1, wb[1]);
    }
}

// ===========================================================================
// a5 (backward substitution) + a6 + a2: e_c = L_c^{-T} y, z = z_f + R_0^T e_c,
// the CG update and the dots.  A thread block takes a range of consecutive
// subdomains of one system.  Per subdomain: its m_i rows of e_c are the
// product of its rows of the backward block of its nested-dissection node
// (L_c^{-T} restricted to the node's rows and the columns of the node and
// its ancestors) with y gathered at those columns; the block reduces them
// in a fixed order into shared memory, then prolongates over the
// subdomain's contiguous rows (basis rows by 16-byte loads).  With many
// right-hand sides the per-subdomain gathers of y cost more than a separate
// backward launch: then e_c comes in precomputed (ec != NULL).  Padded rows
// belong to no subdomain: their z stays 0 and r, q, x are 0.
//
// mode 0: z only (a plain preconditioner application).
// mode 1: first application of a solve: z and rho = r.z (beta = 0).
// mode 2: CG iteration.  For (system, rhs) pairs still iterating,
//         r <- r - alpha q and x <- x + alpha p with alpha = rho / pq (the
//         local solves applied the same fused multiply-add to r on the fly),
//         then r.z, r.r and, for flexible CG, z.q; the last block of a
//         system applies the convergence test and sets beta: rho'/rho (PCG)
//         or -(z.q)/(p.q) (flexible CG).
// ===========================================================================
// Basis row of `m` entries into registers; one 16-byte load per 16 bytes
// when the row is 16-byte aligned and m == MM.
template <typename TP, int MM>
__device__ __forceinline__ void load_basis_row(const TP* __restrict__ pr, int m, bool vec, TP (&v)[MM]) {
    constexpr int PER = 16 / sizeof(TP);
    if (MM % PER == 0 && vec) {
#pragma unroll
        for (int k = 0; k < MM; k += PER) {
            const uint4 u = __ldg(reinterpret_cast<const uint4*>(pr + k));
            const TP* t = reinterpret_cast<const TP*>(&u);
#pragma unroll
            for (int i = 0; i < PER; ++i) v[k + i] = t[i];
        }
    } else {
#pragma unroll
        for (int k = 0; k < MM; ++k) v[k] = (k < m) ? pr[k] : TP(0.f);
    }
}

template <typename TF, typename TP, int LD, int MM>
__global__ void __launch_bounds__(kRedThreads)
k_prolong_update(const SubInfo* __restrict__ subs, const TP* __restrict__ psi, const TF* __restrict__ ec,
                 const TF* __restrict__ yc, const TF* __restrict__ qmat, const CoarseRef* __restrict__ cref, const int32_t* __restrict__ gat,
                 const TF* __restrict__ zf, double* __restrict__ r, const double* __restrict__ q,
                 double* __restrict__ x, const double* __restrict__ p, TF* __restrict__ z, RedLayout R,
                 CgScalars* sc, SolveState* st, int nseg, int flexible, int mode) {
    using AT = typename Acc<TF>::type;
    using V4 = typename std::conditional<sizeof(TF) == 4, float4, double4>::type;
    constexpr int NCG = kRedThreads / LD;            // column groups of the backward product
    constexpr int NW = kRedThreads / 32;
    __shared__ double s_out[kRedMaxNV * kMaxLd];
    __shared__ double s_scr[kRedThreads];
    __shared__ AT s_ec[MM * LD];
    __shared__ AT s_part[NW * MM * LD];
    pdl_wait();
    if (st != nullptr && st->done) return;
    pdl_trigger();
    const int rhs = threadIdx.x % LD;
    const int cg = threadIdx.x / LD;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double alpha = 0.0;
    bool upd = false;
    if (mode == 2) {
        const CgScalars c = sc[(int64_t)R.blk_seg[blockIdx.x] * LD + rhs];
        upd = c.active != 0;
        if (upd) alpha = c.rho / c.pq;
    }
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t s_lo = R.blk_lo[blockIdx.x], s_hi = R.blk_lo[blockIdx.x + 1];
    for (int64_t si = s_lo; si < s_hi; ++si) {
        const SubInfo S = subs[si];
        const int m = S.m;
        const bool coarse = (ec != nullptr || qmat != nullptr) && m > 0;
        if (coarse && ec != nullptr) {
            // e_c computed by a separate backward-substitution launch
            for (int i = threadIdx.x; i < MM * LD; i += kRedThreads)
                s_ec[i] = (i < m * LD) ? (AT)ec[(int64_t)S.coff * LD + i] : AT(0);
        } else if (coarse) {
            // e_c rows of this subdomain: acc[k] = sum_j Q[k][j] y[gat[j]] over this thread's columns
            const CoarseRef cr = cref[si];
            const TF* Q = qmat + cr.q_off;
            const int32_t* G = gat + cr.gat_off;
            AT acc[MM];
#pragma unroll
            for (int k = 0; k < MM; ++k) acc[k] = AT(0);
            for (int c4 = cg; 4 * c4 < cr.K; c4 += NCG) {
                const int j0 = 4 * c4;
                AT yv[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    yv[e] = AT(0);
                    if (j0 + e < cr.K) {
                        const int gi = __ldg(G + j0 + e);
                        if (AMS_COARSE_OK(gi, 2)) yv[e] = (AT)yc[(int64_t)gi * LD + rhs];
                    }
                }
#pragma unroll
                for (int k = 0; k < MM; ++k) {
                    if (k < m) {
                        const V4 qv = *reinterpret_cast<const V4*>(Q + (int64_t)k * cr.ldm + j0);
                        acc[k] += (AT)qv.x * yv[0] + (AT)qv.y * yv[1] + (AT)qv.z * yv[2] + (AT)qv.w * yv[3];
                    }
                }
            }
            // sum over column groups: lanes of a warp with the same rhs, then warps in order
#pragma unroll
            for (int k = 0; k < MM; ++k) {
                AT a = acc[k];
                for (int off = 16; off >= LD; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
                if (lane < LD) s_part[(warp * MM + k) * LD + lane] = a;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < MM * LD; i += kRedThreads) {
                AT a = AT(0);
                for (int w = 0; w < NW; ++w) a += s_part[w * MM * LD + i];
                s_ec[i] = a;
            }
        }
        __syncthreads();
        const bool vec = (m == MM) && ((reinterpret_cast<uintptr_t>(psi + S.psi_off) & 15) == 0);
        const int64_t ne = (int64_t)S.n * LD;
        const int64_t g0 = S.row0 * LD;
#pragma unroll 4
        for (int64_t le = threadIdx.x; le < ne; le += kRedThreads) {
            const int64_t e = g0 + le;
            AT acc = (AT)zf[e];
            AT pe = AT(0);
            if (coarse) {
                TP pv[MM];
                load_basis_row<TP, MM>(psi + S.psi_off + (le / LD) * m, m, vec, pv);
#pragma unroll
                for (int k = 0; k < MM; ++k) pe += (AT)to_d(pv[k]) * s_ec[k * LD + rhs];
            }
            const AT zs = acc + pe;              // z in the apply precision, stored so
            const double zv = widen(zs);         // (FP32 widens exactly: the iterates do not change)
            z[e] = zs;
            if (mode != 0) {
                double rv = r[e];
                const double qv = (upd || (flexible && mode == 2)) ? q[e] : 0.0;
                if (upd) {
                    rv = fma(-alpha, qv, rv);
                    r[e] = rv;
                    // x += alpha p here, or (x == NULL, from 8 right-hand
                    // sides) in the next direction update, marked by xpend
                    if (x != nullptr) x[e] = fma(alpha, p[e], x[e]);
                }
                v[0] = fma(rv, zv, v[0]);
                v[1] = fma(rv, rv, v[1]);
                if (flexible && mode == 2) v[2] = fma(zv, qv, v[2]);
            }
        }
        __syncthreads();                 // s_ec / s_part are reused by the next subdomain
    }
    if (mode == 0) return;
    int sg;
    if (!seg_reduce<4>(v, LD, R, s_out, s_scr, sg)) return;
    const int it = st->it;
    if (threadIdx.x < LD) {
        CgScalars& c = sc[sg * LD + threadIdx.x];
        const double rz = s_out[threadIdx.x];
        const double rr = s_out[LD + threadIdx.x];
        const double zq = s_out[2 * LD + threadIdx.x];
        if (mode == 1) {
            c.rho = rz;
            c.beta = 0.0;
            c.zq = 0.0;
            if (c.active && !isfinite(rz)) {
                st->status = AMS_ERR_BREAKDOWN;
                st->done = 1;
            } else if (c.active && rr <= st->rtol2 * c.fnorm2) {   // x_0 already meets the target
                c.active = 0;
                c.rr = rr;
            } else if (c.active && !(rz > 0.0)) {   // r^T M^{-1} r <= 0: the preconditioner is not SPD
                st->status = AMS_ERR_BREAKDOWN;
                st->done = 1;
            }
        } else if (c.active) {
            c.alpha = c.rho / c.pq;
            c.xpend = 1;   // x += alpha p of this iteration: next direction update or the flush
            c.rr = rr;
            c.iters = it + 1;
            if (!isfinite(rr) || !isfinite(rz)) {
                st->status = AMS_ERR_BREAKDOWN;
                st->done = 1;
            } else if (rr <= st->rtol2 * c.fnorm2) {
                c.active = 0;
                c.beta = 0.0;
            } else if (!flexible && !(rz > 0.0)) {
                // r^T M^{-1} r <= 0 in exact-arithmetic PCG: M is not SPD (the
                // flexible variant, whose M^{-1} is applied in FP32, is only
                // checked on its first residual, in mode 1)
                st->status = AMS_ERR_BREAKDOWN;
                st->done = 1;
            } else {
                c.beta = flexible ? -zq / c.pq : rz / c.rho;
            }
            c.zq = zq;
            c.rho = rz;
        } else {
            c.xpend = 0;   // inactive this iteration: its update (if any) was applied
        }
    }
    if (mode != 2) return;
    if (!last_system(R, nseg)) return;
    if (threadIdx.x == 0) {
        int nact = 0;
        double worst = 0.0;
        for (int i = 0; i < nseg * LD; ++i) {
            nact += sc[i].active;
            if (sc[i].active) worst = fmax(worst, sc[i].rr / sc[i].fnorm2);
        }
        st->nactive = nact;
        st->worst = worst;
        st->it = it + 1;
        if (nact == 0 || it + 1 >= st->maxit) st->done = 1;
    }
}

// End of one body of the device-resident loop: count it and set the while
// node's condition.  The body cap bounds the loop even if no kernel ever
// reported convergence or the iteration cap.
__global__ void k_loop_cond(cudaGraphConditionalHandle h, SolveState* st, int cap) {
    const int b = ++st->bodies;
    cudaGraphSetConditional(h, (!st->done && b < cap) ? 1u : 0u);
}

void launch_loop_cond(cudaStream_t s, cudaGraphConditionalHandle h, SolveState* st, int cap) {
    k_loop_cond<<<1, 1, 0, s>>>(h, st, cap);
}

// ||f||^2 per (system, rhs) and CG scalar initialisation
template <int LD>
__global__ void __launch_bounds__(kRedThreads)
k_init_norms(const double* __restrict__ r, RedLayout R, CgScalars* sc, SolveState* st, int nseg,
             int nrhs) {
    __shared__ double s_out[kRedMaxNV * kMaxLd];
    __shared__ double s_scr[kRedThreads];
    double v[1] = {0.0};
    for (int64_t e = R.blk_lo[blockIdx.x] + threadIdx.x; e < R.blk_lo[blockIdx.x + 1]; e += kRedThreads)
        v[0] = fma(r[e], r[e], v[0]);
    int sg;
    if (!seg_reduce<1>(v, LD, R, s_out, s_scr, sg)) return;
    if (threadIdx.x < LD) {
        CgScalars& c = sc[sg * LD + threadIdx.x];
        c.fnorm2 = s_out[threadIdx.x];
        c.rr = c.fnorm2;
        c.rho = 0.0;
        c.pq = 0.0;
        c.zq = 0.0;
        c.alpha = 0.0;
        c.beta = 0.0;
        c.iters = 0;
        c.xpend = 0;
        c.active = (threadIdx.x < nrhs && c.fnorm2 > 0.0) ? 1 : 0;
    }
    if (!last_system(R, nseg)) return;
    if (threadIdx.x == 0) {
        int nact = 0;
        for (int i = 0; i < nseg * LD; ++i) nact += sc[i].active;
        st->nactive = nact;
        st->it = 0;
        st->xdone_it = 0;
        st->status = 0;
        st->worst = 1.0;
        st->done = (nact == 0);
    }
}

// caller order (col-major n x nrhs) <-> internal node-major rows
__global__ void k_permute_in(const double* __restrict__ f, int64_t n, int nrhs, int ld,
                             const int64_t* __restrict__ int_row, double* __restrict__ r,
                             double scale_zero_x, double* __restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t row = int_row[i];
    if (!AMS_ROW_OK(row, 6)) return;
    for (int k = 0; k < ld; ++k) {
        r[row * ld + k] = k < nrhs ? f[i + (int64_t)k * n] : 0.0;
        if (x != nullptr) x[row * ld + k] = 0.0;
    }
}

template <typename XT>
__global__ void k_permute_out(const XT* __restrict__ x, int64_t n, int nrhs, int ld,
                              const int64_t* __restrict__ int_row, double* __restrict__ u) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t row = int_row[i];
    if (!AMS_ROW_OK(row, 6)) return;
    for (int k = 0; k < nrhs; ++k) u[i + (int64_t)k * n] = widen(x[row * ld + k]);
}

// u += u0 (caller order) for the right-hand sides with f != 0 (a warm
// start solves A e = f - A u0 from e = 0; a zero right-hand side keeps u = 0)
__global__ void k_add_initial_guess(double* __restrict__ u, const double* __restrict__ u0, int64_t n, int nrhs,
                                    const CgScalars* __restrict__ sc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < nrhs; ++k)
        if (sc[k].fnorm2 > 0.0) u[i + (int64_t)k * n] += u0[i + (int64_t)k * n];
}

void launch_add_initial_guess(cudaStream_t s, double* u, const double* u0, int64_t n, int nrhs,
                              const CgScalars* sc) {
    if (n > 0) k_add_initial_guess<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(u, u0, n, nrhs, sc);
}

// a8: dvals[e] = - sum_k lambda_k[row_e] u_k[col_e]  (caller CSR order)
__global__ void k_sddmm(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                        int64_t n, int nrhs, const double* __restrict__ lam,
                        const double* __restrict__ u, double* __restrict__ dvals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int64_t j = colind[e];
        double s = 0.0;
        for (int k = 0; k < nrhs; ++k) s += lam[i + (int64_t)k * n] * u[j + (int64_t)k * n];
        dvals[e] = -s;
    }
}

// sell_val[pos[e]] = vals[e] (caller CSR entry e -> SELL slot)
__global__ void k_scatter_vals(const double* __restrict__ vals, const int64_t* __restrict__ pos, int64_t nnz,
                               double* __restrict__ sell_val) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nnz) sell_val[pos[e]] = vals[e];
}

__global__ void k_zero(double* __restrict__ a, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = 0.0;
}

// ===========================================================================
// host launchers
// ===========================================================================
#define AMS_DISPATCH_LD(ld, F, ...)                     \
    switch (ld) {                                        \
        case 1: F<1>(__VA_ARGS__); break;                \
        case 2: F<2>(__VA_ARGS__); break;                \
        case 4: F<4>(__VA_ARGS__); break;                \
        case 8: F<8>(__VA_ARGS__); break;                \
        case 16: F<16>(__VA_ARGS__); break;              \
        default: F<32>(__VA_ARGS__); break;              \
    }

template <int LD>
static void spmv_ld(const LaunchCtx& L, const double* p, double* q, int with_dot) {
    launch_kernel(L.pdl, k_spmv_dot<LD, 8>, dim3((unsigned)L.nblk), dim3(kRedThreads), 0, L.stream, L.sell_ptr,
                  L.sell_col, L.sell_val, p, q, L.red, L.sc, with_dot ? L.st : nullptr, with_dot);
}
void launch_spmv_dot(const LaunchCtx& L, const double* p, double* q, int with_dot) {
    AMS_DISPATCH_LD(L.ld, spmv_ld, L, p, q, with_dot);
}

template <int LD>
static void dir_ld(const LaunchCtx& L, int prec, const void* z, const double* p_old, double* p_new, double* x) {
    const dim3 g((unsigned)L.nblk), b(kRedThreads);
    const CgScalars* sc = (const CgScalars*)L.sc;
    if (prec == AMS_PREC_FP64) {
        const double* zd = (const double*)z;
        if (x != nullptr)
            launch_kernel(L.pdl, k_dir_update<LD, double, true>, g, b, 0, L.stream, zd, p_old, p_new, x, L.red, sc, L.st);
        else
            launch_kernel(L.pdl, k_dir_update<LD, double, false>, g, b, 0, L.stream, zd, p_old, p_new, x, L.red, sc, L.st);
    } else {
        const float* zf = (const float*)z;
        if (x != nullptr)
            launch_kernel(L.pdl, k_dir_update<LD, float, true>, g, b, 0, L.stream, zf, p_old, p_new, x, L.red, sc, L.st);
        else
            launch_kernel(L.pdl, k_dir_update<LD, float, false>, g, b, 0, L.stream, zf, p_old, p_new, x, L.red, sc, L.st);
    }
}
void launch_dir_update(const LaunchCtx& L, int prec, const void* z, const double* p_old, double* p_new, double* x) {
    AMS_DISPATCH_LD(L.ld, dir_ld, L, prec, z, p_old, p_new, x);
}
template <int LD>
static void flush_ld(const LaunchCtx& L, const double* p, const double* p2, double* x) {
    k_x_flush<LD><<<(unsigned)L.nblk, kRedThreads, 0, L.stream>>>(p, p2, x, L.red, (const CgScalars*)L.sc,
                                                               (const SolveState*)L.st);
}
void launch_x_flush(const LaunchCtx& L, const double* p, const double* p2, double* x) {
    AMS_DISPATCH_LD(L.ld, flush_ld, L, p, p2, x);
}

template <int LD>
static void norms_ld(const LaunchCtx& L, const double* r, int nrhs) {
    k_init_norms<LD><<<L.nblk, kRedThreads, 0, L.stream>>>(r, L.red, L.sc, L.st, L.nseg, nrhs);
}
void launch_init_norms(const LaunchCtx& L, const double* r, int nrhs) {
    AMS_DISPATCH_LD(L.ld, norms_ld, L, r, nrhs);
}

size_t local_solve_smem(int cmax, int ld, size_t tf_bytes, int depth) {
    return ((size_t)(cmax + depth + 1) * blockrow_elems(cmax) + (size_t)(cmax + 1) * 32 * ld + 32 * ld) *
           tf_bytes;
}

// Deepest prefetch (<= 6 block rows) whose staging fits a shared-memory
// budget that still leaves room for several resident blocks per SM.
int local_solve_depth(int cmax, int ld, size_t tf_bytes) {
    const size_t budget = 100 * 1024, hard = 200 * 1024;
    int d = 4;
    while (d > 1 && local_solve_smem(cmax, ld, tf_bytes, d) > budget) --d;
    while (d > 1 && local_solve_smem(cmax, ld, tf_bytes, d) > hard) --d;
    return d;
}

template <typename TF, typename TP, int NR, int MM>
static cudaError_t local_nr(const LocalSolveArgs& a, const void* fac, const void* psi, void* zf,
                            void* rc) {
    const int warps = a.ld / NR;
    const int depth = a.depth > 0 ? a.depth : local_solve_depth(a.cmax, a.ld, sizeof(TF));
    const size_t smem = local_solve_smem(a.cmax, a.ld, sizeof(TF), depth);
    auto kern = k_local_solve<TF, TP, NR, MM>;
    static size_t smem_set = 0;           // per template instance
    if (smem > smem_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        smem_set = smem;
    }
    return launch_kernel(a.pdl, kern, dim3(a.nsub), dim3(warps * 32), smem, a.stream, a.subs, (const TF*)fac, a.in.r,
                         a.in.q, a.in.sc, a.rowscale, (TF*)zf, (const TP*)psi, (TF*)rc, a.ld, a.cmax, depth, a.st);
}

template <typename TF, typename TP>
static cudaError_t local_tp(const LocalSolveArgs& a, const void* fac, const void* psi, void* zf, void* rc) {
    const bool big = a.mmax > 8;
    const int nrmax = sizeof(TF) == 8 ? (big ? 2 : 4) : (big ? 4 : 8);
    const int nr = a.ld < nrmax ? a.ld : nrmax;
    if (big) {
        switch (nr) {
            case 1: return local_nr<TF, TP, 1, 16>(a, fac, psi, zf, rc);
            case 2: return local_nr<TF, TP, 2, 16>(a, fac, psi, zf, rc);
            default: return local_nr<TF, TP, 4, 16>(a, fac, psi, zf, rc);
        }
    }
    switch (nr) {
        case 1: return local_nr<TF, TP, 1, 8>(a, fac, psi, zf, rc);
        case 2: return local_nr<TF, TP, 2, 8>(a, fac, psi, zf, rc);
        case 4: return local_nr<TF, TP, 4, 8>(a, fac, psi, zf, rc);
        default: return local_nr<TF, TP, 8, 8>(a, fac, psi, zf, rc);
    }
}

cudaError_t launch_local_solve(const LocalSolveArgs& a, int prec, const void* fac, const void* psi,
                               void* zf, void* rc) {
    if (prec == AMS_PREC_FP64) return local_tp<double, double>(a, fac, psi, zf, rc);
    if (prec == AMS_PREC_FP32) return local_tp<float, float>(a, fac, psi, zf, rc);
    return local_tp<float, __nv_bfloat16>(a, fac, psi, zf, rc);
}

template <typename TF, typename TP, int LD>
static void prolong_ld(const LaunchCtx& L, const ProlongArgs& a) {
    if (L.nsub == 0) return;
    auto kern = a.mmax > 8 ? k_prolong_update<TF, TP, LD, kMaxM> : k_prolong_update<TF, TP, LD, 8>;
    launch_kernel(L.pdl, kern, dim3((unsigned)L.nblk_sub), dim3(kRedThreads), 0, L.stream, L.subs, (const TP*)a.psi,
                  (const TF*)a.ec, (const TF*)a.yc, (const TF*)a.qmat, a.cref, a.gat, (const TF*)a.zf, a.r, a.q, a.x, a.p,
                  (TF*)a.z,
                  L.red_sub, L.sc, L.st, L.nseg, a.flexible, a.mode);
}
template <typename TF, typename TP>
static void prolong_tp(const LaunchCtx& L, const ProlongArgs& a) {
    switch (L.ld) {
        case 1: prolong_ld<TF, TP, 1>(L, a); break;
        case 2: prolong_ld<TF, TP, 2>(L, a); break;
        case 4: prolong_ld<TF, TP, 4>(L, a); break;
        case 8: prolong_ld<TF, TP, 8>(L, a); break;
        case 16: prolong_ld<TF, TP, 16>(L, a); break;
        default: prolong_ld<TF, TP, 32>(L, a); break;
    }
}
void launch_prolong_update(const LaunchCtx& L, int prec, const ProlongArgs& a) {
    if (prec == AMS_PREC_FP64) prolong_tp<double, double>(L, a);
    else if (prec == AMS_PREC_FP32) prolong_tp<float, float>(L, a);
    else prolong_tp<float, __nv_bfloat16>(L, a);
}

void launch_permute_in(cudaStream_t s, const double* f, int64_t n, int nrhs, int ld,
                       const int64_t* int_row, double* r, double* x) {
    k_permute_in<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f, n, nrhs, ld, int_row, r, 0.0, x);
}
void launch_permute_out(cudaStream_t s, const double* x, int64_t n, int nrhs, int ld,
                        const int64_t* int_row, double* u) {
    k_permute_out<double><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, nrhs, ld, int_row, u);
}
void launch_permute_out_f32(cudaStream_t s, const float* x, int64_t n, int nrhs, int ld,
                            const int64_t* int_row, double* u) {
    k_permute_out<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, nrhs, ld, int_row, u);
}
void launch_sddmm(cudaStream_t s, const int64_t* rowptr, const int32_t* colind, int64_t n, int nrhs,
                  const double* lam, const double* u, double* dvals) {
    k_sddmm<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(rowptr, colind, n, nrhs, lam, u, dvals);
}
void launch_scatter_vals(cudaStream_t s, const double* vals, const int64_t* pos, int64_t nnz, double* sell_val) {
    if (nnz > 0) k_scatter_vals<<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(vals, pos, nnz, sell_val);
}
void launch_zero(cudaStream_t s, double* a, int64_t n) {
    if (n > 0) k_zero<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, n);
}

// ---------------------------------------------------------------------------
// checking-build hooks and self-test (see kernels.cuh)
// ---------------------------------------------------------------------------
AMS_DEBUG_TU_HOOKS(solve)

__global__ void k_debug_selftest() { (void)AMS_ROW_OK(-1, 99); }
void launch_debug_selftest(cudaStream_t s) { k_debug_selftest<<<1, 1, 0, s>>>(); }

}  // namespace ams
