// Local solves for 8 to 32 right-hand sides on the tensor cores (Section 3.2:
// z_f = sum_i R_i^T A_i^{-1} R_i r' with A_i = L_i L_i^T, and the restriction
// r_c = R_0 r' of the coarse correction, Section 3.1, fused in).
//
// With many right-hand sides every step of the block-row triangular solves
// is a dense product of 32x32 factor tiles with 32-row blocks of 8-32
// columns: t = r'_K - sum_d L_{K,K-c+d} Y_{K-c+d}, then Y_K = L_KK^{-1} t
// (forward), and the transposed products backward.  These products run as
// warp-level tensor-core MMAs (m16n8k8, TF32 operands, FP32 accumulation).
// Each FP32 operand is split into a TF32 head and a TF32 tail and the
// product is summed as head*head + head*tail + tail*head, which keeps the
// apply at FP32 accuracy (the dropped tail*tail term is below FP32
// rounding); BF16 basis entries are exact in TF32 and are not split.
//
// Why warp-level MMAs rather than tcgen05: one subdomain's solve is a
// chain of dependent 32-row steps, and tcgen05.mma needs M >= 64 rows per
// instruction from shared memory; stacking independent subdomains into M
// would need their tiles laid out block-diagonally with zero blocks, four
// times the shared memory of the tiles themselves (FP32, twice that with
// the head/tail split), which leaves no room for the copy ring.  The m16n8k8
// fragments come straight from the 4 KB tiles the TMA already stages.
//
// Layout and staging are those of the TMA local solve (k_local_tma.cu):
// forward tiles only, block row K = [ M_K | L_{K,K-c+1} | .. | L_{K,K-1} ],
// M_K[r][q] = L_{K,K-c}[r][q] (q >= r) and (L_KK^{-1})[r][q] (q < r),
// reciprocal pivots per row, 128-byte swizzled 32x32 FP32 tiles in a ring
// of nbuf = cmax + depth + 1 slots with bounded mbarrier waits.  The
// backward sweep reads the same tiles transposed.  Warp w of a block owns
// columns [8 NF w, 8 NF (w+1)) of the subdomain's right-hand sides.
#include <algorithm>
#include <cstdint>

#include <cuda.h>

#include "ams_internal.h"
#include "kernels.cuh"
#include "launch.h"
#include "mma_tf32.cuh"
#include "tma.cuh"

namespace ams {

// Element (r, q) of a 128-byte swizzled 32x32 FP32 tile.
__device__ __forceinline__ float tl(const float* T, int r, int q) {
    return T[r * 32 + ((((q >> 2) ^ r) & 7) << 2) + (q & 3)];
}

// Row stride (floats) of the right-hand-side blocks in shared memory: a
// multiple of 8 words plus 8 (mod 32), so that the B-fragment loads (rows
// t..t+3, columns g..g+7) hit 32 distinct banks.
__host__ __device__ __forceinline__ int mma_row_stride(int ld) { return ld >= 16 ? ld + 8 : 24; }

// Element masks of a tile operand, in the tile's own (r, q) coordinates:
// 0 all, 1 keep q >= r (upper part of M: L_{K,K-c}), 2 keep q < r (strict
// lower part: L_KK^{-1} without its diagonal).  TR: the operand is the
// transposed tile, A(m, k) = T(k, m).
template <int MODE, bool TR>
__device__ __forceinline__ constexpr bool frag_is_zero(int mf, int ks) {
    // rows (m) 16 mf .. 16 mf + 15, columns (k) 8 ks .. 8 ks + 7 of A
    return TR ? (MODE == 1 ? (16 * mf + 15 < 8 * ks) : MODE == 2 ? (16 * mf >= 8 * ks + 7) : false)
              : (MODE == 1 ? (8 * ks + 7 < 16 * mf) : MODE == 2 ? (8 * ks >= 16 * mf + 15) : false);
}

template <int MODE, bool TR>
__device__ __forceinline__ void load_afrag(const float* T, int mf, int ks, int g, int t, float (&a)[4]) {
    const int m0 = 16 * mf + g, m1 = m0 + 8, k0 = 8 * ks + t, k1 = k0 + 4;
    // fragment order: (m0,k0) (m1,k0) (m0,k1) (m1,k1); tile element T(r, q)
    const int r[4] = {TR ? k0 : m0, TR ? k0 : m1, TR ? k1 : m0, TR ? k1 : m1};
    const int q[4] = {TR ? m0 : k0, TR ? m1 : k0, TR ? m0 : k1, TR ? m1 : k1};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        a[i] = tl(T, r[i], q[i]);
        if (MODE == 1 && q[i] < r[i]) a[i] = 0.f;
        if (MODE == 2 && q[i] >= r[i]) a[i] = 0.f;
    }
}

// acc[mf][nf] += A * B for a 32x32 tile operand A (mask MODE, transposed
// when TR) and the 32-row block B (row stride SY, this warp's columns cb..).
template <int MODE, bool TR, int NF>
__device__ __forceinline__ void tile_mma(const float* T, const float* B, int SY, int cb, int g, int t,
                                         float (&acc)[2][NF][4]) {
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        uint32_t bh[NF][2], bl[NF][2];
#pragma unroll
        for (int nf = 0; nf < NF; ++nf) {
            const float* bp = B + (8 * ks + t) * SY + cb + 8 * nf + g;
            split_tf32(bp[0], bh[nf][0], bl[nf][0]);
            split_tf32(bp[4 * SY], bh[nf][1], bl[nf][1]);
        }
#pragma unroll
        for (int mf = 0; mf < 2; ++mf) {
            if (frag_is_zero<MODE, TR>(mf, ks)) continue;
            float a[4];
            load_afrag<MODE, TR>(T, mf, ks, g, t, a);
            uint32_t ah[4], al[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) split_tf32(a[i], ah[i], al[i]);
#pragma unroll
            for (int nf = 0; nf < NF; ++nf) {
                mma_tf32(acc[mf][nf], al, bh[nf][0], bh[nf][1]);
                mma_tf32(acc[mf][nf], ah, bl[nf][0], bl[nf][1]);
                mma_tf32(acc[mf][nf], ah, bh[nf][0], bh[nf][1]);
            }
        }
    }
}

template <int NF>
__device__ __forceinline__ void zero_acc(float (&acc)[2][NF][4]) {
#pragma unroll
    for (int mf = 0; mf < 2; ++mf)
#pragma unroll
        for (int nf = 0; nf < NF; ++nf)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[mf][nf][i] = 0.f;
}

// Accumulator element i of fragment (mf, nf): row 16 mf + g + 8 (i >> 1),
// column cb + 8 nf + 2 t + (i & 1).
template <typename TP, int NF, int MM>
__global__ void __launch_bounds__(128)
k_local_mma(const __grid_constant__ CUtensorMap tmF, const SubInfo* __restrict__ subs,
            const int64_t* __restrict__ tile_row0, const float* __restrict__ piv, const double* __restrict__ rin,
            const double* __restrict__ qin, const CgScalars* __restrict__ csc, float* __restrict__ zf,
            const TP* __restrict__ psi, float* __restrict__ rc, int ld, int cmax, int depth, int64_t budget,
            SolveState* st, int32_t* err, int probe, const int32_t* __restrict__ order) {
    static_assert(MM == 8 || MM == 16, "basis blocks of up to 8 or 16 modes");
    pdl_wait();
    if (st != nullptr && st->done) return;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_align1024(smem_raw);
    const int sid = order != nullptr ? order[blockIdx.x] : (int)blockIdx.x;
    const SubInfo S = subs[sid];
    if (!AMS_ROW_OK(S.row0, 4) || !AMS_ROW_OK(S.row0 + S.n - 1, 4)) return;
    const int c = S.c, nb = S.nb, n = S.n, m = S.m;
    const int D = depth;
    const int nbuf = cmax + D + 1;
    const int SY = mma_row_stride(ld);
    float* tiles = (float*)base;                                        // nbuf * cmax * 1024
    uint64_t* bars = (uint64_t*)(tiles + (size_t)nbuf * cmax * 1024);    // ring_bar_slots(nbuf)
    float* ring = (float*)(bars + ring_bar_slots(nbuf));                 // (cmax + 1) * 32 * SY: y, then x
    float* tmp = ring + (size_t)(cmax + 1) * 32 * SY;                    // 32 * SY
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int cb = warp * 8 * NF;
    const int64_t trow = tile_row0[sid];
    const uint32_t tile_bytes = 4096u * (uint32_t)c;
    uint32_t phase = 0, pend = 0;    // as in k_local_tma: change only when a wait succeeds
    bool ok = true;

    if (threadIdx.x == 0) {
        for (int i = 0; i <= nbuf; ++i) mbar_init(smem_u32(bars + i), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int K) {
        const int slot = K % nbuf;
        if (threadIdx.x == 0) {
            const uint32_t bar = smem_u32(bars + slot);
            mbar_expect_tx(bar, tile_bytes);
            for (int d = 0; d < c; ++d)
                tma_load_2d(smem_u32(tiles + ((size_t)slot * cmax + d) * 1024), &tmF, 0,
                            (int32_t)(trow + ((int64_t)K * c + d) * 32), bar);
        }
        pend |= 1u << slot;
    };
    auto wait_slot = [&](int K) {
        const int slot = K % nbuf;
        if (!mbar_wait(smem_u32(bars + slot), (phase >> slot) & 1u, budget)) {
            ok = false;
            return;
        }
        phase ^= 1u << slot;
        pend &= ~(1u << slot);
    };
    auto slot_tile = [&](int K, int d) -> const float* { return tiles + ((size_t)(K % nbuf) * cmax + d) * 1024; };

    // r' = r - alpha q for this lane's columns of (system, rhs) pairs still iterating
    double al[NF][2];
    bool up[NF][2];
#pragma unroll
    for (int nf = 0; nf < NF; ++nf)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            al[nf][j] = 0.0;
            up[nf][j] = false;
            if (qin != nullptr) {
                const CgScalars cs = csc[(int64_t)S.seg * ld + cb + 8 * nf + 2 * t + j];
                up[nf][j] = cs.active != 0;
                if (up[nf][j]) al[nf][j] = cs.rho / cs.pq;
            }
        }
    float racc[NF][4];   // restriction: rows = modes g, g + 8; columns as the accumulators
#pragma unroll
    for (int nf = 0; nf < NF; ++nf)
#pragma unroll
        for (int i = 0; i < 4; ++i) racc[nf][i] = 0.f;

    // Inputs of the next block row (r and q in FP64, the basis rows of the
    // restriction) are loaded into registers while the current one is
    // computed, so their latency overlaps a whole step.
    double2 rraw[2][2][NF], qraw[2][2][NF];
    constexpr int HM = MM > 8 ? 2 : 1;   // modes g (and g + 8) per lane
    TP praw[4][2][HM];
    auto load_inputs = [&](int K) {
#pragma unroll
        for (int mf = 0; mf < 2; ++mf)
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int row = K * 32 + 16 * mf + g + 8 * h2;
                const bool valid = K < nb && row < n;
                const int64_t grow = S.row0 + row;
#pragma unroll
                for (int nf = 0; nf < NF; ++nf) {
                    const int col = cb + 8 * nf + 2 * t;
                    rraw[mf][h2][nf] = make_double2(0.0, 0.0);
                    qraw[mf][h2][nf] = make_double2(0.0, 0.0);
                    if (valid) {
                        rraw[mf][h2][nf] = *reinterpret_cast<const double2*>(rin + grow * ld + col);
                        if (up[nf][0] || up[nf][1])
                            qraw[mf][h2][nf] = *reinterpret_cast<const double2*>(qin + grow * ld + col);
                    }
                }
            }
    };
    auto load_psi = [&](int K) {
        if (rc != nullptr) {
            // A fragments of Psi_K^T: rows 8 ks + t (+4) of block row K, modes g (and g + 8)
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    const int row = K * 32 + 8 * ks + t + 4 * kk;
                    const TP* pr = psi + S.psi_off + (int64_t)row * m;
#pragma unroll
                    for (int hm = 0; hm < HM; ++hm) {
                        praw[ks][kk][hm] = TP(0.f);
                        if (K < nb && row < n && g + 8 * hm < m) praw[ks][kk][hm] = pr[g + 8 * hm];
                    }
                }
        }
    };
    // ---------------- forward ----------------
    for (int j = 0; j < D && j < nb; ++j) issue(j);
    if (probe) {   // timeout test hook: a bounded wait on a barrier nothing completes
        if (!mbar_wait(smem_u32(bars + nbuf), 0u, budget)) ok = false;
        ok = __syncthreads_and(ok);
    }
    load_inputs(0);
    load_psi(0);
#pragma unroll 1
    for (int K = 0; K < nb && ok; ++K) {
        if (K + D < nb) issue(K + D);
        float rp[2][NF][4];
#pragma unroll
        for (int mf = 0; mf < 2; ++mf)
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2)
#pragma unroll
                for (int nf = 0; nf < NF; ++nf) {
                    const double2 rv = rraw[mf][h2][nf], qv = qraw[mf][h2][nf];
                    rp[mf][nf][2 * h2] = f64_to_f32(up[nf][0] ? fma(-al[nf][0], qv.x, rv.x) : rv.x);
                    rp[mf][nf][2 * h2 + 1] = f64_to_f32(up[nf][1] ? fma(-al[nf][1], qv.y, rv.y) : rv.y);
                }
        load_inputs(K + 1);
        wait_slot(K);
        ok = __syncthreads_and(ok);
        if (!ok) break;
        if (rc != nullptr) {
            // r_c += Psi_K^T r'_K: r' through shared memory into B fragments
#pragma unroll
            for (int mf = 0; mf < 2; ++mf)
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2)
#pragma unroll
                    for (int nf = 0; nf < NF; ++nf)
                        *reinterpret_cast<float2*>(tmp + (16 * mf + g + 8 * h2) * SY + cb + 8 * nf + 2 * t) =
                            make_float2(rp[mf][nf][2 * h2], rp[mf][nf][2 * h2 + 1]);
            __syncwarp();
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                // A = Psi_K^T: A(mode, row) for rows 8 ks + t (+4) of block row K
                float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int kk = 0; kk < 2; ++kk)
#pragma unroll
                    for (int hm = 0; hm < HM; ++hm) a[2 * kk + hm] = to_f(praw[ks][kk][hm]);
                uint32_t ah[4], alo[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) split_tf32(a[i], ah[i], alo[i]);
#pragma unroll
                for (int nf = 0; nf < NF; ++nf) {
                    const float* bp = tmp + (8 * ks + t) * SY + cb + 8 * nf + g;
                    uint32_t b0h, b0l, b1h, b1l;
                    split_tf32(bp[0], b0h, b0l);
                    split_tf32(bp[4 * SY], b1h, b1l);
                    if (sizeof(TP) != 2) mma_tf32(racc[nf], alo, b0h, b1h);   // BF16 entries are exact in TF32
                    mma_tf32(racc[nf], ah, b0l, b1l);
                    mma_tf32(racc[nf], ah, b0h, b1h);
                }
            }
            __syncwarp();
        }
        load_psi(K + 1);   // the basis rows of step K are used: fetch those of K + 1
        // t = r'_K - sum_d L_{K,K-c+d} y_{K-c+d}
        float acc[2][NF][4];
        zero_acc<NF>(acc);
        if (c == 2 && K >= 2) {
            // both band tiles present: separate accumulators, so that the two
            // tiles' MMA chains are independent and interleave
            float acc1[2][NF][4];
            zero_acc<NF>(acc1);
            tile_mma<1, false, NF>(slot_tile(K, 0), ring + (size_t)((K - 2) % 3) * 32 * SY, SY, cb, g, t, acc);
            tile_mma<0, false, NF>(slot_tile(K, 1), ring + (size_t)((K - 1) % 3) * 32 * SY, SY, cb, g, t, acc1);
#pragma unroll
            for (int mf = 0; mf < 2; ++mf)
#pragma unroll
                for (int nf = 0; nf < NF; ++nf)
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[mf][nf][i] += acc1[mf][nf][i];
        } else {
            for (int d = 0; d < c; ++d) {
                const int src = K - c + d;
                if (src < 0) continue;
                const float* Y = ring + (size_t)(src % (c + 1)) * 32 * SY;
                if (d == 0) tile_mma<1, false, NF>(slot_tile(K, 0), Y, SY, cb, g, t, acc);
                else tile_mma<0, false, NF>(slot_tile(K, d), Y, SY, cb, g, t, acc);
            }
        }
#pragma unroll
        for (int mf = 0; mf < 2; ++mf)
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2)
#pragma unroll
                for (int nf = 0; nf < NF; ++nf) {
                    rp[mf][nf][2 * h2] -= acc[mf][nf][2 * h2];
                    rp[mf][nf][2 * h2 + 1] -= acc[mf][nf][2 * h2 + 1];
                    *reinterpret_cast<float2*>(tmp + (16 * mf + g + 8 * h2) * SY + cb + 8 * nf + 2 * t) =
                        make_float2(rp[mf][nf][2 * h2], rp[mf][nf][2 * h2 + 1]);
                }
        __syncwarp();
        // y_K = L_KK^{-1} t = pivot t + (strict lower part of M_K) t
        zero_acc<NF>(acc);
        tile_mma<2, false, NF>(slot_tile(K, 0), tmp, SY, cb, g, t, acc);
        float* Yk = ring + (size_t)(K % (c + 1)) * 32 * SY;
#pragma unroll
        for (int mf = 0; mf < 2; ++mf)
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int r = 16 * mf + g + 8 * h2;
                const int row = K * 32 + r;
                const float pv = row < n ? piv[S.row0 + row] : 1.f;
#pragma unroll
                for (int nf = 0; nf < NF; ++nf) {
                    const float2 y = make_float2(fmaf(pv, rp[mf][nf][2 * h2], acc[mf][nf][2 * h2]),
                                                 fmaf(pv, rp[mf][nf][2 * h2 + 1], acc[mf][nf][2 * h2 + 1]));
                    *reinterpret_cast<float2*>(Yk + r * SY + cb + 8 * nf + 2 * t) = y;
                    if (row < n) *reinterpret_cast<float2*>(zf + (S.row0 + row) * ld + cb + 8 * nf + 2 * t) = y;
                }
            }
        __syncthreads();
    }
    if (rc != nullptr && ok) {
#pragma unroll
        for (int nf = 0; nf < NF; ++nf)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int mode = g + 8 * (i >> 1);
                if (mode < m) rc[(S.coff + mode) * ld + cb + 8 * nf + 2 * t + (i & 1)] = racc[nf][i];
            }
    }
    pdl_trigger();

    // ---------------- backward ----------------
    if (ok)
        for (int j = 0; j < D && nb - 1 - j >= 0; ++j) issue(nb - 1 - j);
    // y of the next block row (written by this lane in the forward sweep)
    // is loaded while the current one is computed
    float2 yraw[2][2][NF];
    auto load_y = [&](int K) {
#pragma unroll
        for (int mf = 0; mf < 2; ++mf)
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int row = K * 32 + 16 * mf + g + 8 * h2;
#pragma unroll
                for (int nf = 0; nf < NF; ++nf) {
                    yraw[mf][h2][nf] = make_float2(0.f, 0.f);
                    if (K >= 0 && row < n)
                        yraw[mf][h2][nf] =
                            *reinterpret_cast<const float2*>(zf + (S.row0 + row) * ld + cb + 8 * nf + 2 * t);
                }
            }
    };
    if (ok) load_y(nb - 1);
#pragma unroll 1
    for (int K = nb - 1; K >= 0 && ok; --K) {
        if (K - D >= 0) issue(K - D);
        float w[2][NF][4];
#pragma unroll
        for (int mf = 0; mf < 2; ++mf)
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2)
#pragma unroll
                for (int nf = 0; nf < NF; ++nf) {
                    w[mf][nf][2 * h2] = yraw[mf][h2][nf].x;
                    w[mf][nf][2 * h2 + 1] = yraw[mf][h2][nf].y;
                }
        load_y(K - 1);
        wait_slot(K);
        ok = __syncthreads_and(ok);
        if (!ok) break;
        // w = y_K - sum_d L_{K+d,K}^T x_{K+d}
        float acc[2][NF][4];
        zero_acc<NF>(acc);
        if (c == 2 && K + 2 < nb) {
            // both transposed band tiles present: independent accumulators (as forward)
            float acc1[2][NF][4];
            zero_acc<NF>(acc1);
            tile_mma<0, true, NF>(slot_tile(K + 1, 1), ring + (size_t)((K + 1) % 3) * 32 * SY, SY, cb, g, t, acc);
            tile_mma<1, true, NF>(slot_tile(K + 2, 0), ring + (size_t)((K + 2) % 3) * 32 * SY, SY, cb, g, t, acc1);
#pragma unroll
            for (int mf = 0; mf < 2; ++mf)
#pragma unroll
                for (int nf = 0; nf < NF; ++nf)
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[mf][nf][i] += acc1[mf][nf][i];
        } else {
            for (int d = 1; d <= c; ++d) {
                const int src = K + d;
                if (src >= nb) break;
                const float* X = ring + (size_t)(src % (c + 1)) * 32 * SY;
                // L_{K+d,K}: dense tile c-d of block row K+d, or (d == c) the upper part of M_{K+c}
                if (d < c) tile_mma<0, true, NF>(slot_tile(src, c - d), X, SY, cb, g, t, acc);
                else tile_mma<1, true, NF>(slot_tile(src, 0), X, SY, cb, g, t, acc);
            }
        }
#pragma unroll
        for (int mf = 0; mf < 2; ++mf)
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2)
#pragma unroll
                for (int nf = 0; nf < NF; ++nf) {
                    w[mf][nf][2 * h2] -= acc[mf][nf][2 * h2];
                    w[mf][nf][2 * h2 + 1] -= acc[mf][nf][2 * h2 + 1];
                    *reinterpret_cast<float2*>(tmp + (16 * mf + g + 8 * h2) * SY + cb + 8 * nf + 2 * t) =
                        make_float2(w[mf][nf][2 * h2], w[mf][nf][2 * h2 + 1]);
                }
        __syncwarp();
        // x_K = L_KK^{-T} w = pivot w + (strict lower part of M_K)^T w
        zero_acc<NF>(acc);
        tile_mma<2, true, NF>(slot_tile(K, 0), tmp, SY, cb, g, t, acc);
        float* Xk = ring + (size_t)(K % (c + 1)) * 32 * SY;
#pragma unroll
        for (int mf = 0; mf < 2; ++mf)
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int r = 16 * mf + g + 8 * h2;
                const int row = K * 32 + r;
                const float pv = row < n ? piv[S.row0 + row] : 1.f;
#pragma unroll
                for (int nf = 0; nf < NF; ++nf) {
                    const float2 x = make_float2(fmaf(pv, w[mf][nf][2 * h2], acc[mf][nf][2 * h2]),
                                                 fmaf(pv, w[mf][nf][2 * h2 + 1], acc[mf][nf][2 * h2 + 1]));
                    *reinterpret_cast<float2*>(Xk + r * SY + cb + 8 * nf + 2 * t) = x;
                    if (row < n) *reinterpret_cast<float2*>(zf + (S.row0 + row) * ld + cb + 8 * nf + 2 * t) = x;
                }
            }
        __syncthreads();
    }
    if (!ok) timeout_drain(bars, nbuf, pend, phase, err, st, threadIdx.x == 0);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t local_mma_smem(int cmax, int ld, int depth) {
    const int nbuf = cmax + depth + 1;
    const int SY = mma_row_stride(ld);
    return 1024 /* alignment slack */ + (size_t)nbuf * cmax * 4096 + (size_t)ring_bar_slots(nbuf) * 8 +
           ((size_t)(cmax + 1) * 32 * SY + 32 * SY) * sizeof(float);
}

// Default ring depth: the deepest (at most 4) whose staging stays within
// 64 KB, so that three or more blocks fit on an SM.
static int local_mma_depth(int cmax, int ld) {
    int d = 4;
    while (d > 1 && local_mma_smem(cmax, ld, d) > 64 * 1024) --d;
    return d;
}

// One launch over all subdomains, or (a.nclass > 1) one per band-width
// group with the ring sized for that width: narrow subdomains then take
// less shared memory and more of their blocks share an SM.
template <typename TP, int NF, int MM>
static cudaError_t mma_nf(const LocalTmaArgs& a, const void* psi, void* zf, void* rc) {
    const int warps = a.ld / (8 * NF);
    auto kern = k_local_mma<TP, NF, MM>;
    static size_t smem_set = 0;
    auto launch = [&](int nsub, int cmax, int nbmax, const int32_t* order) -> cudaError_t {
        // no deeper than the group's block rows: the rest of the ring would stay unused
        const int depth = std::max(1, std::min(a.depth > 0 ? a.depth : local_mma_depth(cmax, a.ld), nbmax));
        const size_t smem = local_mma_smem(cmax, a.ld, depth);
        if (smem > smem_set) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            smem_set = smem;
        }
        return launch_kernel(a.pdl, kern, dim3(nsub), dim3(warps * 32), smem, a.stream, *a.tmF, a.subs,
                             a.tile_row0, a.piv, a.in.r, a.in.q, a.in.sc, (float*)zf, (const TP*)psi, (float*)rc,
                             a.ld, cmax, depth, a.budget, a.st, a.err, a.probe, order);
    };
    if (a.nclass <= 1 || a.order == nullptr) return launch(a.nsub, a.cmax, a.nbmax, nullptr);
    const int32_t* ord = a.order;
    for (int k = 0; k < a.nclass; ++k) {
        if (a.class_n[k] == 0) continue;
        const cudaError_t e = launch(a.class_n[k], a.class_c[k], a.class_nb[k], ord);
        if (e != cudaSuccess) return e;
        ord += a.class_n[k];
    }
    return cudaSuccess;
}

// Right-hand sides per warp: 8 or 16 (a.nr; 0 = 8), at most four warps per
// block.  (32 per warp needs more registers than a thread has.)
static int mma_rhs_per_warp(const LocalTmaArgs& a) {
    int nr = a.nr == 16 && a.ld >= 16 ? 16 : 8;
    while (a.ld / nr > 4) nr *= 2;
    return nr;
}

template <typename TP>
static cudaError_t mma_tp(const LocalTmaArgs& a, const void* psi, void* zf, void* rc) {
    const bool big = a.mmax > 8;
    if (mma_rhs_per_warp(a) == 8) return big ? mma_nf<TP, 1, 16>(a, psi, zf, rc) : mma_nf<TP, 1, 8>(a, psi, zf, rc);
    return big ? mma_nf<TP, 2, 16>(a, psi, zf, rc) : mma_nf<TP, 2, 8>(a, psi, zf, rc);
}

cudaError_t launch_local_mma(const LocalTmaArgs& a, int prec, const void* psi, void* zf, void* rc) {
    if (prec == AMS_PREC_FP32) return mma_tp<float>(a, psi, zf, rc);
    return mma_tp<__nv_bfloat16>(a, psi, zf, rc);
}

AMS_DEBUG_TU_HOOKS(local_mma)

}  // namespace ams
