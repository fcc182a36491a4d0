// Local solves of the reduced-precision preconditioner (Section 3.2 A_i,
// fine-level term sum_i R_i^T A_i^{-1} R_i r) with the factor tiles fed by
// the Tensor Memory Accelerator.
//
// Storage (FP32, one 32x32 tile = 4 KB, row-major inside a tile):
//   forward copy,  block row K: [ M_K | L_{K,K-c+1} | ... | L_{K,K-1} ]
//   backward copy, block row K: [ M_K^T | L_{K,K-c+1}^T | ... ]
// with M_K[r][q] = L_{K,K-c}[r][q] (q >= r) and (L_KK^{-1})[r][q] (q < r),
// plus the reciprocal pivots 1/L_KK[r][r] in a per-row array.  Both copies
// are viewed as 2-D tensors of 32-float rows; one TMA box is one tile,
// written to shared memory with the 128-byte swizzle (16-byte chunk j of
// tile row r lands at chunk j ^ (r mod 8)), so a lane that owns tile row r
// reads its 32 coefficients with eight conflict-free 128-bit loads.  Each
// ring slot has an mbarrier that the TMA completes (expect-tx); every wait
// is bounded and a timeout sets AMS_ERR_DEVICE_TIMEOUT.
//
// Forward sweep (lane = row r of block row K):
//   t = r_K - sum_d L_{K,K-c+d} y_{K-c+d} ;  y_K = L_KK^{-1} t
// Backward sweep (lane = column l of block column K, i.e. row l of the
// transposed tiles):
//   w = y_K - sum_d L_{K+d,K}^T x_{K+d}   ;  x_K = L_KK^{-T} w
#include <cstdint>
#include <cstdio>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "ams_internal.h"
#include "kernels.cuh"
#include "launch.h"
#include "tma.cuh"

namespace ams {

// Row stride (floats) of the y/x ring of the several-RHS kernel: ld + 4 for
// ld >= 2 (conflict-free per-lane row stores, 16-byte aligned rows); one
// right-hand side keeps a contiguous vector.
__host__ __device__ __forceinline__ int local_tma_row_stride(int ld) { return ld >= 2 ? ld + 4 : 1; }

// NR consecutive floats of one ring row (16-byte stores when NR % 4 == 0:
// eight lanes of a quarter warp then cover all 32 banks).
template <int NR>
__device__ __forceinline__ void store_row(float* p, const float (&v)[NR]) {
    if (NR % 4 == 0) {
#pragma unroll
        for (int k = 0; k < NR; k += 4)
            *reinterpret_cast<float4*>(p + k) = make_float4(v[k], v[(k + 1) % NR], v[(k + 2) % NR], v[(k + 3) % NR]);
    } else if (NR == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1 % NR]);
    } else {
#pragma unroll
        for (int j = 0; j < NR; ++j) p[j] = v[j];
    }
}

// Row r of a swizzled 32x32 FP32 tile: 16-byte chunk j (columns 4j..4j+3).
__device__ __forceinline__ float4 tile_chunk(const float* tile, int r, int j) {
    return *reinterpret_cast<const float4*>(tile + r * 32 + ((j ^ (r & 7)) << 2));
}
__device__ __forceinline__ float f4(const float4& v, int e) {
    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

// Keep columns q of chunk j with (q >= lo) when upper, (q < lo) otherwise.
__device__ __forceinline__ float4 mask_chunk(float4 v, int j, int lo, bool upper) {
    const int q0 = 4 * j;
    if (upper) {
        if (q0 + 0 < lo) v.x = 0.f;
        if (q0 + 1 < lo) v.y = 0.f;
        if (q0 + 2 < lo) v.z = 0.f;
        if (q0 + 3 < lo) v.w = 0.f;
    } else {
        if (q0 + 0 >= lo) v.x = 0.f;
        if (q0 + 1 >= lo) v.y = 0.f;
        if (q0 + 2 >= lo) v.z = 0.f;
        if (q0 + 3 >= lo) v.w = 0.f;
    }
    return v;
}

// acc[j] += SIGN * sum_q T[row][q] * vec[q*ld + rhs0 + j] over the kept
// columns.  MODE 0: all; 1: q >= row; 2: q < row; 3: q <= row; 4: q > row.
template <int NR, int MODE>
__device__ __forceinline__ void tile_rowdot(const float* tile, int row, const float* vec, int ld, int rhs0,
                                            float sign, float (&acc)[NR]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float4 v = tile_chunk(tile, row, j);
        if (MODE == 1) v = mask_chunk(v, j, row, true);
        if (MODE == 2) v = mask_chunk(v, j, row, false);
        if (MODE == 3) v = mask_chunk(v, j, row + 1, false);
        if (MODE == 4) v = mask_chunk(v, j, row + 1, true);
        if (NR == 1) {
            const float4 x = *reinterpret_cast<const float4*>(vec + 4 * j);   // ld == 1
            acc[0] += sign * (v.x * x.x + v.y * x.y + v.z * x.z + v.w * x.w);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float cf = sign * f4(v, e);
                const float* xr = vec + (4 * j + e) * ld + rhs0;
                if (NR == 2) {
                    const float2 x = *reinterpret_cast<const float2*>(xr);
                    acc[0] += cf * x.x;
                    acc[1 % NR] += cf * x.y;
                } else {
#pragma unroll
                    for (int k = 0; k < NR; k += 4) {
                        const float4 x = *reinterpret_cast<const float4*>(xr + k);
                        acc[k + 0] += cf * x.x;
                        acc[(k + 1) % NR] += cf * x.y;
                        acc[(k + 2) % NR] += cf * x.z;
                        acc[(k + 3) % NR] += cf * x.w;
                    }
                }
            }
        }
    }
}

template <typename TP, int NR, int MM>
__global__ void __launch_bounds__(256)
k_local_tma(const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmB,
            const SubInfo* __restrict__ subs, const int64_t* __restrict__ tile_row0,
            const float* __restrict__ piv, const double* __restrict__ rin, const double* __restrict__ qin,
            const CgScalars* __restrict__ csc, float* __restrict__ zf, const TP* __restrict__ psi,
            float* __restrict__ rc, int ld, int cmax, int depth, int64_t budget, SolveState* st, int32_t* err,
            int probe) {
    pdl_wait();
    if (st != nullptr && st->done) return;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned tile ring, then mbarriers, y/x ring, scratch
    unsigned char* base = smem_align1024(smem_raw);
    const SubInfo S = subs[blockIdx.x];
    if (!AMS_ROW_OK(S.row0, 5) || !AMS_ROW_OK(S.row0 + S.n - 1, 5)) return;
    const int c = S.c, nb = S.nb, n = S.n;
    const int D = depth;
    const int nbuf = cmax + D + 1;
    float* tiles = (float*)base;                                        // nbuf * cmax * 1024
    uint64_t* bars = (uint64_t*)(tiles + (size_t)nbuf * cmax * 1024);    // ring_bar_slots(nbuf)
    // y/x ring and scratch: rows of lds = ld + 4 floats, so that the 32 lanes
    // storing their own rows hit distinct banks (a row stride of ld floats
    // put every lane on the same bank) while rows stay 16-byte aligned
    const int lds = local_tma_row_stride(ld);
    float* ring = (float*)(bars + ring_bar_slots(nbuf));                 // (cmax+1)*32*lds
    float* tmp = ring + (size_t)(cmax + 1) * 32 * lds;                   // 32*lds
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rhs0 = warp * NR;
    const int m = S.m;
    const int64_t trow = tile_row0[blockIdx.x];      // first tensor row of this subdomain
    const uint32_t tile_bytes = 4096u * (uint32_t)c;
    // Per slot: the parity of its next completion, and whether a copy was
    // issued into it and not yet seen complete.  Both change only when a
    // wait succeeds, so after a wait runs out the exit drain still waits
    // for that slot's copy at the parity it was issued with.  Every thread
    // keeps its own copy (issue and wait are called by all threads).
    uint32_t phase = 0, pend = 0;
    bool ok = true;

    if (threadIdx.x == 0) {
        for (int i = 0; i <= nbuf; ++i) mbar_init(smem_u32(bars + i), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();

    auto issue = [&](const CUtensorMap* map, int K) {
        if (threadIdx.x == 0) {
            const int slot = K % nbuf;
            const uint32_t bar = smem_u32(bars + slot);
            mbar_expect_tx(bar, tile_bytes);
            for (int d = 0; d < c; ++d)
                tma_load_2d(smem_u32(tiles + ((size_t)slot * cmax + d) * 1024), map, 0,
                            (int32_t)(trow + ((int64_t)K * c + d) * 32), bar);
        }
        pend |= 1u << (K % nbuf);
    };
    auto wait_slot = [&](int K) {
        const int slot = K % nbuf;
        const uint32_t par = (phase >> slot) & 1u;
        if (!mbar_wait(smem_u32(bars + slot), par, budget)) {
            ok = false;
            return;
        }
        phase ^= 1u << slot;
        pend &= ~(1u << slot);
    };
    auto slot_tile = [&](int K, int d) -> const float* {
        return tiles + ((size_t)(K % nbuf) * cmax + d) * 1024;
    };

    float racc[MM][NR];
#pragma unroll
    for (int k = 0; k < MM; ++k)
#pragma unroll
        for (int j = 0; j < NR; ++j) racc[k][j] = 0.f;

    // Per-row inputs of block row K (r, basis row, pivot; y in the backward
    // sweep) sit in PF rotating register buffers: the step that consumes
    // buffer u reloads it with row K+PF (forward) or K-PF (backward), so
    // every global load has PF steps to arrive.  The step loop is unrolled
    // by PF so that buffer indices are compile-time constants.
    constexpr int PF = (NR <= 2) ? 4 : 2;
    // Loaded values stay in their loaded type until use (see the
    // one-right-hand-side kernel below).
    // r' = r - alpha q for (system, rhs) pairs still iterating
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
    double bt[PF][NR], bq[PF][NR];
    TP bp[PF][MM];
    float bv[PF];
    auto load_fwd = [&](int K, double (&tv)[NR], double (&qv)[NR], TP (&pv)[MM], float& pvt) {
        const int row = K * 32 + lane;
        const bool valid = K < nb && row < n;
        const int64_t grow = S.row0 + row;
        pvt = 1.f;
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            tv[j] = 0.0;
            qv[j] = 0.0;
        }
#pragma unroll
        for (int k = 0; k < MM; ++k) pv[k] = TP(0.f);
        if (valid) {
            pvt = piv[grow];
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                tv[j] = rin[grow * ld + rhs0 + j];
                if (upd[j]) qv[j] = qin[grow * ld + rhs0 + j];
            }
            if (rc != nullptr) {
#pragma unroll
                for (int k = 0; k < MM; ++k)
                    if (k < m) pv[k] = psi[S.psi_off + (int64_t)row * m + k];
            }
        }
    };
#pragma unroll
    for (int u = 0; u < PF; ++u) load_fwd(u, bt[u], bq[u], bp[u], bv[u]);

    auto fwd_step = [&](int K, double (&tb)[NR], double (&qb)[NR], TP (&pb)[MM], float& vb) {
        if (K + D < nb) issue(&tmF, K + D);
        float t[NR], pv[MM];
        const float pvt = vb;
#pragma unroll
        for (int j = 0; j < NR; ++j) t[j] = f64_to_f32(upd[j] ? fma(-al[j], qb[j], tb[j]) : tb[j]);
#pragma unroll
        for (int k = 0; k < MM; ++k) pv[k] = to_f(pb[k]);
        load_fwd(K + PF, tb, qb, pb, vb);
        wait_slot(K);
        ok = __syncthreads_and(ok);      // uniform decision across the block
        if (!ok) return;
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
            const float* ys = ring + (size_t)(src % (c + 1)) * 32 * lds;
            if (d == 0) tile_rowdot<NR, 1>(slot_tile(K, d), lane, ys, lds, rhs0, -1.f, t);
            else tile_rowdot<NR, 0>(slot_tile(K, d), lane, ys, lds, rhs0, -1.f, t);
        }
        store_row<NR>(tmp + lane * lds + rhs0, t);
        __syncwarp();
        float y[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) y[j] = pvt * t[j];
        tile_rowdot<NR, 2>(slot_tile(K, 0), lane, tmp, lds, rhs0, 1.f, y);
        float* yr = ring + (size_t)(K % (c + 1)) * 32 * lds;
        store_row<NR>(yr + lane * lds + rhs0, y);
        if (valid) {
#pragma unroll
            for (int j = 0; j < NR; ++j) zf[grow * ld + rhs0 + j] = y[j];
        }
        __syncthreads();
    };

    // ---------------- forward ----------------
    for (int j = 0; j < D && j < nb; ++j) issue(&tmF, j);
    if (probe) {   // timeout test hook: a bounded wait on a barrier nothing completes
        if (!mbar_wait(smem_u32(bars + nbuf), 0u, budget)) ok = false;
        ok = __syncthreads_and(ok);
    }
#pragma unroll 1
    for (int K0 = 0; K0 < nb && ok; K0 += PF) {
#pragma unroll
        for (int u = 0; u < PF; ++u)
            if (K0 + u < nb && ok) fwd_step(K0 + u, bt[u], bq[u], bp[u], bv[u]);
    }
    if (rc != nullptr && ok) {
#pragma unroll
        for (int k = 0; k < MM; ++k)
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                float v = racc[k][j];
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if (lane == 0 && k < m) rc[(S.coff + k) * ld + rhs0 + j] = v;
            }
    }
    pdl_trigger();
    // ---------------- backward ----------------
    float bw[PF][NR];
    auto load_bwd = [&](int K, float (&wv)[NR], float& pvt) {
        const int row = K * 32 + lane;
        const bool valid = K >= 0 && row < n;
        const int64_t grow = S.row0 + row;
        pvt = 1.f;
#pragma unroll
        for (int j = 0; j < NR; ++j) wv[j] = 0.f;
        if (valid) {
            pvt = piv[grow];
#pragma unroll
            for (int j = 0; j < NR; ++j) wv[j] = zf[grow * ld + rhs0 + j];
        }
    };
    auto bwd_step = [&](int K, float (&wb)[NR], float& vb) {
        if (K - D >= 0) issue(&tmB, K - D);
        float w[NR];
        const float pvt = vb;
#pragma unroll
        for (int j = 0; j < NR; ++j) w[j] = wb[j];
        load_bwd(K - PF, wb, vb);
        wait_slot(K);
        ok = __syncthreads_and(ok);
        if (!ok) return;
        const int row = K * 32 + lane;
        const bool valid = row < n;
        const int64_t grow = S.row0 + row;
        for (int d = 1; d <= c; ++d) {
            const int src = K + d;
            if (src >= nb) break;
            const float* xs = ring + (size_t)(src % (c + 1)) * 32 * lds;
            // transposed tile of L_{K+d,K}: dense tile c-d of block row K+d,
            // or (d == c) the upper part of M_{K+c} (rows r <= lane of M^T)
            if (d < c) tile_rowdot<NR, 0>(slot_tile(src, c - d), lane, xs, lds, rhs0, -1.f, w);
            else tile_rowdot<NR, 3>(slot_tile(src, 0), lane, xs, lds, rhs0, -1.f, w);
        }
        store_row<NR>(tmp + lane * lds + rhs0, w);
        __syncwarp();
        float x[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) x[j] = pvt * w[j];
        // L_KK^{-T}: strict lower part of M_K read as row `lane` of M_K^T (r > lane)
        tile_rowdot<NR, 4>(slot_tile(K, 0), lane, tmp, lds, rhs0, 1.f, x);
        float* xr = ring + (size_t)(K % (c + 1)) * 32 * lds;
        store_row<NR>(xr + lane * lds + rhs0, x);
        if (valid) {
#pragma unroll
            for (int j = 0; j < NR; ++j) zf[grow * ld + rhs0 + j] = x[j];
        }
        __syncthreads();
    };
    if (ok) {
#pragma unroll
        for (int u = 0; u < PF; ++u) load_bwd(nb - 1 - u, bw[u], bv[u]);
        for (int j = 0; j < D && nb - 1 - j >= 0; ++j) issue(&tmB, nb - 1 - j);
    }
#pragma unroll 1
    for (int K0 = nb - 1; K0 >= 0 && ok; K0 -= PF) {
#pragma unroll
        for (int u = 0; u < PF; ++u)
            if (K0 - u >= 0 && ok) bwd_step(K0 - u, bw[u], bv[u]);
    }
    if (!ok) timeout_drain(bars, nbuf, pend, phase, err, st, threadIdx.x == 0);
}


// ---------------------------------------------------------------------------
// One right-hand side: one warp per subdomain, forward tiles only.
//
// With a single vector each step is a chain of two dependent 32x32 products
// (the off-diagonal update, then L_KK^{-1}), so the kernel is bound by the
// latency of that chain and by the bytes of the factor, not by arithmetic.
// This variant trims both:
//   * the backward sweep reads the forward tiles by column (lane l reads
//     column l of a tile: element (r, l) lies in bank ((l/4) ^ (r mod 8))*4
//     + l mod 4 of row r, so the 32 lanes of a load hit 32 distinct banks),
//     so the transposed copy is never read and the block rows that the
//     forward sweep left in the ring are reused without a reload;
//   * y stays in shared memory between the sweeps and x overwrites it in
//     place (step K reads y_K and x_{K+1..K+c} only);
//   * the row of M_K is loaded once for both of its parts; the triangular
//     masks act per 4-column chunk (a 0/1 weight per chunk, plus the one
//     chunk that holds the diagonal), and each 32-term dot is summed as a
//     tree of eight 4-term dots.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dot4(const float4& a, const float4& b) {
    return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)));
}
__device__ __forceinline__ float4 mul4(const float4& a, const float4& b) {
    return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}
__device__ __forceinline__ float sum8(const float (&c)[8]) {
    return ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
}
__device__ __forceinline__ float wsum8(const float (&w)[8], const float (&c)[8]) {
    const float a = fmaf(w[1], c[1], w[0] * c[0]);
    const float b = fmaf(w[3], c[3], w[2] * c[2]);
    const float d = fmaf(w[5], c[5], w[4] * c[4]);
    const float e = fmaf(w[7], c[7], w[6] * c[6]);
    return (a + b) + (d + e);
}
// Column `lane` of a swizzled tile against a broadcast vector v[0..31]:
// c[j] = sum_{r in chunk j} T[r][lane] v[r].
__device__ __forceinline__ void col_chunks(const float* T, const int (&csw)[8], const float* v, float (&c)[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float4 x = *reinterpret_cast<const float4*>(v + 4 * j);
        const int r = 4 * j;
        const float a0 = T[(r + 0) * 32 + csw[(r + 0) & 7]];
        const float a1 = T[(r + 1) * 32 + csw[(r + 1) & 7]];
        const float a2 = T[(r + 2) * 32 + csw[(r + 2) & 7]];
        const float a3 = T[(r + 3) * 32 + csw[(r + 3) & 7]];
        c[j] = fmaf(a3, x.w, fmaf(a2, x.z, fmaf(a1, x.y, a0 * x.x)));
    }
}

// Packed FP32 pairs (FFMA2, sm_100 and later): a 32-term dot product in
// 16 two-wide fused multiply-adds on four independent accumulators.
__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float pdot16(const float2 (&a)[16], const float* v) {
    float2 s0 = make_float2(0.f, 0.f), s1 = s0, s2 = s0, s3 = s0;
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
        const float4 v0 = *reinterpret_cast<const float4*>(v + 4 * j);
        const float4 v1 = *reinterpret_cast<const float4*>(v + 4 * j + 4);
        s0 = __ffma2_rn(a[2 * j], lo2(v0), s0);
        s1 = __ffma2_rn(a[2 * j + 1], hi2(v0), s1);
        s2 = __ffma2_rn(a[2 * j + 2], lo2(v1), s2);
        s3 = __ffma2_rn(a[2 * j + 3], hi2(v1), s3);
    }
    const float2 s = __fadd2_rn(__fadd2_rn(s0, s1), __fadd2_rn(s2, s3));
    return s.x + s.y;
}
// Column `lane` of a swizzled tile as 16 row pairs (2i, 2i+1).
__device__ __forceinline__ void col_pairs(const float* T, const int (&csw)[8], float2 (&c)[16]) {
#pragma unroll
    for (int i = 0; i < 16; ++i)
        c[i] = make_float2(T[(2 * i) * 32 + csw[(2 * i) & 7]], T[(2 * i + 1) * 32 + csw[(2 * i + 1) & 7]]);
}

// Basis row of one subdomain row (m <= MM entries) as raw 16-byte words when
// the row is 16-byte aligned and m == MM, element by element otherwise.
template <typename TP, int MM>
struct BasisRow {
    static constexpr int PER = 16 / (int)sizeof(TP);
    static constexpr int NW = (MM * (int)sizeof(TP) + 15) / 16;
    uint4 w[NW];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int i = 0; i < NW; ++i) w[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    __device__ __forceinline__ void load(const TP* __restrict__ pr, int m, bool vec) {
        if (MM % PER == 0 && vec) {
#pragma unroll
            for (int i = 0; i < NW; ++i) w[i] = __ldg(reinterpret_cast<const uint4*>(pr) + i);
        } else {
            TP* e = reinterpret_cast<TP*>(w);
#pragma unroll
            for (int k = 0; k < MM; ++k)
                if (k < m) e[k] = pr[k];
        }
    }
    __device__ __forceinline__ float get(int k) const { return to_f(reinterpret_cast<const TP*>(w)[k]); }
    // entries 2i and 2i+1 (a BF16 pair is widened with two integer operations)
    __device__ __forceinline__ float2 get2(int i) const {
        if constexpr (sizeof(TP) == 2) {
            const uint32_t u = reinterpret_cast<const uint32_t*>(w)[i];
            return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
        } else {
            return make_float2(get(2 * i), get(2 * i + 1));
        }
    }
};

// C1: every subdomain has c == 1 (one 32x32 tile per block row).  The
// backward sweep then keeps column `lane` of M_K in registers after step K
// and forms the step K-1 term sum_{r <= lane} M_K[r][lane] x_K[r] at once,
// so every tile column is read from shared memory once.
template <typename TP, int MM, bool C1>
__global__ void __launch_bounds__(32, 8)
k_local_tma1(const __grid_constant__ CUtensorMap tmF, const SubInfo* __restrict__ subs,
             const int64_t* __restrict__ tile_row0, const float* __restrict__ piv,
             const double* __restrict__ rin, const double* __restrict__ qin,
             const CgScalars* __restrict__ csc, float* __restrict__ zf, const TP* __restrict__ psi,
             float* __restrict__ rc, int cmax, int nbmax, int depth, int l2mode, int l2keep, int64_t budget,
             SolveState* st, int32_t* err, int probe) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_align1024(smem_raw);
    const SubInfo S = subs[blockIdx.x];
    if (!AMS_ROW_OK(S.row0, 5) || !AMS_ROW_OK(S.row0 + S.n - 1, 5)) return;
    const int c = C1 ? 1 : S.c;
    const int nb = S.nb, n = S.n, m = S.m;
    const int D = depth;
    const int nbuf = cmax + D + 1;
    // Block rows nb-nbuf .. nb-1 stay in the ring from the forward sweep to
    // the backward one; rows below Rres are loaded twice.
    const int Rres = nb > nbuf ? nb - nbuf : 0;
    float* tiles = (float*)base;                                        // nbuf * cmax * 1024
    uint64_t* bars = (uint64_t*)(tiles + (size_t)nbuf * cmax * 1024);    // ring_bar_slots(nbuf)
    float* yv = (float*)(bars + ring_bar_slots(nbuf));                   // nbmax * 32: y, then x
    float* tmp = yv + (size_t)nbmax * 32;                                // 32
    const int lane = threadIdx.x;
    const int jr = lane >> 2, er = lane & 3;
    const int64_t trow = tile_row0[blockIdx.x];
    const uint32_t tile_bytes = 4096u * (uint32_t)c;
    const int slot_floats = cmax * 1024;
    // parity of each slot's next completion, and the slots with a copy in
    // flight; both change only when a wait succeeds (see k_local_tma)
    uint32_t phase = 0, pend = 0;
    bool ok = true;

    // per-lane offsets and masks, fixed for the whole kernel
    int rsw[8], csw[8];
    float2 mk[16], mg[16];                           // 1 where index >= lane / index > lane, pairs (2i, 2i+1)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        rsw[j] = lane * 32 + ((j ^ (lane & 7)) << 2);   // chunk j of tile row `lane`
        csw[j] = ((jr ^ j) << 2) + er;                 // element (r, lane) sits at r*32 + csw[r & 7]
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        mk[i] = make_float2(2 * i >= lane ? 1.f : 0.f, 2 * i + 1 >= lane ? 1.f : 0.f);
        mg[i] = make_float2(2 * i > lane ? 1.f : 0.f, 2 * i + 1 > lane ? 1.f : 0.f);
    }
    const float2 neg1 = make_float2(-1.f, -1.f);

    if (lane == 0) {
        for (int i = 0; i <= nbuf; ++i) mbar_init(smem_u32(bars + i), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncwarp();

    // ring slots are tracked incrementally (no division in the step loop)
    auto wrap_up = [&](int sl) { return sl >= nbuf ? sl - nbuf : sl; };
    auto wrap_dn = [&](int sl) { return sl < 0 ? sl + nbuf : sl; };
    // L2 priorities of the tile copies (l2mode > 0): a copy that reads a
    // block row for the last time (a resident row's forward load, a backward
    // reload, a forward load whose reload is far away) is evict-first; the
    // forward loads of the l2keep rows below Rres, which the backward sweep
    // reloads soonest, keep normal (l2mode 1) or evict-last (2) priority.
    uint64_t pol_dead = 0, pol_keep = 0;
    if (l2mode > 0 && lane == 0) {
        pol_dead = l2_policy_evict_first();
        pol_keep = l2mode == 2 ? l2_policy_evict_last() : l2_policy_evict_normal();
    }
    auto issue = [&](int K, int slot, bool reload) {
        if (lane == 0) {
            const uint32_t bar = smem_u32(bars + slot);
            mbar_expect_tx(bar, tile_bytes);
            const bool keep = !reload && K < Rres && K >= Rres - l2keep;
            const uint64_t pol = keep ? pol_keep : pol_dead;
            for (int d = 0; d < c; ++d) {
                const uint32_t dst = smem_u32(tiles + slot * slot_floats + d * 1024);
                const int32_t y = (int32_t)(trow + ((int64_t)K * c + d) * 32);
                if (l2mode > 0)
                    tma_load_2d_hint(dst, &tmF, 0, y, bar, pol);
                else
                    tma_load_2d(dst, &tmF, 0, y, bar);
            }
        }
        pend |= 1u << slot;
    };
    auto wait_slot = [&](int slot) {
        if (!mbar_wait(smem_u32(bars + slot), (phase >> slot) & 1u, budget)) {
            ok = false;
            return;
        }
        phase ^= 1u << slot;
        pend &= ~(1u << slot);
    };

    static_assert(MM % 2 == 0, "basis rows are accumulated in pairs");
    float2 racc[MM / 2];
#pragma unroll
    for (int k = 0; k < MM / 2; ++k) racc[k] = make_float2(0.f, 0.f);

    // Per-row inputs of block row K+PF are loaded while step K runs.  They
    // stay in the loaded type until the step that uses them: a conversion
    // or a select right after the load would wait for it there.  Basis rows
    // and pivots are setup data; r and q are written by the previous
    // kernels and are read only after pdl_wait().
    constexpr int PF = 4;
    const float* vp = piv + S.row0 + lane;
    const bool vec = (m == MM) && ((reinterpret_cast<uintptr_t>(psi + S.psi_off) & 15) == 0);
    const TP* pp = rc != nullptr ? psi + S.psi_off + (int64_t)lane * m : nullptr;
    double bt[PF], bq[PF];
    BasisRow<TP, MM> bp[PF];
    float bv[PF];
    auto load_static = [&](int K, BasisRow<TP, MM>& pv, float& pvt) {
        const int row = K * 32 + lane;
        pvt = 1.f;
        pv.clear();
        if (K < nb && row < n) {
            pvt = vp[K * 32];
            if (rc != nullptr) pv.load(pp + (int64_t)K * 32 * m, m, vec);
        }
    };
    // first block rows of the factor and their setup inputs, ahead of the wait
    for (int j = 0; j < D && j < nb; ++j) issue(j, j, false);
#pragma unroll
    for (int u = 0; u < PF; ++u) load_static(u, bp[u], bv[u]);
    pdl_wait();
    if (st != nullptr && st->done) {   // converged: leave once the first copies have landed
        drain_copies(bars, nbuf, pend, phase);
        return;
    }
    if (probe) {   // timeout test hook: a bounded wait on a barrier nothing completes
        if (!mbar_wait(smem_u32(bars + nbuf), 0u, budget)) ok = false;
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
            timeout_drain(bars, nbuf, pend, phase, err, st, lane == 0);
            return;
        }
    }
    // r' = r - alpha q when this subdomain's system is still iterating
    double alpha = 0.0;
    bool upd = false;
    if (qin != nullptr) {
        const CgScalars cs = csc[S.seg];
        upd = cs.active != 0;
        if (upd) alpha = cs.rho / cs.pq;
    }
    const double* rp = rin + S.row0 + lane;
    const double* qp = upd ? qin + S.row0 + lane : nullptr;
    auto load_dyn = [&](int K, double& tv, double& qv) {
        const int row = K * 32 + lane;
        tv = 0.0;
        qv = 0.0;
        if (K < nb && row < n) {
            tv = rp[K * 32];
            if (upd) qv = qp[K * 32];
        }
    };
#pragma unroll
    for (int u = 0; u < PF; ++u) load_dyn(u, bt[u], bq[u]);

    int sK = 0;   // slot of block row K
    auto fwd_step = [&](int K, double& tb, double& qb, BasisRow<TP, MM>& pb, float& vb) {
        if (K + D < nb) issue(K + D, wrap_up(sK + D), false);
        // the FP64 pipe is nearly idle in this kernel: the hardware narrowing
        // is one instruction where the integer-pipe one is about a dozen
        float t = __double2float_rn(upd ? fma(-alpha, qb, tb) : tb);
        const float pvt = vb;
        if (rc != nullptr) {
            const float2 t2 = make_float2(t, t);
#pragma unroll
            for (int k = 0; k < MM / 2; ++k) racc[k] = __ffma2_rn(pb.get2(k), t2, racc[k]);
        }
        load_static(K + PF, pb, vb);
        load_dyn(K + PF, tb, qb);
        wait_slot(sK);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) return;
        const float* T = tiles + sK * slot_floats;
        // row `lane` of M_K split exactly into its two triangles: mu (q >= lane,
        // from L_{K,K-c}) and ml (q < lane, from L_KK^{-1})
        float2 mu[16], ml[16];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 m4 = *reinterpret_cast<const float4*>(T + rsw[j]);
            mu[2 * j] = __fmul2_rn(lo2(m4), mk[2 * j]);
            mu[2 * j + 1] = __fmul2_rn(hi2(m4), mk[2 * j + 1]);
            ml[2 * j] = __ffma2_rn(mu[2 * j], neg1, lo2(m4));
            ml[2 * j + 1] = __ffma2_rn(mu[2 * j + 1], neg1, hi2(m4));
        }
        // t = r_K - sum_d L_{K,K-c+d} y_{K-c+d}
        if (!C1) {
#pragma unroll 1
            for (int d = 1; d < c; ++d) {
                const int src = K - c + d;
                if (src < 0) continue;
                const float* Td = T + d * 1024;
                float2 dp[16];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 m4 = *reinterpret_cast<const float4*>(Td + rsw[j]);
                    dp[2 * j] = lo2(m4);
                    dp[2 * j + 1] = hi2(m4);
                }
                t -= pdot16(dp, yv + src * 32);
            }
        }
        if (K >= c) t -= pdot16(mu, yv + (K - c) * 32);
        tmp[lane] = t;
        __syncwarp();
        // y_K = L_KK^{-1} t: pivot times t plus the strict lower part of M_K
        const float y = fmaf(pvt, t, pdot16(ml, tmp));
        yv[K * 32 + lane] = y;
        sK = wrap_up(sK + 1);
        __syncwarp();
    };

    // ---------------- forward ----------------
#pragma unroll 1
    for (int K0 = 0; K0 < nb && ok; K0 += PF) {
#pragma unroll
        for (int u = 0; u < PF; ++u)
            if (K0 + u < nb && ok) fwd_step(K0 + u, bt[u], bq[u], bp[u], bv[u]);
    }
    pdl_trigger();
    if (rc != nullptr && ok) {
#pragma unroll
        for (int k = 0; k < MM; ++k) {
            float v = (k & 1) ? racc[k / 2].y : racc[k / 2].x;
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0 && k < m) rc[S.coff + k] = v;
        }
    }

    // ---------------- backward ----------------
    // Block rows Rres .. nb-1 are still in the ring; older ones are
    // reloaded D steps ahead of their use.
    auto load_bwd = [&](int K, float& pvt) {
        const int row = K * 32 + lane;
        pvt = 1.f;
        if (K >= 0 && row < n) pvt = vp[K * 32];
    };
    float ucarry = 0.f;   // C1: sum_{r <= lane} M_{K+1}[r][lane] x_{K+1}[r] for the next step
    sK = (nb - 1) % nbuf;
    auto bwd_step = [&](int K, float& vb) {
        if (K - D >= 0 && K - D < Rres) issue(K - D, wrap_dn(sK - D), true);
        const float pvt = vb;
        load_bwd(K - PF, vb);
        if (K < Rres) wait_slot(sK);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) return;
        float w = yv[K * 32 + lane];
        const float* Tm = tiles + sK * slot_floats;   // M_K
        if (C1) {
            w -= ucarry;
        } else {
            // w = y_K - sum_d L_{K+d,K}^T x_{K+d}
#pragma unroll 1
            for (int d = 1; d < c; ++d) {
                const int src = K + d;
                if (src >= nb) break;
                float2 cp[16];
                col_pairs(tiles + wrap_up(sK + d) * slot_floats + (c - d) * 1024, csw, cp);
                w -= pdot16(cp, yv + src * 32);
            }
            if (K + c < nb) {   // L_{K+c,K}: upper part of M_{K+c}, rows r <= lane of column lane
                const float* Tc = tiles + wrap_up(sK + c) * slot_floats;
                const float* v = yv + (K + c) * 32;
                float2 cp[16], cl[16];
                col_pairs(Tc, csw, cp);
#pragma unroll
                for (int i = 0; i < 16; ++i) cl[i] = __ffma2_rn(__fmul2_rn(cp[i], mg[i]), neg1, cp[i]);
                w -= pdot16(cl, v);
            }
        }
        tmp[lane] = w;
        __syncwarp();
        // x_K = L_KK^{-T} w: rows r > lane of column lane of M_K.  Column
        // `lane` splits exactly into au (rows r > lane, from L_KK^{-1}) and
        // al (rows r <= lane, from L_{K,K-c}).  (Reloading the transposed
        // tile instead, to read the column as a row, measured slower: the
        // reloads of the forward tiles find part of them still in L2, those
        // of a second array find nothing.)
        float2 au[16], al[16];
        col_pairs(Tm, csw, au);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float2 a2 = au[i];
            au[i] = __fmul2_rn(a2, mg[i]);
            al[i] = __ffma2_rn(au[i], neg1, a2);
        }
        const float x = fmaf(pvt, w, pdot16(au, tmp));
        yv[K * 32 + lane] = x;
        const int row = K * 32 + lane;
        if (row < n) zf[S.row0 + row] = x;
        __syncwarp();
        if (C1 && K > 0) {
            // term of step K-1: L_{K,K-1} is the upper part of M_K (rows r <= lane of column lane)
            ucarry = pdot16(al, yv + K * 32);
        }
        sK = wrap_dn(sK - 1);
    };
    if (ok) {
#pragma unroll
        for (int u = 0; u < PF; ++u) load_bwd(nb - 1 - u, bv[u]);
    }
#pragma unroll 1
    for (int K0 = nb - 1; K0 >= 0 && ok; K0 -= PF) {
#pragma unroll
        for (int u = 0; u < PF; ++u)
            if (K0 - u >= 0 && ok) bwd_step(K0 - u, bv[u]);
    }
    if (!ok) timeout_drain(bars, nbuf, pend, phase, err, st, lane == 0);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t local_tma_smem(int cmax, int ld, int depth) {
    const int nbuf = cmax + depth + 1;
    const int lds = local_tma_row_stride(ld);
    return 1024 /* alignment slack */ + (size_t)nbuf * cmax * 4096 + (size_t)ring_bar_slots(nbuf) * 8 +
           ((size_t)(cmax + 1) * 32 * lds + 32 * lds) * sizeof(float);
}

// Prefetch depth: block rows in flight per subdomain.  Deeper rings hide
// more TMA latency but cost shared memory; the single-warp blocks of the
// one-right-hand-side case must stay small enough for about eight resident
// blocks per SM.
int local_tma_depth(int cmax, int ld) {
    const size_t budget = (ld == 1) ? 32 * 1024 : 100 * 1024;
    int d = 6;
    while (d > 1 && local_tma_smem(cmax, ld, d) > budget) --d;
    return d;
}

template <typename TP, int NR, int MM>
static cudaError_t tma_nr(const LocalTmaArgs& a, const void* psi, void* zf, void* rc) {
    const int warps = a.ld / NR;
    const int depth = a.depth > 0 ? a.depth : local_tma_depth(a.cmax, a.ld);
    const size_t smem = local_tma_smem(a.cmax, a.ld, depth);
    auto kern = k_local_tma<TP, NR, MM>;
    static size_t smem_set = 0;
    if (smem > smem_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        smem_set = smem;
    }
    return launch_kernel(a.pdl, kern, dim3(a.nsub), dim3(warps * 32), smem, a.stream, *a.tmF, *a.tmB, a.subs,
                         a.tile_row0, a.piv, a.in.r, a.in.q, a.in.sc, (float*)zf, (const TP*)psi, (float*)rc, a.ld,
                         a.cmax, depth, a.budget, a.st, a.err, a.probe);
}

template <typename TP>
static cudaError_t tma_tp(const LocalTmaArgs& a, const void* psi, void* zf, void* rc) {
    const bool big = a.mmax > 8;
    const int nrmax = big ? 4 : 8;
    int nr = a.ld < nrmax ? a.ld : nrmax;
    // fewer right-hand sides per warp: more warps per block (at most 8, the kernel's launch bound)
    if (a.nr > 0 && a.nr < nr && a.ld / a.nr <= 8) nr = a.nr;
    if (big) {
        switch (nr) {
            case 1: return tma_nr<TP, 1, 16>(a, psi, zf, rc);
            case 2: return tma_nr<TP, 2, 16>(a, psi, zf, rc);
            default: return tma_nr<TP, 4, 16>(a, psi, zf, rc);
        }
    }
    switch (nr) {
        case 1: return tma_nr<TP, 1, 8>(a, psi, zf, rc);
        case 2: return tma_nr<TP, 2, 8>(a, psi, zf, rc);
        case 4: return tma_nr<TP, 4, 8>(a, psi, zf, rc);
        default: return tma_nr<TP, 8, 8>(a, psi, zf, rc);
    }
}

size_t local_tma1_smem(int cmax, int nbmax, int depth) {
    const int nbuf = cmax + depth + 1;
    return 1024 /* alignment slack */ + (size_t)nbuf * cmax * 4096 + (size_t)ring_bar_slots(nbuf) * 8 +
           ((size_t)nbmax * 32 + 32) * sizeof(float);
}

// Depth for the one-right-hand-side kernel: as deep as possible (at most 6)
// while about seven single-warp blocks still fit on an SM.
static int local_tma1_depth(int cmax, int nbmax) {
    int d = 6;
    while (d > 2 && local_tma1_smem(cmax, nbmax, d) > 31 * 1024) --d;
    return d;
}

template <typename TP, int MM, bool C1>
static cudaError_t tma1(const LocalTmaArgs& a, const void* psi, void* zf, void* rc) {
    const int depth = a.depth > 0 ? a.depth : local_tma1_depth(a.cmax, a.nbmax);
    const size_t smem = local_tma1_smem(a.cmax, a.nbmax, depth);
    auto kern = k_local_tma1<TP, MM, C1>;
    static size_t smem_set = 0;
    if (smem > smem_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        smem_set = smem;
    }
    return launch_kernel(a.pdl, kern, dim3(a.nsub), dim3(32), smem, a.stream, *a.tmF, a.subs, a.tile_row0,
                         a.piv,
                         a.in.r, a.in.q, a.in.sc, (float*)zf, (const TP*)psi, (float*)rc, a.cmax, a.nbmax, depth,
                         a.l2mode, a.l2keep, a.budget, a.st, a.err, a.probe);
}

// The one-right-hand-side kernel keeps y for a whole subdomain in shared
// memory; wider subdomains use the general kernel.
static bool use_tma1(const LocalTmaArgs& a) {
    return a.ld == 1 && local_tma1_smem(a.cmax, a.nbmax, 2) <= 200 * 1024;
}

size_t local_tma_launch_smem(const LocalTmaArgs& a, int depth) {
    if (use_tma1(a)) return local_tma1_smem(a.cmax, a.nbmax, depth);
    return a.ld >= 8 ? local_mma_smem(a.cmax, a.ld, depth) : local_tma_smem(a.cmax, a.ld, depth);
}

cudaError_t launch_local_tma(const LocalTmaArgs& a, int prec, const void* psi, void* zf, void* rc) {
    // 8 or more right-hand sides: the tile products on the tensor cores
    if (!use_tma1(a) && a.ld >= 8) return launch_local_mma(a, prec, psi, zf, rc);
    if (use_tma1(a)) {
        const bool big = a.mmax > 8, c1 = a.cmax == 1;
        if (prec == AMS_PREC_FP32) {
            if (big) return c1 ? tma1<float, 16, true>(a, psi, zf, rc) : tma1<float, 16, false>(a, psi, zf, rc);
            return c1 ? tma1<float, 8, true>(a, psi, zf, rc) : tma1<float, 8, false>(a, psi, zf, rc);
        }
        if (big)
            return c1 ? tma1<__nv_bfloat16, 16, true>(a, psi, zf, rc) : tma1<__nv_bfloat16, 16, false>(a, psi, zf, rc);
        return c1 ? tma1<__nv_bfloat16, 8, true>(a, psi, zf, rc) : tma1<__nv_bfloat16, 8, false>(a, psi, zf, rc);
    }
    if (prec == AMS_PREC_FP32) return tma_tp<float>(a, psi, zf, rc);
    return tma_tp<__nv_bfloat16>(a, psi, zf, rc);
}

// 2-D view [rows x 32] FP32 of a tile array; one box = one 32x32 tile,
// 128-byte swizzle in shared memory.
cudaError_t make_tile_map(void* base, int64_t rows, CUtensorMap* out) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorSymbolNotFound;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const cuuint64_t dims[2] = {32, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {32 * sizeof(float)};
    const cuuint32_t box[2] = {32, 32};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

AMS_DEBUG_TU_HOOKS(local_tma)

}  // namespace ams
