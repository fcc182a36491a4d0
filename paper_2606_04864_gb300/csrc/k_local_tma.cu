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

namespace ams {

// ---------------------------------------------------------------------------
// mbarrier / TMA primitives
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false when the budget runs out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int64_t budget) {
    for (int64_t i = 0; i < budget; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
        ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
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
            const float* __restrict__ piv, const double* __restrict__ rin, float* __restrict__ zf,
            const TP* __restrict__ psi, float* __restrict__ rc, int ld, int cmax, int depth,
            int64_t budget, SolveState* st) {
    if (st != nullptr && st->done) return;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned tile ring, then mbarriers, y/x ring, scratch
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const SubInfo S = subs[blockIdx.x];
    const int c = S.c, nb = S.nb, n = S.n;
    const int D = depth;
    const int nbuf = cmax + D + 1;
    float* tiles = (float*)base;                                        // nbuf * cmax * 1024
    uint64_t* bars = (uint64_t*)(tiles + (size_t)nbuf * cmax * 1024);    // nbuf (padded to even)
    float* ring = (float*)(bars + ((nbuf + 1) & ~1));                    // (cmax+1)*32*ld
    float* tmp = ring + (size_t)(cmax + 1) * 32 * ld;                    // 32*ld
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rhs0 = warp * NR;
    const int m = S.m;
    const int64_t trow = tile_row0[blockIdx.x];      // first tensor row of this subdomain
    const uint32_t tile_bytes = 4096u * (uint32_t)c;
    uint32_t phase = 0;                              // parity bit per slot
    bool ok = true;

    if (threadIdx.x == 0) {
        for (int i = 0; i < nbuf; ++i) mbar_init(smem_u32(bars + i), 1);
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
    };
    auto wait_slot = [&](int K) {
        const int slot = K % nbuf;
        const uint32_t par = (phase >> slot) & 1u;
        if (!mbar_wait(smem_u32(bars + slot), par, budget)) ok = false;
        phase ^= 1u << slot;
    };
    auto slot_tile = [&](int K, int d) -> const float* {
        return tiles + ((size_t)(K % nbuf) * cmax + d) * 1024;
    };

    float racc[MM][NR];
#pragma unroll
    for (int k = 0; k < MM; ++k)
#pragma unroll
        for (int j = 0; j < NR; ++j) racc[k][j] = 0.f;

    // inputs of block row K, prefetched two block rows ahead
    auto load_fwd = [&](int K, float (&tv)[NR], float (&pv)[MM], float& pvt) {
        const int row = K * 32 + lane;
        const bool valid = K < nb && row < n;
        const int64_t grow = S.row0 + row;
#pragma unroll
        for (int j = 0; j < NR; ++j) tv[j] = valid ? (float)rin[grow * ld + rhs0 + j] : 0.f;
#pragma unroll
        for (int k = 0; k < MM; ++k)
            pv[k] = (rc != nullptr && valid && k < m) ? to_f(psi[S.psi_off + (int64_t)row * m + k]) : 0.f;
        pvt = (K < nb) ? piv[S.row0 + min(row, n - 1)] : 1.f;
        if (!valid) pvt = 1.f;
    };
    float tn0[NR], pn0[MM], tn1[NR], pn1[MM], pv0, pv1;
    load_fwd(0, tn0, pn0, pv0);
    load_fwd(1, tn1, pn1, pv1);

    // ---------------- forward ----------------
    for (int j = 0; j < D && j < nb; ++j) issue(&tmF, j);
    for (int K = 0; K < nb && ok; ++K) {
        if (K + D < nb) issue(&tmF, K + D);
        float t[NR], pv[MM];
        const float pvt = pv0;
#pragma unroll
        for (int j = 0; j < NR; ++j) { t[j] = tn0[j]; tn0[j] = tn1[j]; }
#pragma unroll
        for (int k = 0; k < MM; ++k) { pv[k] = pn0[k]; pn0[k] = pn1[k]; }
        pv0 = pv1;
        load_fwd(K + 2, tn1, pn1, pv1);
        wait_slot(K);
        ok = __syncthreads_and(ok);      // uniform decision across the block
        if (!ok) break;
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
            const float* ys = ring + (size_t)(src % (c + 1)) * 32 * ld;
            if (d == 0) tile_rowdot<NR, 1>(slot_tile(K, d), lane, ys, ld, rhs0, -1.f, t);
            else tile_rowdot<NR, 0>(slot_tile(K, d), lane, ys, ld, rhs0, -1.f, t);
        }
#pragma unroll
        for (int j = 0; j < NR; ++j) tmp[lane * ld + rhs0 + j] = t[j];
        __syncwarp();
        float y[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) y[j] = pvt * t[j];
        tile_rowdot<NR, 2>(slot_tile(K, 0), lane, tmp, ld, rhs0, 1.f, y);
        float* yr = ring + (size_t)(K % (c + 1)) * 32 * ld;
#pragma unroll
        for (int j = 0; j < NR; ++j) yr[lane * ld + rhs0 + j] = y[j];
        if (valid) {
#pragma unroll
            for (int j = 0; j < NR; ++j) zf[grow * ld + rhs0 + j] = y[j];
        }
        __syncthreads();
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
    // ---------------- backward ----------------
    auto load_bwd = [&](int K, float (&wv)[NR], float& pvt) {
        const int row = K * 32 + lane;
        const bool valid = K >= 0 && row < n;
        const int64_t grow = S.row0 + row;
#pragma unroll
        for (int j = 0; j < NR; ++j) wv[j] = valid ? zf[grow * ld + rhs0 + j] : 0.f;
        pvt = valid ? piv[grow] : 1.f;
    };
    float wn0[NR], wn1[NR], q0, q1;
    if (ok) {
        load_bwd(nb - 1, wn0, q0);
        load_bwd(nb - 2, wn1, q1);
        for (int j = 0; j < D && nb - 1 - j >= 0; ++j) issue(&tmB, nb - 1 - j);
    }
    for (int K = nb - 1; K >= 0 && ok; --K) {
        if (K - D >= 0) issue(&tmB, K - D);
        float w[NR];
        const float pvt = q0;
#pragma unroll
        for (int j = 0; j < NR; ++j) { w[j] = wn0[j]; wn0[j] = wn1[j]; }
        q0 = q1;
        load_bwd(K - 2, wn1, q1);
        wait_slot(K);
        ok = __syncthreads_and(ok);
        if (!ok) break;
        const int row = K * 32 + lane;
        const bool valid = row < n;
        const int64_t grow = S.row0 + row;
        for (int d = 1; d <= c; ++d) {
            const int src = K + d;
            if (src >= nb) break;
            const float* xs = ring + (size_t)(src % (c + 1)) * 32 * ld;
            // transposed tile of L_{K+d,K}: dense tile c-d of block row K+d,
            // or (d == c) the upper part of M_{K+c} (rows r <= lane of M^T)
            if (d < c) tile_rowdot<NR, 0>(slot_tile(src, c - d), lane, xs, ld, rhs0, -1.f, w);
            else tile_rowdot<NR, 3>(slot_tile(src, 0), lane, xs, ld, rhs0, -1.f, w);
        }
#pragma unroll
        for (int j = 0; j < NR; ++j) tmp[lane * ld + rhs0 + j] = w[j];
        __syncwarp();
        float x[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) x[j] = pvt * w[j];
        // L_KK^{-T}: strict lower part of M_K read as row `lane` of M_K^T (r > lane)
        tile_rowdot<NR, 4>(slot_tile(K, 0), lane, tmp, ld, rhs0, 1.f, x);
        float* xr = ring + (size_t)(K % (c + 1)) * 32 * ld;
#pragma unroll
        for (int j = 0; j < NR; ++j) xr[lane * ld + rhs0 + j] = x[j];
        if (valid) {
#pragma unroll
            for (int j = 0; j < NR; ++j) zf[grow * ld + rhs0 + j] = x[j];
        }
        __syncthreads();
    }
    if (!ok) {
        // record the timeout and drain this block's copies in flight (bounded)
        if (threadIdx.x == 0 && st != nullptr) {
            atomicExch(&st->status, (int)AMS_ERR_DEVICE_TIMEOUT);
            st->done = 1;
        }
        for (int i = 0; i < nbuf; ++i) mbar_wait(smem_u32(bars + i), (phase >> i) & 1u, budget);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t local_tma_smem(int cmax, int ld, int depth) {
    const int nbuf = cmax + depth + 1;
    return 1024 /* alignment slack */ + (size_t)nbuf * cmax * 4096 + (size_t)((nbuf + 1) & ~1) * 8 +
           ((size_t)(cmax + 1) * 32 * ld + 32 * ld) * sizeof(float);
}

int local_tma_depth(int cmax, int ld) {
    int d = 4;
    while (d > 1 && local_tma_smem(cmax, ld, d) > 100 * 1024) --d;
    return d;
}

template <typename TP, int NR, int MM>
static cudaError_t tma_nr(const LocalTmaArgs& a, const void* psi, void* zf, void* rc) {
    const int warps = a.ld / NR;
    const int depth = local_tma_depth(a.cmax, a.ld);
    const size_t smem = local_tma_smem(a.cmax, a.ld, depth);
    auto kern = k_local_tma<TP, NR, MM>;
    static size_t smem_set = 0;
    if (smem > smem_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        smem_set = smem;
    }
    kern<<<a.nsub, warps * 32, smem, a.stream>>>(*a.tmF, *a.tmB, a.subs, a.tile_row0, a.piv, a.rin, (float*)zf,
                                                  (const TP*)psi, (float*)rc, a.ld, a.cmax, depth, a.budget, a.st);
    return cudaGetLastError();
}

template <typename TP>
static cudaError_t tma_tp(const LocalTmaArgs& a, const void* psi, void* zf, void* rc) {
    const bool big = a.mmax > 8;
    const int nrmax = big ? 4 : 8;
    const int nr = a.ld < nrmax ? a.ld : nrmax;
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

cudaError_t launch_local_tma(const LocalTmaArgs& a, int prec, const void* psi, void* zf, void* rc) {
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

}  // namespace ams
