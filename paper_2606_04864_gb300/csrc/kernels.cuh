// Device helpers shared by the AMS kernels: deterministic segmented
// reductions, asynchronous shared-memory copies, small conversions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "ams_internal.h"

namespace ams {

// ---------------------------------------------------------------------------
// conversions of stored operands
// ---------------------------------------------------------------------------
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(double v) { return (float)v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

// FP32 <-> FP64 conversions on the integer pipe.  FP64 instructions are
// scarce on this GPU (about 1/64 of the FP32 rate) and a conversion between
// the two formats occupies the FP64 pipe.  For inputs whose result is a
// normal number the bit manipulation below gives exactly the IEEE results
// (widening is exact; narrowing rounds to nearest, ties to even, and a
// carry out of the mantissa moves into the exponent, up to infinity); every
// other input (zero, subnormal, infinity, NaN, out of range) takes the
// hardware conversion.
__device__ __forceinline__ double f32_to_f64(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)f;
    const uint64_t d = ((uint64_t)(u >> 31) << 63) | ((uint64_t)(e + 896u) << 52) |
                       ((uint64_t)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}
__device__ __forceinline__ float f64_to_f32(double x) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t e = (uint32_t)(b >> 52) & 0x7ffu;
    if (e < 897u || e > 1150u) return (float)x;        // result not a normal float before rounding
    const uint64_t m = b & 0xfffffffffffffull;
    uint32_t r = ((uint32_t)(b >> 63) << 31) | ((e - 896u) << 23) | (uint32_t)(m >> 29);
    const uint32_t rem = (uint32_t)(m & 0x1fffffffu);
    r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;
    return __uint_as_float(r);
}
__device__ __forceinline__ double widen(float v) { return f32_to_f64(v); }
__device__ __forceinline__ double widen(double v) { return v; }

template <typename T> struct Acc { using type = float; };
template <> struct Acc<double> { using type = double; };

template <typename T> __device__ __forceinline__ T from_d(double v);
template <> __device__ __forceinline__ float from_d<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ double from_d<double>(double v) { return v; }

// ---------------------------------------------------------------------------
// Checking build (-DAMS_DEBUG): index checks on the gathers of the solve
// kernels.  A failed check records its site number in this translation
// unit's error word (the first one wins) and the access is skipped (the
// value read as 0, or the subdomain left out); the host API reads the words
// after each call and returns AMS_ERR_CUDA naming the site.  Nothing traps.
// The bounds (internal rows, coarse rows) are per process: one handle at a
// time in the checking build.  In the release build the checks compile to
// `true` and the hooks do nothing.
// Sites: 1 SpMV column, 2 prolongation gather of y, 3 coarse-product
// gather, 4 several-RHS local solve rows, 5 one/few-RHS local solve rows,
// 6 caller-order permutation, 99 the self-test.
// ---------------------------------------------------------------------------
struct DebugBounds {
    int64_t n_rows;     // internal rows of all systems (padded)
    int64_t n_coarse;   // coarse rows of all systems
};
#ifdef AMS_DEBUG
static __constant__ DebugBounds c_dbg_bounds;
static __device__ int32_t g_dbg_site;
__device__ __forceinline__ bool dbg_index_ok(int64_t i, int64_t hi, int site) {
    if (i >= 0 && i < hi) return true;
    atomicCAS(&g_dbg_site, 0, site);
    return false;
}
#define AMS_ROW_OK(i, site) ::ams::dbg_index_ok((int64_t)(i), ::ams::c_dbg_bounds.n_rows, (site))
#define AMS_COARSE_OK(i, site) ::ams::dbg_index_ok((int64_t)(i), ::ams::c_dbg_bounds.n_coarse, (site))
#define AMS_DEBUG_TU_HOOKS(tu)                                                            \
    void debug_set_bounds_##tu(int64_t n_rows, int64_t n_coarse) {                        \
        const DebugBounds b{n_rows, n_coarse};                                            \
        cudaMemcpyToSymbol(c_dbg_bounds, &b, sizeof(b));                                  \
    }                                                                                     \
    int32_t debug_take_site_##tu() {                                                      \
        int32_t v = 0;                                                                    \
        if (cudaMemcpyFromSymbol(&v, g_dbg_site, sizeof(v)) != cudaSuccess) return -1;    \
        if (v != 0) {                                                                     \
            const int32_t z = 0;                                                          \
            cudaMemcpyToSymbol(g_dbg_site, &z, sizeof(z));                                \
        }                                                                                 \
        return v;                                                                         \
    }
#else
#define AMS_ROW_OK(i, site) true
#define AMS_COARSE_OK(i, site) true
#define AMS_DEBUG_TU_HOOKS(tu)                                                            \
    void debug_set_bounds_##tu(int64_t, int64_t) {}                                       \
    int32_t debug_take_site_##tu() { return 0; }
#endif

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  Kernels of the solve loop are launched so
// that they may start while the previous kernel on the stream drains: work
// that reads only setup data (matrix, factor tiles, basis) runs first, then
// pdl_wait() blocks until the previous grid has completed and its writes
// are visible.  Every such kernel calls pdl_wait() before it reads anything
// another solve kernel writes (including the solve state) and before any
// early exit, so completion stays transitive along the stream.
// pdl_trigger() lets the next kernel launch once every block of this one
// has passed it.  Both are no-ops for a normal launch.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// ---------------------------------------------------------------------------
// cp.async (16-byte, L2-only) staging into shared memory
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
// 16 bytes when `valid`, else 16 zero bytes (nothing is read from gmem)
__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::); }
// wait until at most n of this thread's committed groups are pending (n <= 7)
__device__ __forceinline__ void cp_async_wait_n(int n) {
    switch (n) {
        case 0: asm volatile("cp.async.wait_group 0;\n" ::); break;
        case 1: asm volatile("cp.async.wait_group 1;\n" ::); break;
        case 2: asm volatile("cp.async.wait_group 2;\n" ::); break;
        case 3: asm volatile("cp.async.wait_group 3;\n" ::); break;
        case 4: asm volatile("cp.async.wait_group 4;\n" ::); break;
        case 5: asm volatile("cp.async.wait_group 5;\n" ::); break;
        case 6: asm volatile("cp.async.wait_group 6;\n" ::); break;
        default: asm volatile("cp.async.wait_group 7;\n" ::); break;
    }
}

// Copy `bytes` (multiple of 16, both addresses 16-byte aligned) with the
// whole thread block.
__device__ __forceinline__ void block_copy_async(void* smem, const void* gmem, int64_t bytes) {
    const int64_t n16 = bytes >> 4;
    char* s = (char*)smem;
    const char* g = (const char*)gmem;
    for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) cp_async16(s + 16 * i, g + 16 * i);
}

// ---------------------------------------------------------------------------
// Deterministic segmented reduction.
//
// A "reduction block" covers a contiguous range of elements of a node-major
// vector (whole kRedElems-element chunks of a single system, since systems
// are padded to kRowAlign rows), or a contiguous range of subdomains of a
// single system; a system's blocks are consecutive.  Each thread block of a reduction kernel handles one reduction
// block and produces NV partial values per right-hand side.  Partials are
// summed in a fixed order in two levels: groups of kRedGroup blocks (the
// last block of a group to finish sums the group), then all groups of a
// system (the last group to finish sums them and calls the finisher).  The
// order of every floating-point sum is fixed, so results are bitwise
// reproducible.
// ---------------------------------------------------------------------------
struct RedLayout {
    const int64_t* blk_lo;     // block b covers [blk_lo[b], blk_lo[b+1]) (elements or subdomains)
    const int32_t* blk_seg;    // reduction block -> system
    const int32_t* seg_blk0;   // system -> first reduction block
    const int32_t* seg_nblk;   // system -> number of reduction blocks
    const int32_t* seg_grp0;   // system -> first group
    double* part1;             // [nblk][NV][ld]
    double* part2;             // [ngroups][NV][ld]
    int32_t* cnt1;             // [ngroups]   zero at rest
    int32_t* cnt2;             // [nseg]      zero at rest
    int32_t* cnt3;             // [1]         zero at rest (systems finished)
};

// Sum `count` vectors of `nv` doubles (vector j at src + j*stride) in a
// fixed order using all threads of the block; result lands in dst[0..nv).
// nv is a power of two <= blockDim.x (a power of two).  Thread t adds the
// vectors j = t/nv, t/nv + blockDim.x/nv, ... of component t % nv; threads
// of one warp that share a component combine by xor shuffles, and the
// per-warp (or, for nv >= 32, per-thread) partials are added in index order
// after a single barrier.  Uses `scratch` (blockDim.x doubles).
__device__ inline void block_sum_vectors(const double* src, int count, int64_t stride, int nv,
                                         double* dst, double* scratch) {
    const int t = threadIdx.x;
    const int lanes_per = blockDim.x / nv;        // threads per component
    const int v = t % nv;
    double s = 0.0;
    for (int j = t / nv; j < count; j += lanes_per) s += __ldcg(src + (int64_t)j * stride + v);
    if (nv < 32) {
        for (int off = 16; off >= nv; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if ((t & 31) < nv) scratch[(t >> 5) * nv + v] = s;
        __syncthreads();
        if (t < nv) {
            double a = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += scratch[w * nv + t];
            dst[t] = a;
        }
    } else {
        scratch[t] = s;
        __syncthreads();
        if (t < nv) {
            double a = 0.0;
            for (int k = 0; k < lanes_per; ++k) a += scratch[k * nv + t];
            dst[t] = a;
        }
    }
    __syncthreads();
}

// seg_reduce: reduce per-thread partials `val[NV]` (thread t's right-hand
// side is t % ld) to per-block totals, then run the cross-block sum.
// Returns true in exactly one thread block per system, after which
// `out[v*ld + rhs]` (shared memory, NV*ld doubles) holds the system totals
// for every thread of that block.
//
// Ordering: the block's partial is written, the block synchronises, and one
// thread issues a GPU-scope fence and the counter increment; the block that
// sees the last count fences once more before reading the partials (.cg
// loads).  When a system has at most kRedDirect partial vectors the last
// block sums them directly (one serial stage); otherwise groups of
// kRedGroup blocks are summed first (two stages).
// Cross-block stage for block `b` of system `seg`, whose NV*ld totals are
// in out[] (shared memory).  Returns true in exactly one block per system,
// with the system totals in out[].  `scratch` holds blockDim.x doubles;
// requires blockDim.x % nvl == 0.
__device__ inline bool cross_blocks(int b, int seg, int nvl, const RedLayout& R, double* out,
                                    double* scratch) {
    const int t = threadIdx.x;
    __shared__ int s_last;
    const int nblk = R.seg_nblk[seg];
    const int lb = b - R.seg_blk0[seg];
    if (t < nvl) R.part1[(int64_t)b * nvl + t] = out[t];
    __syncthreads();
    if (nblk <= kRedDirect) {
        if (t == 0) {
            __threadfence();
            s_last = (atomicAdd(R.cnt2 + seg, 1) == nblk - 1);
        }
        __syncthreads();
        if (!s_last) return false;
        if (t == 0) __threadfence();
        __syncthreads();
        block_sum_vectors(R.part1 + (int64_t)R.seg_blk0[seg] * nvl, nblk, nvl, nvl, out, scratch);
        if (t == 0) R.cnt2[seg] = 0;
        return true;
    }
    const int g = R.seg_grp0[seg] + lb / kRedGroup;
    const int gsize = min(kRedGroup, nblk - (lb / kRedGroup) * kRedGroup);
    if (t == 0) {
        __threadfence();
        s_last = (atomicAdd(R.cnt1 + g, 1) == gsize - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    if (t == 0) __threadfence();
    __syncthreads();
    // 2) group sum
    const int gb0 = R.seg_blk0[seg] + (lb / kRedGroup) * kRedGroup;
    block_sum_vectors(R.part1 + (int64_t)gb0 * nvl, gsize, nvl, nvl, out, scratch);
    if (t == 0) R.cnt1[g] = 0;
    if (t < nvl) R.part2[(int64_t)g * nvl + t] = out[t];
    __syncthreads();
    const int ngrp = (nblk + kRedGroup - 1) / kRedGroup;
    if (t == 0) {
        __threadfence();
        s_last = (atomicAdd(R.cnt2 + seg, 1) == ngrp - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    if (t == 0) __threadfence();
    __syncthreads();
    // 3) system sum
    block_sum_vectors(R.part2 + (int64_t)R.seg_grp0[seg] * nvl, ngrp, nvl, nvl, out, scratch);
    if (t == 0) R.cnt2[seg] = 0;
    return true;
}

template <int NV>
__device__ bool seg_reduce(const double (&val)[NV], int ld, const RedLayout& R, double* out,
                           double* scratch, int& seg_out) {
    static_assert(NV <= kRedMaxNV, "partial buffers hold kRedMaxNV values per right-hand side");
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int warp = t >> 5;
    const int nwarp = blockDim.x >> 5;
    // 1) block totals per (v, rhs)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double x = val[v];
        for (int off = 16; off >= ld; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        // lanes 0..ld-1 hold the warp sums for rhs = lane
        if (lane < ld) scratch[warp * 32 + lane] = x;
        __syncthreads();
        if (t < ld) {
            double s = 0.0;
            for (int w = 0; w < nwarp; ++w) s += scratch[w * 32 + t];
            out[v * ld + t] = s;
        }
        __syncthreads();
    }
    const int b = blockIdx.x;
    const int seg = R.blk_seg[b];
    seg_out = seg;
    return cross_blocks(b, seg, NV * ld, R, out, scratch);
}

// After a system's finisher ran: count finished systems; the last one
// returns true (one thread block per launch) and resets the counter.
__device__ inline bool last_system(const RedLayout& R, int nseg) {
    if (nseg == 1) return true;
    __shared__ int s_last2;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last2 = (atomicAdd(R.cnt3, 1) == nseg - 1);
        if (s_last2) {
            R.cnt3[0] = 0;
            __threadfence();
        }
    }
    __syncthreads();
    return s_last2;
}

}  // namespace ams
