// Allocation-free CSR SpMV with a fused dot product.
//
// Some callers cannot allocate device memory at the point where they need a
// matrix-vector product: code running while another framework captures a
// CUDA graph (cudaMalloc is not permitted during capture), code built on a
// host framework that hands out all device memory from its own fixed pool,
// and real-time or embedded callers that forbid allocation after start-up.
// This entry point needs no handle and allocates nothing: the per-block
// partial sums of the dot product and the arrival counter live in one
// file-scope device array of fixed size, which every GPU that loads the
// library keeps until the process exits.
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "ams_internal.h"

namespace ams {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaRowsPerThread = 4;
constexpr int kNaRowsPerBlock = kNaThreads * kNaRowsPerThread;   // 1024
constexpr int kNaMaxBlocks = 8192;                               // n <= 8,388,608 rows
constexpr int64_t kNaMaxRows = (int64_t)kNaMaxBlocks * kNaRowsPerBlock;

// [0, kNaMaxBlocks): one partial dot per thread block; [kNaMaxBlocks]: the
// arrival counter (as a 64-bit integer).  64 KB + 256 B per device.
static __device__ __align__(256) double g_noalloc_scratch[kNaMaxBlocks + 32];

__global__ void __launch_bounds__(kNaThreads)
k_csr_spmv_dot_noalloc(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                       const double* __restrict__ vals, const double* __restrict__ x, double* __restrict__ y,
                       double* __restrict__ xy, double* __restrict__ scratch) {
    __shared__ double red[kNaThreads];
    __shared__ int s_last;
    const int t = threadIdx.x;
    double dot = 0.0;
#pragma unroll
    for (int k = 0; k < kNaRowsPerThread; ++k) {
        const int64_t r = (int64_t)blockIdx.x * kNaRowsPerBlock + t + k * kNaThreads;
        if (r < n) {
            double s = 0.0;
            for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) s += vals[e] * x[colind[e]];
            y[r] = s;
            dot += x[r] * s;
        }
    }
    // block total in a fixed-shape tree
    red[t] = dot;
    __syncthreads();
    for (int h = kNaThreads / 2; h >= 1; h >>= 1) {
        if (t < h) red[t] += red[t + h];
        __syncthreads();
    }
    unsigned long long* counter = reinterpret_cast<unsigned long long*>(scratch + kNaMaxBlocks);
    if (t == 0) {
        scratch[blockIdx.x] = red[0];
        __threadfence();
        s_last = (atomicAdd(counter, 1ull) == (unsigned long long)(gridDim.x - 1));
        if (s_last) __threadfence();
    }
    __syncthreads();
    if (!s_last) return;
    // the last block sums the partials in block order (deterministic)
    double s = 0.0;
    for (int b = t; b < (int)gridDim.x; b += kNaThreads) s += __ldcg(scratch + b);
    red[t] = s;
    __syncthreads();
    for (int h = kNaThreads / 2; h >= 1; h >>= 1) {
        if (t < h) red[t] += red[t + h];
        __syncthreads();
    }
    if (t == 0) {
        *xy = red[0];
        *counter = 0ull;
    }
}

// Identity of the current CUDA context (cuCtxGetId: unique for the life of
// the process, so a context re-created after cudaDeviceReset gets a new
// one), through the driver entry points the runtime exposes; 0 if the
// driver does not provide it.
typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);

unsigned long long current_context_id() {
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (PfnCtxGetCurrent)fn;
        fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (PfnCtxGetId)fn;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS)
        return id;
    return 0;
}

// Device address of the scratch array, resolved once per device and
// context: a device reset ends the context that held the old address, and
// the first call in the new context resolves it again.
struct ScratchAddr {
    unsigned long long ctx = 0;
    double* ptr = nullptr;
};
std::mutex g_na_mu;
std::vector<ScratchAddr> g_na_ptr;

ams_status noalloc_scratch(int dev, double** out) {
    std::lock_guard<std::mutex> lock(g_na_mu);
    if ((int)g_na_ptr.size() <= dev) g_na_ptr.resize(dev + 1);
    const unsigned long long ctx = current_context_id();
    ScratchAddr& a = g_na_ptr[dev];
    if (!a.ptr || a.ctx != ctx) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error(std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e));
            return AMS_ERR_CUDA;
        }
        a.ptr = (double*)p;
        a.ctx = ctx;
    }
    *out = a.ptr;
    return AMS_OK;
}

}  // namespace
}  // namespace ams

extern "C" ams_status ams_csr_spmv_dot_noalloc(int64_t n, const int64_t* rowptr, const int32_t* colind,
                                               const double* vals, const double* x, double* y, double* xy,
                                               void* stream) {
    using namespace ams;
    if (n < 0 || n > kNaMaxRows) {
        set_error("ams_csr_spmv_dot_noalloc: n = " + std::to_string(n) + " exceeds the scratch limit of " +
                  std::to_string(kNaMaxRows) + " rows");
        return AMS_ERR_INVALID_ARG;
    }
    if (!rowptr || !colind || !vals || !x || !y || !xy) {
        set_error("ams_csr_spmv_dot_noalloc: null pointer");
        return AMS_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return AMS_ERR_CUDA;
    }
    double* scratch = nullptr;
    const ams_status st = noalloc_scratch(dev, &scratch);
    if (st != AMS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        e = cudaMemsetAsync(xy, 0, sizeof(double), s);
    } else {
        // the arrival counter must start at zero
        e = cudaMemsetAsync(scratch + kNaMaxBlocks, 0, sizeof(unsigned long long), s);
        if (e == cudaSuccess) {
            const unsigned grid = (unsigned)((n + kNaRowsPerBlock - 1) / kNaRowsPerBlock);
            k_csr_spmv_dot_noalloc<<<grid, kNaThreads, 0, s>>>(n, rowptr, colind, vals, x, y, xy, scratch);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) {
        set_error(std::string("ams_csr_spmv_dot_noalloc: ") + cudaGetErrorString(e));
        return AMS_ERR_CUDA;
    }
    return AMS_OK;
}
