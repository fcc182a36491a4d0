// Diagnostic: the solve kernels convert between FP32 and FP64 on the
// integer pipe (f32_to_f64 / f64_to_f32 in kernels.cuh); this entry point
// compares those conversions with the hardware conversions over a caller's
// set of values.
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "ams_internal.h"
#include "kernels.cuh"

namespace ams {
namespace {

__global__ void k_check_conversions(const double* __restrict__ x, int64_t n, unsigned long long* bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    const float a = f64_to_f32(v), b = (float)v;
    // NaN payloads may differ between the two paths: compare NaN-ness only
    const bool narrow_ok = (isnan(a) && isnan(b)) || __float_as_uint(a) == __float_as_uint(b);
    const double c = f32_to_f64(b), d = (double)b;
    const bool widen_ok = (isnan(c) && isnan(d)) || __double_as_longlong(c) == __double_as_longlong(d);
    if (!narrow_ok) atomicAdd(bad, 1ull);
    if (!widen_ok) atomicAdd(bad + 1, 1ull);
}

}  // namespace
}  // namespace ams

extern "C" ams_status ams_check_conversions(const double* x, int64_t n, int64_t* narrow_bad, int64_t* widen_bad) {
    using namespace ams;
    if (n < 0 || (n > 0 && x == nullptr) || !narrow_bad || !widen_bad) {
        set_error("ams_check_conversions: invalid arguments");
        return AMS_ERR_INVALID_ARG;
    }
    unsigned long long* d_bad = nullptr;
    cudaError_t e = cudaMalloc(&d_bad, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(d_bad, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess && n > 0) {
        k_check_conversions<<<(unsigned)((n + 255) / 256), 256>>>(x, n, d_bad);
        e = cudaGetLastError();
    }
    unsigned long long h_bad[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h_bad, d_bad, sizeof(h_bad), cudaMemcpyDeviceToHost);
    if (d_bad) cudaFree(d_bad);
    if (e != cudaSuccess) {
        set_error(std::string("ams_check_conversions: ") + cudaGetErrorString(e));
        return AMS_ERR_CUDA;
    }
    *narrow_bad = (int64_t)h_bad[0];
    *widen_bad = (int64_t)h_bad[1];
    return AMS_OK;
}
