// Warp-level tensor-core products in TF32 with FP32 accumulation, and the
// head/tail split that keeps FP32 accuracy: x = head + tail with both
// TF32, a*b summed as tail_a*head_b + head_a*tail_b + head_a*head_b (the
// dropped tail*tail term lies below FP32 rounding).
#pragma once

#include <cstdint>

namespace ams {

// TF32 value (as its 32-bit pattern) nearest to x
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return r;
}
// x = head + tail (+ below FP32 resolution), head and tail TF32
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}
// d += a b, a 16x8 (row), b 8x8 (col), TF32 in, FP32 accumulate
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

}  // namespace ams
