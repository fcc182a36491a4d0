// Kernels of the multiplicative two-grid cycle (the two-grid algorithm
// stated with the coarse space in Section 3.2: pre-smoothing, coarse-grid
// correction, post-smoothing), with the damped local solves
// S = omega sum_i R_i^T A_i^{-1} R_i as the smoother before and after the
// correction.  The local solves, the coarse substitutions and the
// prolongation are the additive path's kernels; this file adds the pieces
// the cycle needs in between:
//   k_tg_resid    w = r' - A v   (r' = r - alpha q formed as the local
//                                 solves form it; v the FP32/FP64 iterate)
//   k_tg_scale    z_f <- omega z_f
//   k_tg_restrict r_c = R_0 w    (restriction of a residual that is not
//                                 the local solves' input)
//   k_tg_combine  z_f <- x^2 + omega z_f
#include <algorithm>
#include <cstdint>

#include "ams_internal.h"
#include "kernels.cuh"
#include "launch.h"

namespace ams {

static unsigned tg_blocks_pw(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

template <typename T> __device__ __forceinline__ double tg_widen(T v);
template <> __device__ __forceinline__ double tg_widen<float>(float v) { return f32_to_f64(v); }
template <> __device__ __forceinline__ double tg_widen<double>(double v) { return v; }

// w = r' - A v over the element layout of the SpMV (block ranges of
// (row, rhs) elements, one system per block).  TA: the matrix values and
// the accumulation, FP64, or FP32 inside the reduced-precision apply (the
// cycle's residual is part of the preconditioner application; r' keeps
// the FP64 formation of the local solves' input).
template <int LD, typename TV, typename TA>
__global__ void __launch_bounds__(kRedThreads)
k_tg_resid(const int64_t* __restrict__ sell_ptr, const int32_t* __restrict__ sell_col,
           const TA* __restrict__ sell_val, const TV* __restrict__ v, const double* __restrict__ r,
           const double* __restrict__ q, RedLayout R, const CgScalars* __restrict__ sc,
           const SolveState* st, double* __restrict__ w) {
    pdl_wait();
    if (st != nullptr && st->done) return;
    const int rhs = threadIdx.x % LD;
    double alpha = 0.0;
    bool upd = false;
    if (q != nullptr) {
        const CgScalars c = sc[(int64_t)R.blk_seg[blockIdx.x] * LD + rhs];
        upd = c.active != 0;
        if (upd) alpha = c.rho / c.pq;
    }
    const int64_t lo = R.blk_lo[blockIdx.x], hi = R.blk_lo[blockIdx.x + 1];
    for (int64_t e = lo + threadIdx.x; e < hi; e += kRedThreads) {
        const int64_t row = e / LD;
        const int64_t sl = row >> 5;
        const int lane = (int)(row & 31);
        const int64_t b0 = __ldg(sell_ptr + sl);
        const int width = (int)((__ldg(sell_ptr + sl + 1) - b0) >> 5);
        TA acc = TA(0);
        for (int j = 0; j < width; ++j) {
            const int64_t o = b0 + 32 * j + lane;
            const TV vj = v[(int64_t)__ldg(sell_col + o) * LD + rhs];
            if constexpr (sizeof(TA) == 8) acc = fma(__ldg(sell_val + o), tg_widen<TV>(vj), acc);
            else acc = fmaf(__ldg(sell_val + o), (float)vj, acc);
        }
        const double rv = upd ? fma(-alpha, q[e], r[e]) : r[e];
        w[e] = rv - tg_widen<TA>(acc);
    }
}

template <typename TF>
__global__ void k_tg_scale(TF* __restrict__ zf, double omega, int64_t n, const SolveState* st) {
    if (st != nullptr && st->done) return;
    // in the apply precision (FP32 for the reduced-precision modes)
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        zf[e] = (TF)omega * zf[e];
}

template <typename TF>
__global__ void k_tg_combine(TF* __restrict__ zf, const TF* __restrict__ x2, double omega, int64_t n,
                             const SolveState* st) {
    if (st != nullptr && st->done) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (sizeof(TF) == 8) zf[e] = fma(omega, zf[e], x2[e]);
        else zf[e] = fmaf((float)omega, zf[e], x2[e]);   // apply precision (x2 = z, stored in it)
    }
}

// r_c[(coff + k) ld + rhs] = sum over the subdomain's rows of
// Psi_i[row][k] w[row, rhs]; one warp per (subdomain, rhs).
template <typename TF, typename TP, int MM>
__global__ void __launch_bounds__(256)
k_tg_restrict(const SubInfo* __restrict__ subs, int nsub, const TP* __restrict__ psi,
              const double* __restrict__ w, TF* __restrict__ rc, int ld, const SolveState* st) {
    if (st != nullptr && st->done) return;
    const int lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (gw >= (int64_t)nsub * ld) return;
    const int sub = (int)(gw / ld), rhs = (int)(gw % ld);
    const SubInfo S = subs[sub];
    const int m = S.m;
    if (m == 0) return;
    double acc[MM];
#pragma unroll
    for (int k = 0; k < MM; ++k) acc[k] = 0.0;
    for (int i = lane; i < S.n; i += 32) {
        const double wv = w[(S.row0 + i) * ld + rhs];
        const TP* pr = psi + S.psi_off + (int64_t)i * m;
#pragma unroll
        for (int k = 0; k < MM; ++k)
            if (k < m) acc[k] = fma(to_d(pr[k]), wv, acc[k]);
    }
#pragma unroll
    for (int k = 0; k < MM; ++k) {
        double a = acc[k];
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (lane == 0 && k < m) rc[(S.coff + k) * ld + rhs] = (TF)a;
    }
}

// r_c = R_0 w for 8 or more right-hand sides: one block per subdomain,
// thread (rhs, row group) reads whole rows of w (all right-hand sides of a
// row are contiguous, so the reads coalesce) and accumulates the m_i mode
// sums of its rows in the apply precision; the row groups are summed in a
// fixed order in shared memory.
template <typename TF, typename TP, int MM, int LD>
__global__ void __launch_bounds__(256)
k_tg_restrict_rows(const SubInfo* __restrict__ subs, const TP* __restrict__ psi, const double* __restrict__ w,
                   TF* __restrict__ rc, const SolveState* st) {
    if (st != nullptr && st->done) return;
    constexpr int RG = 256 / LD;                     // row groups
    using A = typename Acc<TF>::type;
    __shared__ A part[RG][MM][LD];
    const SubInfo S = subs[blockIdx.x];
    const int m = S.m;
    if (m == 0) return;
    const int rhs = threadIdx.x % LD, rg = threadIdx.x / LD;
    A acc[MM];
#pragma unroll
    for (int k = 0; k < MM; ++k) acc[k] = A(0);
    for (int i = rg; i < S.n; i += RG) {
        const A wv = (A)w[(S.row0 + i) * LD + rhs];
        const TP* pr = psi + S.psi_off + (int64_t)i * m;
#pragma unroll
        for (int k = 0; k < MM; ++k)
            if (k < m) acc[k] += (A)to_d(pr[k]) * wv;
    }
#pragma unroll
    for (int k = 0; k < MM; ++k) part[rg][k][rhs] = acc[k];
    __syncthreads();
    for (int o = threadIdx.x; o < m * LD; o += 256) {
        const int k = o / LD, h = o % LD;
        A sum = A(0);
        for (int g = 0; g < RG; ++g) sum += part[g][k][h];
        rc[(S.coff + k) * LD + h] = (TF)sum;
    }
}

// ---------------------------------------------------------------------------
// Damping of the cycle: power steps on T = (sum_i R_i^T A_i^{-1} R_i) A.
// T is self-adjoint in the A inner product, so with y = A x and z = S y the
// Rayleigh quotient (y . z) / (x . y) rises towards lambda_max(T) per
// system.  Partials cover kRowAlign rows each (one system per block, since
// systems are padded to that many rows) and are summed in block order.
// ---------------------------------------------------------------------------
template <typename TZ>
__global__ void __launch_bounds__(256)
k_pw_partials(const double* __restrict__ x, const double* __restrict__ y, const TZ* __restrict__ z, int64_t nrows,
              double* __restrict__ part) {
    __shared__ double s[3][256];
    const int64_t lo = blockIdx.x * (int64_t)kRowAlign;
    const int64_t hi = lo + kRowAlign < nrows ? lo + kRowAlign : nrows;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += 256) {
        const double yi = y[i], zi = tg_widen<TZ>(z[i]);
        a = fma(x[i], yi, a);
        b = fma(yi, zi, b);
        c = fma(zi, zi, c);
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    s[2][threadIdx.x] = c;
    __syncthreads();
    for (int h = 128; h >= 1; h >>= 1) {
        if (threadIdx.x < h)
            for (int k = 0; k < 3; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 3) part[3 * (int64_t)blockIdx.x + threadIdx.x] = s[threadIdx.x][0];
}

// Per system: sums of its blocks' partials (x.y, y.z, z.z) and 1/||z||.
__global__ void k_pw_finish(const double* __restrict__ part, const int64_t* __restrict__ sys_blk0, int nsys,
                            double* __restrict__ out, double* __restrict__ inv_norm) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int64_t k = sys_blk0[s]; k < sys_blk0[s + 1]; ++k) {
        a += part[3 * k];
        b += part[3 * k + 1];
        c += part[3 * k + 2];
    }
    out[3 * s] = a;
    out[3 * s + 1] = b;
    out[3 * s + 2] = c;
    inv_norm[s] = c > 0.0 ? 1.0 / sqrt(c) : 0.0;
}

// x = z / ||z|| (per system)
template <typename TZ>
__global__ void k_pw_normalize(const TZ* __restrict__ z, const int32_t* __restrict__ blk_sys,
                               const double* __restrict__ inv_norm, int64_t nrows, double* __restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrows; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = tg_widen<TZ>(z[i]) * inv_norm[blk_sys[i / kRowAlign]];
}

void launch_power_step(cudaStream_t s, int prec, const double* x, const double* y, const void* z, int64_t nrows,
                       const int64_t* sys_blk0, const int32_t* blk_sys, int nsys, double* part, double* out,
                       double* inv_norm, double* x_next) {
    const unsigned nblk = (unsigned)((nrows + kRowAlign - 1) / kRowAlign);
    if (prec == AMS_PREC_FP64) {
        k_pw_partials<double><<<nblk, 256, 0, s>>>(x, y, (const double*)z, nrows, part);
        k_pw_finish<<<(nsys + 127) / 128, 128, 0, s>>>(part, sys_blk0, nsys, out, inv_norm);
        k_pw_normalize<double><<<tg_blocks_pw(nrows), 256, 0, s>>>((const double*)z, blk_sys, inv_norm, nrows, x_next);
    } else {
        k_pw_partials<float><<<nblk, 256, 0, s>>>(x, y, (const float*)z, nrows, part);
        k_pw_finish<<<(nsys + 127) / 128, 128, 0, s>>>(part, sys_blk0, nsys, out, inv_norm);
        k_pw_normalize<float><<<tg_blocks_pw(nrows), 256, 0, s>>>((const float*)z, blk_sys, inv_norm, nrows, x_next);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int LD, typename TV>
static void resid_ld_t(const LaunchCtx& L, const TV* v, const ResidIn& in, double* w) {
    if (L.sell_val32 != nullptr)
        launch_kernel(false, k_tg_resid<LD, TV, float>, dim3((unsigned)L.nblk), dim3(kRedThreads), 0, L.stream,
                      L.sell_ptr, L.sell_col, L.sell_val32, v, in.r, in.q, L.red, in.sc, (const SolveState*)L.st, w);
    else
        launch_kernel(false, k_tg_resid<LD, TV, double>, dim3((unsigned)L.nblk), dim3(kRedThreads), 0, L.stream,
                      L.sell_ptr, L.sell_col, L.sell_val, v, in.r, in.q, L.red, in.sc, (const SolveState*)L.st, w);
}
template <int LD>
static void resid_ld(const LaunchCtx& L, const void* v, int v_kind, const ResidIn& in, double* w) {
    if (v_kind == 0) resid_ld_t<LD, float>(L, (const float*)v, in, w);
    else resid_ld_t<LD, double>(L, (const double*)v, in, w);
}
void launch_tg_resid(const LaunchCtx& L, const void* v, int v_is_fp64, const ResidIn& in, double* w) {
    switch (L.ld) {
        case 1: resid_ld<1>(L, v, v_is_fp64, in, w); break;
        case 2: resid_ld<2>(L, v, v_is_fp64, in, w); break;
        case 4: resid_ld<4>(L, v, v_is_fp64, in, w); break;
        case 8: resid_ld<8>(L, v, v_is_fp64, in, w); break;
        case 16: resid_ld<16>(L, v, v_is_fp64, in, w); break;
        default: resid_ld<32>(L, v, v_is_fp64, in, w); break;
    }
}

static unsigned tg_blocks(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (unsigned)std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 16);
}

__global__ void k_round_to_f32(const double* __restrict__ a, int64_t n, float* __restrict__ b) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        b[e] = __double2float_rn(a[e]);
}

void launch_round_to_f32(cudaStream_t s, const double* a, int64_t n, float* b) {
    if (n > 0) k_round_to_f32<<<tg_blocks(n), 256, 0, s>>>(a, n, b);
}

void launch_tg_scale(const LaunchCtx& L, int prec, void* zf, double omega, int64_t n) {
    if (prec == AMS_PREC_FP64)
        k_tg_scale<double><<<tg_blocks(n), 256, 0, L.stream>>>((double*)zf, omega, n, L.st);
    else
        k_tg_scale<float><<<tg_blocks(n), 256, 0, L.stream>>>((float*)zf, omega, n, L.st);
}

void launch_tg_combine(const LaunchCtx& L, int prec, void* zf, const void* x2, double omega, int64_t n) {
    if (prec == AMS_PREC_FP64)
        k_tg_combine<double><<<tg_blocks(n), 256, 0, L.stream>>>((double*)zf, (const double*)x2, omega, n, L.st);
    else
        k_tg_combine<float><<<tg_blocks(n), 256, 0, L.stream>>>((float*)zf, (const float*)x2, omega, n, L.st);
}

template <typename TF, typename TP, int MM>
static bool restrict_rows(const LaunchCtx& L, const void* psi, const double* w, void* rc) {
    switch (L.ld) {
        case 8: k_tg_restrict_rows<TF, TP, MM, 8><<<L.nsub, 256, 0, L.stream>>>(L.subs, (const TP*)psi, w, (TF*)rc, L.st); return true;
        case 16: k_tg_restrict_rows<TF, TP, MM, 16><<<L.nsub, 256, 0, L.stream>>>(L.subs, (const TP*)psi, w, (TF*)rc, L.st); return true;
        case 32: k_tg_restrict_rows<TF, TP, MM, 32><<<L.nsub, 256, 0, L.stream>>>(L.subs, (const TP*)psi, w, (TF*)rc, L.st); return true;
        default: return false;
    }
}

template <typename TF, typename TP>
static void restrict_t(const LaunchCtx& L, const void* psi, const double* w, void* rc, int mmax) {
    if (L.nsub > 0 && (mmax > 8 ? restrict_rows<TF, TP, kMaxM>(L, psi, w, rc) : restrict_rows<TF, TP, 8>(L, psi, w, rc)))
        return;
    const int64_t warps = (int64_t)L.nsub * L.ld;
    const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
    if (mmax > 8)
        k_tg_restrict<TF, TP, kMaxM><<<blocks, 256, 0, L.stream>>>(L.subs, L.nsub, (const TP*)psi, w, (TF*)rc,
                                                                   L.ld, L.st);
    else
        k_tg_restrict<TF, TP, 8><<<blocks, 256, 0, L.stream>>>(L.subs, L.nsub, (const TP*)psi, w, (TF*)rc, L.ld,
                                                              L.st);
}
void launch_tg_restrict(const LaunchCtx& L, int prec, const void* psi, const double* w, void* rc, int mmax) {
    if (prec == AMS_PREC_FP64) restrict_t<double, double>(L, psi, w, rc, mmax);
    else if (prec == AMS_PREC_FP32) restrict_t<float, float>(L, psi, w, rc, mmax);
    else restrict_t<float, __nv_bfloat16>(L, psi, w, rc, mmax);
}

}  // namespace ams
