// Setup-phase kernels (FP64) of the AMS preconditioner.
//
//  * local matrices A_i = R_i A R_i^T and \hat A_i, S_i (Section 3.2) in a
//    band layout, their band Cholesky factors, and the packing of a factor
//    into the block-row layout of the solve (inverted 32x32 diagonal blocks);
//  * the local generalized eigenproblems \hat A_i psi = lambda S_i psi
//    (Eq. algebraic-eigenproblem) by shift-invert subspace iteration with
//    Rayleigh-Ritz on the pencil, using the factor of \hat A_i + sigma S_i;
//  * the Galerkin product A_0 = R_0 A R_0^T (Section 3.1);
//  * extraction of the nested-dissection blocks of L_c^{-1} for the coarse
//    solve from the dense inverse factor.
#include <cstdint>
#include <cstdio>

#include "ams_internal.h"
#include "kernels.cuh"
#include "launch.h"

namespace ams {

// band element (i, j), j in [i - bw, i]
__device__ __forceinline__ int64_t bidx(int64_t i, int64_t j, int bw) {
    return i * (bw + 1) + (j - i + bw);
}

// ---------------------------------------------------------------------------
__global__ void k_band_assemble(const SubInfo* __restrict__ subs, const int64_t* __restrict__ band_off,
                                const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                const double* __restrict__ vals, double* __restrict__ band, int mode,
                                double sigma, double* __restrict__ S, double* __restrict__ ahat_diag) {
    const SubInfo Sb = subs[blockIdx.x];
    const int bw = 32 * Sb.c;
    double* B = band + band_off[blockIdx.x];
    const int N = 32 * Sb.nb;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double* row = B + (int64_t)i * (bw + 1);
        for (int t = 0; t <= bw; ++t) row[t] = 0.0;
        if (i >= Sb.n) {
            row[bw] = 1.0;
            continue;
        }
        const int64_t g = Sb.row0 + i;
        double off = 0.0, dA = 0.0;
        for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) {
            const int64_t j = (int64_t)colind[e] - Sb.row0;
            const double v = vals[e];
            if (j == i) {
                dA = v;
            } else if (j >= 0 && j < Sb.n) {
                off += v;
                if (j < i) row[j - i + bw] = v;
            }
        }
        const double ah = -off;                   // \hat A_ii: minus the off-diagonal row sum
        const double s = (ah != 0.0) ? ah : dA;   // S_ii (zero weight -> A_ii)
        row[bw] = (mode == 0) ? dA : ah + sigma * s;
        if (S != nullptr) S[g] = s;
        if (ahat_diag != nullptr) ahat_diag[g] = ah;
    }
}

// Right-looking band Cholesky, one thread block per subdomain, in place.
__global__ void k_band_cholesky(const SubInfo* __restrict__ subs, const int64_t* __restrict__ band_off,
                                double* __restrict__ band, int32_t* status) {
    const SubInfo Sb = subs[blockIdx.x];
    const int bw = 32 * Sb.c;
    double* B = band + band_off[blockIdx.x];
    const int N = 32 * Sb.nb;
    __shared__ double s_d;
    for (int j = 0; j < N; ++j) {
        if (threadIdx.x == 0) {
            double a = B[bidx(j, j, bw)];
            if (!(a > 0.0) || !isfinite(a)) {
                atomicExch(status, (int)AMS_ERR_NOT_SPD);
                a = 1.0;
            }
            a = sqrt(a);
            B[bidx(j, j, bw)] = a;
            s_d = a;
        }
        __syncthreads();
        const double d = s_d;
        const int iend = min(j + bw, N - 1);
        for (int t = threadIdx.x; t < iend - j; t += blockDim.x) {
            const int i = j + 1 + t;
            B[bidx(i, j, bw)] /= d;
        }
        __syncthreads();
        const int w = iend - j;
        for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
            const int a = t / w, b = t % w;
            if (b > a) continue;
            const int i = j + 1 + a, k = j + 1 + b;
            B[bidx(i, k, bw)] -= B[bidx(i, j, bw)] * B[bidx(k, j, bw)];
        }
        __syncthreads();
    }
}

// One warp per (subdomain, block row): inverse of the 32x32 diagonal block
// by forward substitution on the identity (lane = column), then the packed
// block row [M | dense tiles | pivots] in FP64 and/or FP32.
__global__ void k_band_pack(const SubInfo* __restrict__ subs, const int64_t* __restrict__ band_off,
                            const int2* __restrict__ work, const double* __restrict__ band,
                            const int64_t* __restrict__ out_off, double* __restrict__ out64,
                            float* __restrict__ out32) {
    const int2 wk = work[blockIdx.x];
    const int s = wk.x, K = wk.y;
    const SubInfo Sb = subs[s];
    const int c = Sb.c, bw = 32 * c;
    const double* B = band + band_off[s];
    const int lane = threadIdx.x;
    const int64_t r0 = 32LL * K;
    // column `lane` of L_KK^{-1}
    double x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        double acc = (i == lane) ? 1.0 : 0.0;
#pragma unroll
        for (int k = 0; k < i; ++k) acc -= B[bidx(r0 + i, r0 + k, bw)] * x[k];
        x[i] = (i >= lane) ? acc / B[bidx(r0 + i, r0 + i, bw)] : 0.0;
    }
    const int64_t brs = blockrow_elems(c);
    const int64_t o = out_off[s] + (int64_t)K * brs;
    auto put = [&](int64_t idx, double v) {
        if (out64) out64[o + idx] = v;
        if (out32) out32[o + idx] = (float)v;
    };
    // strict lower part of M: Dinv[r][lane] for r > lane ; pivots
#pragma unroll
    for (int r = 0; r < 32; ++r)
        if (r > lane) put(tile_idx(r, lane), x[r]);
    put((int64_t)c * 1024 + lane, x[lane]);
    // upper part of M: L_{K,K-c}[r][q], q >= r ; lane = q
    const int64_t cb = 32LL * (K - c);
    for (int r = 0; r <= lane; ++r) {
        const int64_t col = cb + lane, row = r0 + r;
        const double v = (col >= 0 && col >= row - bw) ? B[bidx(row, col, bw)] : 0.0;
        put(tile_idx(r, lane), v);
    }
    // dense tiles t = 1..c-1 : L_{K,K-c+t}
    for (int t = 1; t < c; ++t) {
        const int64_t cbt = 32LL * (K - c + t);
        for (int r = 0; r < 32; ++r) {
            const int64_t col = cbt + lane, row = r0 + r;
            const double v = (col >= 0 && col >= row - bw) ? B[bidx(row, col, bw)] : 0.0;
            put((int64_t)t * 1024 + tile_idx(r, lane), v);
        }
    }
}

// Same factor, TMA tile layout: forward tiles row-major, backward tiles
// transposed, reciprocal pivots per row (FP32).  One warp per (subdomain,
// block row); lane = tile column.
__global__ void k_band_pack_tiles(const SubInfo* __restrict__ subs, const int64_t* __restrict__ band_off,
                                  const int2* __restrict__ work, const double* __restrict__ band,
                                  const int64_t* __restrict__ out_off, float* __restrict__ fwd,
                                  float* __restrict__ bwd, float* __restrict__ piv) {
    const int2 wk = work[blockIdx.x];
    const int s = wk.x, K = wk.y;
    const SubInfo Sb = subs[s];
    const int c = Sb.c, bw = 32 * c;
    const double* B = band + band_off[s];
    const int lane = threadIdx.x;
    const int64_t r0 = 32LL * K;
    double x[32];   // column `lane` of L_KK^{-1}
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        double acc = (i == lane) ? 1.0 : 0.0;
#pragma unroll
        for (int k = 0; k < i; ++k) acc -= B[bidx(r0 + i, r0 + k, bw)] * x[k];
        x[i] = (i >= lane) ? acc / B[bidx(r0 + i, r0 + i, bw)] : 0.0;
    }
    auto Lval = [&](int64_t row, int64_t col) -> double {
        return (col >= 0 && col >= row - bw && col <= row) ? B[bidx(row, col, bw)] : 0.0;
    };
    const int64_t tbase = out_off[s] + (int64_t)K * c * 1024;
    // tile 0: M_K (upper part from L_{K,K-c}, strict lower part from L_KK^{-1})
    const int64_t cb = 32LL * (K - c);
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const float v = (float)(lane >= r ? Lval(r0 + r, cb + lane) : x[r]);
        fwd[tbase + r * 32 + lane] = v;
        bwd[tbase + lane * 32 + r] = v;
    }
    for (int t = 1; t < c; ++t) {
        const int64_t cbt = 32LL * (K - c + t);
        for (int r = 0; r < 32; ++r) {
            const float v = (float)Lval(r0 + r, cbt + lane);
            fwd[tbase + (int64_t)t * 1024 + r * 32 + lane] = v;
            bwd[tbase + (int64_t)t * 1024 + lane * 32 + r] = v;
        }
    }
    const int64_t row = r0 + lane;
    if (row < Sb.n) {
        double d = 0.0;
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if (i == lane) d = x[i];
        piv[Sb.row0 + row] = (float)d;
    }
}

// ---------------------------------------------------------------------------
// eigensolver pieces
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__global__ void k_eig_init(const SubInfo* __restrict__ subs, int P, double* __restrict__ X) {
    const SubInfo Sb = subs[blockIdx.x];
    for (int t = threadIdx.x; t < Sb.n * P; t += blockDim.x) {
        const int i = t / P, a = t % P;
        double v = 0.0;
        if (a < Sb.p) {
            if (a == 0) {
                v = 1.0;
            } else {
                const uint64_t h = splitmix64(((uint64_t)(Sb.row0 + i) << 6) ^ (uint64_t)a);
                v = (double)(h >> 11) * (2.0 / 9007199254740992.0) - 1.0;
            }
        }
        X[(Sb.row0 + i) * P + a] = v;
    }
}

// (\hat A Y)_i = ahat_ii Y_i + sum_{j in Omega, j != i} A_ij Y_j
__device__ inline void ahat_mult(const SubInfo& Sb, int P, const int64_t* rowptr, const int32_t* colind,
                                 const double* vals, const double* ahat_diag, const double* Y,
                                 double* AY) {
    for (int t = threadIdx.x; t < Sb.n * P; t += blockDim.x) {
        const int i = t / P, a = t % P;
        const int64_t g = Sb.row0 + i;
        double s = ahat_diag[g] * Y[g * P + a];
        for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) {
            const int64_t j = colind[e];
            if (j != g && j >= Sb.row0 && j < Sb.row0 + Sb.n) s += vals[e] * Y[j * P + a];
        }
        AY[g * P + a] = s;
    }
}

// Rayleigh-Ritz on span(Y) for the pencil (\hat A, S):
//   G = Y^T S Y = R^T R,  C = R^{-T} (Y^T \hat A Y) R^{-1} = W Theta W^T,
//   T = R^{-1} W  (new basis X = Y T is S-orthonormal, Ritz values Theta).
// orth_only = 1: only the S-orthonormalisation T = R^{-1} (same span; no
// Ritz values), for the subspace iterations between convergence checks.
// One thread block per subdomain; the small dense work is done by warp 0,
// the Jacobi rotations by the whole block.
__global__ void __launch_bounds__(256)
k_eig_rr(const SubInfo* __restrict__ subs, int P, const int64_t* __restrict__ rowptr,
         const int32_t* __restrict__ colind, const double* __restrict__ vals,
         const double* __restrict__ S, const double* __restrict__ ahat_diag,
         const double* __restrict__ Y, double* __restrict__ AY, double* __restrict__ Tout,
         double* __restrict__ theta, int32_t* status, int orth_only) {
    const SubInfo Sb = subs[blockIdx.x];
    const int p = Sb.p;
    if (p == 0) return;
    extern __shared__ double sm[];
    double* G = sm;                 // P*P
    double* H = G + P * P;          // P*P
    double* W = H + P * P;          // P*P
    double* Rm = W + P * P;         // P*P (R, then R^{-1})
    double* ev = Rm + P * P;        // P
    if (!orth_only) ahat_mult(Sb, P, rowptr, colind, vals, ahat_diag, Y, AY);
    __syncthreads();
    // Gram matrices (upper triangles): one warp per pair (a, b), lanes over
    // the subdomain's rows, partial sums combined by a fixed shuffle tree
    {
        const int wid = threadIdx.x >> 5, wl = threadIdx.x & 31, nw = blockDim.x >> 5;
        const int npairs = p * (p + 1) / 2;
        for (int pr = wid; pr < npairs; pr += nw) {
            int a = 0, rem = pr;
            while (rem >= p - a) {
                rem -= p - a;
                ++a;
            }
            const int b = a + rem;
            double g = 0.0, h = 0.0;
            for (int i = wl; i < Sb.n; i += 32) {
                const int64_t r = Sb.row0 + i;
                const double ya = Y[r * P + a];
                g += S[r] * ya * Y[r * P + b];
                if (!orth_only) h += ya * AY[r * P + b];
            }
            for (int off = 16; off > 0; off >>= 1) {
                g += __shfl_xor_sync(0xffffffffu, g, off);
                h += __shfl_xor_sync(0xffffffffu, h, off);
            }
            if (wl == 0) {
                G[a * P + b] = g;
                G[b * P + a] = g;
                H[a * P + b] = h;
                H[b * P + a] = h;
            }
        }
    }
    __syncthreads();
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < 32) {
    // symmetrise H (Y^T \hat A Y is symmetric up to rounding)
    for (int a = 0; a < p; ++a) {
        if (lane < p && lane > a) {
            const double v = 0.5 * (H[a * P + lane] + H[lane * P + a]);
            H[a * P + lane] = v;
            H[lane * P + a] = v;
        }
    }
    __syncwarp();
    // Cholesky G = R^T R (R upper), by columns; R stored in Rm
    for (int j = 0; j < p; ++j) {
        if (lane == 0) {
            double d = G[j * P + j];
            for (int k = 0; k < j; ++k) d -= Rm[k * P + j] * Rm[k * P + j];
            if (!(d > 0.0)) {
                atomicExch(status, 1);
                d = 1e-300;
            }
            Rm[j * P + j] = sqrt(d);
        }
        __syncwarp();
        // one reciprocal per pivot, taken by lane 0 and broadcast (an FP64
        // division per lane would occupy the narrow FP64 pipe 31 times over)
        double rpiv = 0.0;
        if (lane == 0) rpiv = 1.0 / Rm[j * P + j];
        rpiv = __shfl_sync(0xffffffffu, rpiv, 0);
        if (lane > j && lane < p) {
            double v = G[j * P + lane];
            for (int k = 0; k < j; ++k) v -= Rm[k * P + j] * Rm[k * P + lane];
            Rm[j * P + lane] = v * rpiv;
        }
        if (lane < j) Rm[j * P + lane] = 0.0;   // lower part zero
        __syncwarp();
    }
    // R^{-1} (upper) by columns: lane = column; reciprocal pivots first
    // (one division per lane), then multiplications only
    if (lane < p) ev[lane] = 1.0 / Rm[lane * P + lane];
    __syncwarp();
    if (lane < p) {
        const int c = lane;
        double col[32];
        for (int i = 0; i < 32; ++i) col[i] = 0.0;
        for (int i = c; i >= 0; --i) {
            double v = (i == c) ? 1.0 : 0.0;
            for (int k = i + 1; k <= c; ++k) v -= Rm[i * P + k] * col[k];
            col[i] = v * ev[i];
        }
        __syncwarp(0xffffffffu >> (32 - p));
        for (int i = 0; i < p; ++i) W[i * P + c] = col[i];       // W temporarily holds R^{-1}
    }
    __syncwarp();
    for (int t = lane; t < p * p; t += 32) Rm[t / p * P + t % p] = W[t / p * P + t % p];
    __syncwarp();
    if (orth_only) {   // T = R^{-1}  (P x P, zero beyond p)
        double* T = Tout + (int64_t)blockIdx.x * P * P;
        for (int t = lane; t < P * P; t += 32) {
            const int a = t / P, b = t % P;
            T[t] = (a < p && b < p && a <= b) ? Rm[a * P + b] : 0.0;
        }
    }
    }   // tid < 32
    __syncthreads();
    if (orth_only) return;
    if (tid < 32) {
    // C = R^{-T} H R^{-1}: first HR = H R^{-1} into W, then C into G
    for (int t = lane; t < p * p; t += 32) {
        const int a = t / p, b = t % p;
        double s = 0.0;
        for (int k = 0; k <= b; ++k) s += H[a * P + k] * Rm[k * P + b];
        W[a * P + b] = s;
    }
    __syncwarp();
    for (int t = lane; t < p * p; t += 32) {
        const int a = t / p, b = t % p;
        double s = 0.0;
        for (int k = 0; k <= a; ++k) s += Rm[k * P + a] * W[k * P + b];
        G[a * P + b] = s;
    }
    __syncwarp();
    for (int t = lane; t < p * p; t += 32) {       // exact symmetry, W = I
        const int a = t / p, b = t % p;
        if (b > a) {
            const double v = 0.5 * (G[a * P + b] + G[b * P + a]);
            G[a * P + b] = v;
            G[b * P + a] = v;
        }
        W[a * P + b] = (a == b) ? 1.0 : 0.0;
    }
    __syncwarp();
    }   // tid < 32
    __syncthreads();
    // Jacobi on C (in G), rotations accumulated in W.  Each round applies
    // pp/2 disjoint rotations at once (round-robin pairing of the pp = p
    // rounded up to even indices; the pad index, when p is odd, pairs with
    // nothing): first the columns of G and W (G J, W J), then the rows of G
    // (J^T G J), every thread of the block taking (pair, row) items.
    {
        const int pp = p + (p & 1), half = pp / 2;
        double* cs = H;            // H is free until the sort: per-pair cosines,
        double* sn = H + P;        // sines
        int* pij = reinterpret_cast<int*>(H + 2 * P);   // and (i, j), 2 ints per pair
        __shared__ double red_off[8], red_dia[8];
        for (int sweep = 0; sweep < 30; ++sweep) {
            double off = 0.0, dia = 0.0;
            for (int t = tid; t < p * p; t += blockDim.x) {
                const int a = t / p, b = t % p;
                const double v = G[a * P + b];
                if (a != b) off += v * v; else dia += v * v;
            }
            for (int o = 16; o > 0; o >>= 1) {
                off += __shfl_xor_sync(0xffffffffu, off, o);
                dia += __shfl_xor_sync(0xffffffffu, dia, o);
            }
            if (lane == 0) {
                red_off[tid >> 5] = off;
                red_dia[tid >> 5] = dia;
            }
            __syncthreads();
            off = 0.0;
            dia = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {   // same order in every thread
                off += red_off[w];
                dia += red_dia[w];
            }
            __syncthreads();
            if (off <= 1e-34 * dia || off == 0.0) break;
            for (int r = 0; r < pp - 1; ++r) {
                if (tid < half) {
                    // round r: (pp-1, r) and ((r + k) mod (pp-1), (r - k) mod (pp-1)), k = 1 .. half-1
                    int a = tid == 0 ? pp - 1 : (r + tid) % (pp - 1);
                    int b = tid == 0 ? r : (r - tid + (pp - 1)) % (pp - 1);
                    const int i = min(a, b), j = max(a, b);
                    double c = 1.0, sg = 0.0;
                    if (j < p) {
                        const double aij = G[i * P + j];
                        if (aij != 0.0) {
                            const double aii = G[i * P + i], ajj = G[j * P + j];
                            const double tau = (ajj - aii) / (2.0 * aij);
                            const double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                            c = 1.0 / sqrt(1.0 + tt * tt);
                            sg = tt * c;
                        }
                    }
                    cs[tid] = c;
                    sn[tid] = sg;
                    pij[2 * tid] = i;
                    pij[2 * tid + 1] = j;
                }
                __syncthreads();
                for (int e = tid; e < half * p; e += blockDim.x) {   // columns: G J and W J
                    const int k = e / p, row = e % p;
                    const int i = pij[2 * k], j = pij[2 * k + 1];
                    if (j >= p || sn[k] == 0.0) continue;
                    const double c = cs[k], sg = sn[k];
                    const double gi = G[row * P + i], gj = G[row * P + j];
                    G[row * P + i] = c * gi - sg * gj;
                    G[row * P + j] = sg * gi + c * gj;
                    const double wi = W[row * P + i], wj = W[row * P + j];
                    W[row * P + i] = c * wi - sg * wj;
                    W[row * P + j] = sg * wi + c * wj;
                }
                __syncthreads();
                for (int e = tid; e < half * p; e += blockDim.x) {   // rows: J^T (G J)
                    const int k = e / p, col = e % p;
                    const int i = pij[2 * k], j = pij[2 * k + 1];
                    if (j >= p || sn[k] == 0.0) continue;
                    const double c = cs[k], sg = sn[k];
                    const double gi = G[i * P + col], gj = G[j * P + col];
                    G[i * P + col] = c * gi - sg * gj;
                    G[j * P + col] = sg * gi + c * gj;
                }
                __syncthreads();
                if (tid < half) {
                    const int i = pij[2 * tid], j = pij[2 * tid + 1];
                    if (j < p && sn[tid] != 0.0) {
                        G[i * P + j] = 0.0;
                        G[j * P + i] = 0.0;
                    }
                }
                __syncthreads();
            }
        }
    }
    if (tid >= 32) return;
    // sort eigenvalues ascending (selection sort of column order)
    if (lane == 0) {
        int ord[32];
        for (int a = 0; a < p; ++a) { ord[a] = a; ev[a] = G[a * P + a]; }
        for (int a = 0; a < p; ++a) {
            int best = a;
            for (int b = a + 1; b < p; ++b)
                if (ev[ord[b]] < ev[ord[best]]) best = b;
            const int tmp = ord[a]; ord[a] = ord[best]; ord[best] = tmp;
        }
        for (int a = 0; a < p; ++a) {
            theta[(int64_t)blockIdx.x * P + a] = ev[ord[a]];
            H[a] = (double)ord[a];
        }
    }
    __syncwarp();
    // T = R^{-1} W[:, ord]  (P x P, zero beyond p)
    double* T = Tout + (int64_t)blockIdx.x * P * P;
    for (int t = lane; t < P * P; t += 32) {
        const int a = t / P, b = t % P;
        double s = 0.0;
        if (a < p && b < p) {
            const int cb = (int)H[b];
            for (int k = a; k < p; ++k) s += Rm[a * P + k] * W[k * P + cb];
        }
        T[t] = s;
    }
}

__global__ void k_eig_update(int64_t nrows_pad, int P, const int32_t* __restrict__ sub_of_row,
                             const SubInfo* __restrict__ subs, const double* __restrict__ Y,
                             const double* __restrict__ T, double* __restrict__ X) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nrows_pad * P) return;
    const int64_t row = t / P;
    const int a = (int)(t % P);
    const int s = sub_of_row[row];
    if (s < 0) return;
    const int p = subs[s].p;
    const double* Tm = T + (int64_t)s * P * P;
    double v = 0.0;
    for (int b = 0; b < p; ++b) v += Y[row * P + b] * Tm[b * P + a];
    X[t] = v;
}

// residual norms ||\hat A x_k - theta_k S x_k||_{S^{-1}} for k < ncheck
__global__ void k_eig_resid(const SubInfo* __restrict__ subs, int P, const int64_t* __restrict__ rowptr,
                            const int32_t* __restrict__ colind, const double* __restrict__ vals,
                            const double* __restrict__ S, const double* __restrict__ ahat_diag,
                            const double* __restrict__ X, const double* __restrict__ theta, int ncheck,
                            double* __restrict__ resid) {
    const SubInfo Sb = subs[blockIdx.x];
    __shared__ double red[256];
    const int kmax = min(ncheck, Sb.p);
    double worst = 0.0;
    for (int k = 0; k < kmax; ++k) {
        const double th = theta[(int64_t)blockIdx.x * P + k];
        double acc = 0.0;
        for (int i = threadIdx.x; i < Sb.n; i += blockDim.x) {
            const int64_t g = Sb.row0 + i;
            double s = ahat_diag[g] * X[g * P + k];
            for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) {
                const int64_t j = colind[e];
                if (j != g && j >= Sb.row0 && j < Sb.row0 + Sb.n) s += vals[e] * X[j * P + k];
            }
            const double rr = s - th * S[g] * X[g * P + k];
            acc += rr * rr / S[g];
        }
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        worst = fmax(worst, sqrt(red[0]));
        __syncthreads();
    }
    if (threadIdx.x == 0) resid[blockIdx.x] = worst;
}

// Sign convention (largest-magnitude entry positive, lowest index on ties)
// and copy of the kept columns into the compact basis (row stride m_i).
__global__ void k_eig_finalize(const SubInfo* __restrict__ subs, int P, const double* __restrict__ X,
                               double* __restrict__ psi64) {
    const SubInfo Sb = subs[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = warp; k < Sb.m; k += nw) {
        double best = -1.0;
        int bi = 0x7fffffff;
        for (int i = lane; i < Sb.n; i += 32) {
            const double v = fabs(X[(Sb.row0 + i) * P + k]);
            if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        const double sgn = X[(Sb.row0 + bi) * P + k] < 0 ? -1.0 : 1.0;
        for (int i = lane; i < Sb.n; i += 32)
            psi64[Sb.psi_off + (int64_t)i * Sb.m + k] = sgn * X[(Sb.row0 + i) * P + k];
    }
}

__global__ void k_psi_round(int64_t n, const double* __restrict__ psi64, int prec,
                            double* __restrict__ used, float* __restrict__ p32,
                            __nv_bfloat16* __restrict__ p16) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = psi64[i];
    double u = v;
    if (prec == AMS_PREC_FP32) {
        const float f = (float)v;
        p32[i] = f;
        u = (double)f;
    } else if (prec == AMS_PREC_FP32_BF16) {
        const __nv_bfloat16 b = __double2bfloat16(v);
        p16[i] = b;
        u = (double)__bfloat162float(b);
    }
    used[i] = u;
}

// ---------------------------------------------------------------------------
// Galerkin product: block (I, J) of A_0 = sum_{i in I, j in J}
// psi_I[i,:]^T A_ij psi_J[j,:].  One thread block per subdomain I; thread
// (k, l) owns entry (k, l) of every neighbour block and walks the rows of
// I in order, so sums are deterministic.
// ---------------------------------------------------------------------------
__global__ void k_galerkin(const SubInfo* __restrict__ subs, const int64_t* __restrict__ rowptr,
                           const int32_t* __restrict__ colind, const double* __restrict__ vals,
                           const int32_t* __restrict__ sub_of_row, const double* __restrict__ psi,
                           const int64_t* __restrict__ nbr_ptr, const int32_t* __restrict__ nbr,
                           int max_nbr, int mmax, double* __restrict__ Ac, int64_t ldA, int64_t coff0,
                           int sub0) {
    extern __shared__ double acc[];             // max_nbr * mmax * mmax
    __shared__ int s_nbr[256];
    const int I = sub0 + blockIdx.x;
    const SubInfo SI = subs[I];
    const int64_t nb0 = nbr_ptr[I], nnb = nbr_ptr[I + 1] - nb0;
    for (int t = threadIdx.x; t < nnb; t += blockDim.x) s_nbr[t] = nbr[nb0 + t];
    for (int t = threadIdx.x; t < max_nbr * mmax * mmax; t += blockDim.x) acc[t] = 0.0;
    __syncthreads();
    const int k = threadIdx.x / mmax, l = threadIdx.x % mmax;
    if (k < SI.m) {
        for (int i = 0; i < SI.n; ++i) {
            const int64_t g = SI.row0 + i;
            const double pik = psi[SI.psi_off + (int64_t)i * SI.m + k];
            for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) {
                const int64_t j = colind[e];
                const int J = sub_of_row[j];
                const SubInfo SJ = subs[J];
                if (l >= SJ.m) continue;
                int slot = 0;
                while (slot < nnb && s_nbr[slot] != J) ++slot;
                const double pjl = psi[SJ.psi_off + (j - SJ.row0) * SJ.m + l];
                acc[(slot * mmax + k) * mmax + l] += pik * vals[e] * pjl;
            }
        }
    }
    __syncthreads();
    if (k < SI.m) {
        for (int slot = 0; slot < nnb; ++slot) {
            const SubInfo SJ = subs[s_nbr[slot]];
            if (l < SJ.m)
                Ac[(SI.coff - coff0 + k) * ldA + (SJ.coff - coff0 + l)] = acc[(slot * mmax + k) * mmax + l];
        }
    }
}

// Extraction of node matrices from the dense inverse factor (column-major,
// lower triangle: Linv(i, j) at i + j*ldL, zero for i < j).  One thread
// block per chunk; desc (8 x int64 per chunk): out_off (of the node matrix),
// K (its row length), kind (0 forward block R_s, 1 backward block Q_t), a
// (first coarse row of the node), cstart (first row of its subtree),
// rng_off | nrng << 32 (gather ranges of the backward block), e0, e1
// (element range of this chunk).
__global__ void k_extract(const int64_t* __restrict__ desc, const int32_t* __restrict__ rng,
                          const double* __restrict__ Linv, int64_t ldL, double* __restrict__ out64,
                          float* __restrict__ out32) {
    const int64_t* D = desc + 8 * (int64_t)blockIdx.x;
    const int64_t out_off = D[0], K = D[1] & 0xffffffff, ldm = D[1] >> 32, kind = D[2], a = D[3], cstart = D[4];
    const int rng_off = (int)(D[5] & 0xffffffff), nrng = (int)(D[5] >> 32);
    const int64_t e0 = D[6], e1 = D[7];   // element range over rows x ldm
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int64_t r = e / ldm, kk = e % ldm;
        double v = 0.0;
        if (kk < K) {
            int64_t i, j;
            if (kind == 0) {            // forward: row a+r, column cstart+kk
                i = a + r;
                j = cstart + kk;
            } else {                    // backward: row g(kk), column a+r
                int64_t k2 = kk, g = 0;
                for (int q = 0; q < nrng; ++q) {
                    const int64_t s0 = rng[2 * (rng_off + q)], len = rng[2 * (rng_off + q) + 1];
                    if (k2 < len) { g = s0 + k2; break; }
                    k2 -= len;
                }
                i = g;
                j = a + r;
            }
            v = (i >= j) ? Linv[i + j * ldL] : 0.0;
        }
        if (out64) out64[out_off + e] = v;
        if (out32) out32[out_off + e] = (float)v;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_band_assemble(const BandArgs& a, double* band, int mode, double sigma, double* S,
                          double* ahat_diag) {
    k_band_assemble<<<a.nsub, 256, 0, a.stream>>>(a.subs, a.band_off, a.rowptr, a.colind, a.vals, band,
                                                  mode, sigma, S, ahat_diag);
}
void launch_band_cholesky(const BandArgs& a, double* band, int32_t* status) {
    k_band_cholesky<<<a.nsub, 256, 0, a.stream>>>(a.subs, a.band_off, band, status);
}
void launch_band_pack_work(cudaStream_t s, int nwork, const SubInfo* subs, const int64_t* band_off,
                           const int2* work, const double* band, const int64_t* out_off, double* out64,
                           float* out32) {
    k_band_pack<<<nwork, 32, 0, s>>>(subs, band_off, work, band, out_off, out64, out32);
}
void launch_band_pack_tiles(cudaStream_t s, int nwork, const SubInfo* subs, const int64_t* band_off,
                            const int2* work, const double* band, const int64_t* out_off, float* fwd, float* bwd,
                            float* piv) {
    k_band_pack_tiles<<<nwork, 32, 0, s>>>(subs, band_off, work, band, out_off, fwd, bwd, piv);
}
void launch_eig_init(cudaStream_t s, int nsub, const SubInfo* subs, int P, double* X) {
    k_eig_init<<<nsub, 256, 0, s>>>(subs, P, X);
}
void launch_eig_rr(cudaStream_t s, int nsub, const SubInfo* subs, int P, const int64_t* rowptr,
                   const int32_t* colind, const double* vals, const double* S, const double* ahat_diag,
                   const double* Y, double* AY, double* T, double* theta, int32_t* status, int orth_only) {
    const size_t smem = (size_t)(4 * P * P + P) * sizeof(double);
    cudaFuncSetAttribute(k_eig_rr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_eig_rr<<<nsub, 256, smem, s>>>(subs, P, rowptr, colind, vals, S, ahat_diag, Y, AY, T, theta, status,
                                     orth_only);
}
void launch_eig_update(cudaStream_t s, int64_t nrows_pad, int P, const int32_t* sub_of_row,
                       const SubInfo* subs, const double* Y, const double* T, double* X) {
    const int64_t tot = nrows_pad * P;
    k_eig_update<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(nrows_pad, P, sub_of_row, subs, Y, T, X);
}
void launch_eig_resid(cudaStream_t s, int nsub, const SubInfo* subs, int P, const int64_t* rowptr,
                      const int32_t* colind, const double* vals, const double* S,
                      const double* ahat_diag, const double* X, const double* theta, int ncheck,
                      double* resid) {
    k_eig_resid<<<nsub, 256, 0, s>>>(subs, P, rowptr, colind, vals, S, ahat_diag, X, theta, ncheck, resid);
}
void launch_eig_finalize(cudaStream_t s, int nsub, const SubInfo* subs, int P, const double* X,
                         const double* S, double* psi64) {
    (void)S;
    k_eig_finalize<<<nsub, 256, 0, s>>>(subs, P, X, psi64);
}
void launch_psi_round(cudaStream_t s, int64_t n, const double* psi64, int prec, double* psi_used,
                      float* psi32, __nv_bfloat16* psi16) {
    if (n > 0) k_psi_round<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, psi64, prec, psi_used, psi32, psi16);
}
void launch_galerkin(cudaStream_t s, int nsub, const SubInfo* subs, const int64_t* rowptr,
                     const int32_t* colind, const double* vals, const int32_t* sub_of_row,
                     const double* psi, const int64_t* nbr_ptr, const int32_t* nbr, int max_nbr,
                     int mmax, double* Ac, int64_t ldA, int64_t coff0, int sub0) {
    const size_t smem = (size_t)max_nbr * mmax * mmax * sizeof(double);
    cudaFuncSetAttribute(k_galerkin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int threads = ((mmax * mmax + 31) / 32) * 32;
    k_galerkin<<<nsub, threads, smem, s>>>(subs, rowptr, colind, vals, sub_of_row, psi, nbr_ptr, nbr,
                                           max_nbr, mmax, Ac, ldA, coff0, sub0);
}
void launch_extract_chunks(cudaStream_t s, int nchunks, const int64_t* desc, const int32_t* rng,
                           const double* Linv, int64_t ldL, double* out64, float* out32) {
    if (nchunks > 0) k_extract<<<nchunks, 256, 0, s>>>(desc, rng, Linv, ldL, out64, out32);
}

}  // namespace ams
