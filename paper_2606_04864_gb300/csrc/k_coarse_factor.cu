// Cholesky factor of the coarse matrix A_0 (Section 3.1) and the inverse of
// that factor, L_c^{-1}, whose nested-dissection blocks the coarse solve
// multiplies by.  FP64 throughout, on 64 x 64 tiles of the dense N_c x N_c
// column-major array, skipping every tile that the nested-dissection order
// of the subdomain graph keeps zero.
//
// Structure.  The coarse rows are ordered by a nested-dissection tree of the
// subdomain graph, each tree node a contiguous row range, children before
// parents.  A_0(r, c) != 0 only for neighbouring subdomains, and neighbours
// are never split into different child subtrees, so with node(r) the node
// owning row r:
//     L(r, c) and L^{-1}(r, c) (r >= c) can be non-zero only where node(r)
//     is node(c) or an ancestor of it.
// A product L(r, l) X(l, c) of two such entries is non-zero only where
// node(r) is an ancestor-or-self of node(c) as well, so every entry outside
// the pattern stays an exact zero through the factorisation and the
// inversion.  A tile is kept when any of its entries lies in the pattern;
// an update of a tile outside it is a sum of exact zeros and is skipped.
//
// Factorisation (right-looking, by column tile k):
//     L_kk = chol(A_kk), kept with its inverse L_kk^{-1};
//     L_ik = A_ik L_kk^{-T}                   for kept tiles i > k;
//     A_ij -= L_ik L_jk^T                     for kept tiles i >= j > k.
// Inversion (X = L^{-1}, right-looking over row tile k of X):
//     X_kk = L_kk^{-1};
//     X_ic -= L_ik X_kc                       for kept i > k, c <= k,
// and X_ic = L_ii^{-1} X_ic once the last update of X_ic has landed (the
// step that applies it is known from the pattern, so the same thread block
// finishes the tile).
#include <algorithm>
#include <cstdint>
#include <vector>

#include "ams_internal.h"
#include "launch.h"

namespace ams {

namespace {

constexpr int TB = 64;          // tile edge
constexpr int TKC = 32;         // contraction chunk staged in shared memory
constexpr int TP = TB + 1;      // padded shared-memory row
constexpr int TTHREADS = 256;   // 16 x 16 threads, 4 x 4 outputs each

__device__ __forceinline__ int tile_rows(int64_t nc, int t) {
    const int64_t r = nc - (int64_t)t * TB;
    return r < TB ? (int)r : TB;
}

// acc[a][b] += sum_kk Aop(m, kk) Bop(kk, n), m = tx + 16a, n = ty + 16b,
// kk < kdim, with Aop(m, kk) = A[m + kk*lda] (zero for m >= am) and
// Bop(kk, n) = BT ? B[n + kk*ldb] : B[kk + n*ldb] (zero for n >= bn).
template <bool BT>
__device__ __forceinline__ void tile_gemm(double (&acc)[4][4], const double* __restrict__ A, int64_t lda, int am,
                                          const double* __restrict__ B, int64_t ldb, int bn, int kdim,
                                          double (*As)[TP], double (*Bs)[TP]) {
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int k0 = 0; k0 < kdim; k0 += TKC) {
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int m = tid & 63, kk = (tid >> 6) + 4 * s;
            As[kk][m] = (m < am && k0 + kk < kdim) ? A[m + (int64_t)(k0 + kk) * lda] : 0.0;
        }
        if (BT) {
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const int n = tid & 63, kk = (tid >> 6) + 4 * s;
                Bs[kk][n] = (n < bn && k0 + kk < kdim) ? B[n + (int64_t)(k0 + kk) * ldb] : 0.0;
            }
        } else {
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const int kk = tid & 31, n = (tid >> 5) + 8 * s;
                Bs[kk][n] = (n < bn && k0 + kk < kdim) ? B[(k0 + kk) + (int64_t)n * ldb] : 0.0;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < TKC; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][tx + 16 * i];
                b[i] = Bs[kk][ty + 16 * i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void zero_acc(double (&acc)[4][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
}

// C[m][n] = acc (SUB = false) or C[m][n] -= acc (SUB = true), m < cm, n < cn.
template <bool SUB>
__device__ __forceinline__ void tile_store(const double (&acc)[4][4], double* __restrict__ C, int64_t ldc, int cm,
                                           int cn) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int n = ty + 16 * j;
        if (n >= cn) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int m = tx + 16 * i;
            if (m >= cm) continue;
            double* p = C + m + (int64_t)n * ldc;
            *p = SUB ? *p - acc[i][j] : acc[i][j];
        }
    }
}

// Diagonal tile t: L_tt = chol(A_tt) in place (lower triangle), its inverse
// into invd[t] (64 x 64 column-major; identity on the padding of a ragged
// last tile) and into the diagonal tile of X.  A pivot that is not positive
// records its coarse row in *bad (min over tiles) and is replaced by 1 so
// that the sweep stays finite; the host reports the failure.
__global__ void __launch_bounds__(TTHREADS) k_tile_potrf(double* __restrict__ A, double* __restrict__ X, int64_t nc,
                                                         int t, double* __restrict__ invd,
                                                         unsigned long long* __restrict__ bad) {
    extern __shared__ double sm[];
    double(*S)[TP] = reinterpret_cast<double(*)[TP]>(sm);             // S[r][c]
    double(*Li)[TP] = reinterpret_cast<double(*)[TP]>(sm + TB * TP);  // Li[r][c]
    const int nr = tile_rows(nc, t);
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)t * TB * (nc + 1);
    for (int e = tid; e < TB * TB; e += TTHREADS) {
        const int r = e & 63, c = e >> 6;   // r fastest: coalesced column reads
        double v;
        if (r < nr && c < nr) v = (r >= c) ? A[base + r + (int64_t)c * nc] : 0.0;
        else v = (r == c) ? 1.0 : 0.0;
        S[r][c] = v;
    }
    __shared__ double s_rs;         // reciprocal of the current pivot
    __shared__ double s_inv[TB];    // reciprocal pivots, for the inverse
    __syncthreads();
    for (int j = 0; j < TB; ++j) {
        // one thread takes the pivot's square root and reciprocal (FP64
        // square root and division are long sequences on this GPU's narrow
        // FP64 pipe: not once per thread)
        if (tid == 0) {
            double d = S[j][j];
            if (!(d > 0.0)) {
                atomicMin(bad, (unsigned long long)((int64_t)t * TB + j));
                d = 1.0;
            }
            const double sq = sqrt(d);
            S[j][j] = sq;
            s_rs = 1.0 / sq;
            s_inv[j] = s_rs;
        }
        __syncthreads();
        const double rs = s_rs;
        for (int r = j + 1 + tid; r < TB; r += TTHREADS) S[r][j] *= rs;
        __syncthreads();
        for (int e = tid; e < TB * TB; e += TTHREADS) {
            const int r = e >> 6, c = e & 63;
            if (c > j && r >= c) S[r][c] = fma(-S[r][j], S[c][j], S[r][c]);
        }
        __syncthreads();
    }
    // inverse of the lower-triangular S, column c by four lanes of one warp
    {
        const int c = tid >> 2, q = tid & 3;
        if (q == 0) Li[c][c] = s_inv[c];
        __syncwarp();
        for (int r = 1; r < TB; ++r) {
            double s = 0.0;
            if (r > c)
                for (int l = c + q; l < r; l += 4) s = fma(S[r][l], Li[l][c], s);
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            if (r > c && q == 0) Li[r][c] = -s * s_inv[r];
            __syncwarp();
        }
        for (int r = q; r < c; r += 4) Li[r][c] = 0.0;
    }
    __syncthreads();
    double* iv = invd + (int64_t)t * TB * TB;
    for (int e = tid; e < TB * TB; e += TTHREADS) {
        const int r = e & 63, c = e >> 6;
        iv[r + c * TB] = Li[r][c];
        if (r < nr && c < nr) {
            if (r >= c) A[base + r + (int64_t)c * nc] = S[r][c];
            X[base + r + (int64_t)c * nc] = Li[r][c];
        }
    }
}

// Column step k of the factorisation: L_ik = A_ik L_kk^{-T}, one block per
// kept row tile i > k (rows[blockIdx.x]).
__global__ void __launch_bounds__(TTHREADS) k_tile_trsm(double* __restrict__ A, int64_t nc, int k,
                                                        const int32_t* __restrict__ rows,
                                                        const double* __restrict__ invd) {
    __shared__ double As[TKC][TP], Bs[TKC][TP];
    const int i = rows[blockIdx.x];
    const int mi = tile_rows(nc, i), mk = tile_rows(nc, k);
    double* Cik = A + (int64_t)i * TB + (int64_t)k * TB * nc;
    double acc[4][4];
    zero_acc(acc);
    tile_gemm<true>(acc, Cik, nc, mi, invd + (int64_t)k * TB * TB, TB, mk, mk, As, Bs);
    tile_store<false>(acc, Cik, nc, mi, mk);
}

// Column step k of the factorisation: A_ij -= L_ik L_jk^T for the kept
// pairs (pairs[blockIdx.x] = (i, j), i >= j > k).
__global__ void __launch_bounds__(TTHREADS) k_tile_update(double* __restrict__ A, int64_t nc, int k,
                                                          const int2* __restrict__ pairs) {
    __shared__ double As[TKC][TP], Bs[TKC][TP];
    const int2 p = pairs[blockIdx.x];
    const int mi = tile_rows(nc, p.x), mj = tile_rows(nc, p.y), mk = tile_rows(nc, k);
    const double* Lik = A + (int64_t)p.x * TB + (int64_t)k * TB * nc;
    const double* Ljk = A + (int64_t)p.y * TB + (int64_t)k * TB * nc;
    double acc[4][4];
    zero_acc(acc);
    tile_gemm<true>(acc, Lik, nc, mi, Ljk, nc, mj, mk, As, Bs);
    tile_store<true>(acc, A + (int64_t)p.x * TB + (int64_t)p.y * TB * nc, nc, mi, mj);
}

// Row step k of the inversion: X_ic -= L_ik X_kc for the kept pairs
// (tasks[blockIdx.x] = (i, c | last << 31), i > k >= c); on the pair's last
// update, X_ic = L_ii^{-1} X_ic.
__global__ void __launch_bounds__(TTHREADS) k_tile_inv_step(const double* __restrict__ A, double* __restrict__ X,
                                                            int64_t nc, int k, const int2* __restrict__ tasks,
                                                            const double* __restrict__ invd) {
    __shared__ double As[TKC][TP], Bs[TKC][TP];
    const int2 p = tasks[blockIdx.x];
    const int i = p.x, c = p.y & 0x7fffffff;
    const bool last = (p.y >> 31) & 1;
    const int mi = tile_rows(nc, i), mc = tile_rows(nc, c), mk = tile_rows(nc, k);
    double* Xic = X + (int64_t)i * TB + (int64_t)c * TB * nc;
    double acc[4][4];
    zero_acc(acc);
    tile_gemm<false>(acc, A + (int64_t)i * TB + (int64_t)k * TB * nc, nc, mi,
                     X + (int64_t)k * TB + (int64_t)c * TB * nc, nc, mc, mk, As, Bs);
    tile_store<true>(acc, Xic, nc, mi, mc);
    if (!last) return;
    __syncthreads();   // the block's own global writes are visible to it after the barrier
    zero_acc(acc);
    tile_gemm<false>(acc, invd + (int64_t)i * TB * TB, TB, mi, Xic, nc, mc, mi, As, Bs);
    tile_store<false>(acc, Xic, nc, mi, mc);
}

}  // namespace

// ---------------------------------------------------------------------------
// host: the kept tiles and the task lists of every step
// ---------------------------------------------------------------------------
void build_coarse_tile_plan(const std::vector<NDNode>& nodes, int64_t nc, CoarseTilePlan& P) {
    P = CoarseTilePlan{};
    P.nc = nc;
    const int T = (int)((nc + TB - 1) / TB);
    P.T = T;
    if (T == 0) return;
    auto first_tile = [](int64_t row) { return (int)(row / TB); };
    // kept tiles of each column tile K (rows >= K), from the nodes that own
    // K's columns and their ancestors
    std::vector<std::vector<int32_t>> colpat(T), rowpat(T);
    std::vector<int32_t> stamp(T, -1);
    std::vector<uint64_t> kept((size_t)T * ((T + 63) / 64), 0);
    const size_t wpr = (size_t)(T + 63) / 64;
    auto is_kept = [&](int i, int j) { return (kept[(size_t)j * wpr + (i >> 6)] >> (i & 63)) & 1u; };
    size_t q0 = 0;   // first node whose range may reach column tile K
    for (int K = 0; K < T; ++K) {
        const int64_t c0 = (int64_t)K * TB, c1 = std::min<int64_t>(nc, c0 + TB);
        auto& col = colpat[K];
        auto mark = [&](int64_t r0, int64_t r1) {   // rows [r0, r1), r1 > r0
            for (int I = std::max(K, first_tile(r0)); I <= first_tile(r1 - 1); ++I)
                if (stamp[I] != K) {
                    stamp[I] = K;
                    col.push_back(I);
                }
        };
        mark(c0, c0 + 1);   // the diagonal tile
        while (q0 < nodes.size() && nodes[q0].a + nodes[q0].k <= c0) ++q0;
        for (size_t q = q0; q < nodes.size() && nodes[q].a < c1; ++q) {
            if (nodes[q].k == 0) continue;
            mark(std::max<int64_t>(nodes[q].a, c0), nodes[q].a + nodes[q].k);
            for (int32_t p = nodes[q].parent; p >= 0; p = nodes[p].parent)
                if (nodes[p].k > 0) mark(nodes[p].a, nodes[p].a + nodes[p].k);
        }
        std::sort(col.begin(), col.end());
        for (int32_t I : col) {
            kept[(size_t)K * wpr + (I >> 6)] |= uint64_t(1) << (I & 63);
            rowpat[I].push_back(K);   // K ascending: each row list is sorted
        }
        P.kept_tiles += (int64_t)col.size();
    }
    // factorisation steps
    P.trsm_ptr.assign(T + 1, 0);
    P.upd_ptr.assign(T + 1, 0);
    for (int k = 0; k < T; ++k) {
        const auto& col = colpat[k];   // col[0] == k
        for (size_t a = 1; a < col.size(); ++a) P.trsm.push_back(col[a]);
        for (size_t a = 1; a < col.size(); ++a)
            for (size_t b = 1; b <= a; ++b)
                if (is_kept(col[a], col[b])) {
                    P.upd.push_back(col[a]);
                    P.upd.push_back(col[b]);
                }
        P.trsm_ptr[k + 1] = (int64_t)P.trsm.size();
        P.upd_ptr[k + 1] = (int64_t)P.upd.size() / 2;
    }
    // inversion steps; then flag each pair's last update (latest step)
    P.inv_ptr.assign(T + 1, 0);
    for (int k = 0; k < T; ++k) {
        const auto& col = colpat[k];
        for (size_t a = 1; a < col.size(); ++a)
            for (int32_t c : rowpat[k])
                if (is_kept(col[a], c)) {
                    P.inv.push_back(col[a]);
                    P.inv.push_back(c);
                }
        P.inv_ptr[k + 1] = (int64_t)P.inv.size() / 2;
    }
    std::vector<uint64_t> seen(kept.size(), 0);
    for (int64_t t = (int64_t)P.inv.size() / 2 - 1; t >= 0; --t) {
        const int i = P.inv[2 * t], c = P.inv[2 * t + 1];
        uint64_t& w = seen[(size_t)c * wpr + (i >> 6)];
        const uint64_t bit = uint64_t(1) << (i & 63);
        if (!(w & bit)) {
            w |= bit;
            P.inv[2 * t + 1] = (int32_t)((uint32_t)c | 0x80000000u);
        }
    }
    const double tile_fma = (double)TB * TB * TB;
    P.fma = tile_fma * ((double)P.upd.size() / 2 + (double)P.trsm.size() + (double)P.inv.size() / 2);
}

size_t coarse_tile_invd_elems(int T) { return (size_t)T * TB * TB; }

void launch_coarse_tile_factor(cudaStream_t s, const CoarseTilePlan& P, const int32_t* d_trsm, const int2* d_upd,
                               const int2* d_inv, double* d_A, double* d_X, double* d_invd,
                               unsigned long long* d_bad) {
    const int T = P.T;
    if (T == 0) return;
    const size_t psmem = 2 * TB * TP * sizeof(double);
    cudaFuncSetAttribute(k_tile_potrf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
    k_tile_potrf<<<1, TTHREADS, psmem, s>>>(d_A, d_X, P.nc, 0, d_invd, d_bad);
    for (int k = 0; k < T; ++k) {
        const int64_t nt = P.trsm_ptr[k + 1] - P.trsm_ptr[k];
        if (nt > 0) k_tile_trsm<<<(unsigned)nt, TTHREADS, 0, s>>>(d_A, P.nc, k, d_trsm + P.trsm_ptr[k], d_invd);
        const int64_t nu = P.upd_ptr[k + 1] - P.upd_ptr[k];
        if (nu > 0) k_tile_update<<<(unsigned)nu, TTHREADS, 0, s>>>(d_A, P.nc, k, d_upd + P.upd_ptr[k]);
        if (k + 1 < T) k_tile_potrf<<<1, TTHREADS, psmem, s>>>(d_A, d_X, P.nc, k + 1, d_invd, d_bad);
    }
    for (int k = 0; k + 1 < T; ++k) {
        const int64_t ni = P.inv_ptr[k + 1] - P.inv_ptr[k];
        if (ni > 0)
            k_tile_inv_step<<<(unsigned)ni, TTHREADS, 0, s>>>(d_A, d_X, P.nc, k, d_inv + P.inv_ptr[k], d_invd);
    }
}

}  // namespace ams
