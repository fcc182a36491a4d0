// Launch descriptors and launcher declarations for the AMS kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ams_internal.h"
#include "kernels.cuh"

namespace ams {

// Everything the per-row reduction kernels need for one solve shape.
// Launch `kern` on `stream`; with pdl the launch carries the programmatic
// stream serialization attribute (the kernel must call pdl_wait(), see
// kernels.cuh).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_kernel(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                 cudaStream_t stream, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

struct LaunchCtx {
    cudaStream_t stream;
    int ld;                  // right-hand-side stride (power of two)
    int64_t nblk;            // blocks of red
    int nseg;                // systems
    RedLayout red;           // element blocks
    RedLayout red_sub;       // blocks of consecutive subdomains
    int64_t nblk_sub;        // blocks of red_sub
    int nsub;                // subdomains
    CgScalars* sc;           // [nseg][ld]
    SolveState* st;
    bool pdl;                // solve-loop kernels: programmatic dependent launch
    const int64_t* sell_ptr;
    const int32_t* sell_col;
    const double* sell_val;
    const float* sell_val32;   // FP32 copy of the values for the two-grid cycle's residuals, or NULL
    const int32_t* sub_of_row;
    const SubInfo* subs;
};

// Residual used by the local solves: r' = r - alpha q (alpha = rho / pq of
// the subdomain's (system, rhs)) for pairs still iterating when q is
// non-NULL, r itself otherwise.
struct ResidIn {
    const double* r;
    const double* q;         // NULL: no update
    const CgScalars* sc;     // [nseg][ld]
};

struct LocalSolveArgs {
    cudaStream_t stream;
    int nsub;
    const SubInfo* subs;
    ResidIn in;
    const double* rowscale;  // NULL or per-row scale applied to the input
    int ld;
    int cmax;
    int mmax;
    const SolveState* st;
    bool pdl;
    int depth;               // ring depth (block rows in flight); 0: chosen from the band width
};

struct LocalTmaArgs {
    cudaStream_t stream;
    int nsub;
    const SubInfo* subs;
    const struct CUtensorMap_st* tmF;
    const struct CUtensorMap_st* tmB;
    const int64_t* tile_row0;
    const float* piv;
    ResidIn in;
    int ld;
    int cmax;
    int mmax;
    int nbmax;          // largest number of 32-row block rows of a subdomain
    int64_t budget;
    SolveState* st;
    bool pdl;
    int depth;               // ring depth (block rows in flight); 0: chosen from the band width
    int nr;                  // several-RHS kernel: right-hand sides per warp (1, 2, 4, 8); 0: default
    int l2mode;              // one-RHS kernel, L2 priority of factor tiles: 0 none, 1 evict-first on
                             // tiles read for the last time, 2 as 1 plus evict-last on kept tiles
    int l2keep;              // block rows below the ring's resident ones whose forward load is
                             // kept (not marked evict-first): the backward sweep reloads them soonest
    int32_t* err;            // status word set to AMS_ERR_DEVICE_TIMEOUT when a wait runs out (or NULL)
    int probe;               // 1: every block first waits on a barrier nothing completes (timeout test)
    // several-RHS kernel: subdomains grouped by band width, one launch per
    // group sized for its own width (nclass <= 1: one launch over all)
    int nclass = 0;
    const int* class_c = nullptr;        // host: band tiles of each group
    const int* class_n = nullptr;        // host: subdomains of each group
    const int* class_nb = nullptr;       // host: most block rows of a subdomain in each group
    const int32_t* order = nullptr;      // device: subdomain ids, group after group
};

struct CoarseLaunch {
    cudaStream_t stream;
    int nitems;
    const CoarseItem* items;
    const void* mat;
    const int32_t* rng;
    const int32_t* gat;      // per-node column gather lists (backward items)
    void* partial;
    int32_t* cnt;
    const SolveState* st;
    bool pdl;
};

// q = A p, and p.q per (system, rhs) when with_dot
void launch_spmv_dot(const LaunchCtx& L, const double* p, double* q, int with_dot);
// p_new = z + beta p_old (per system and right-hand side)
// p_new = z + beta p_old, and the previous iteration's x += alpha p_old
// where that is still pending
void launch_dir_update(const LaunchCtx& L, int prec, const void* z, const double* p_old, double* p_new, double* x);
// after the loop: the last iteration's pending x += alpha p
void launch_x_flush(const LaunchCtx& L, const double* p, const double* p2, double* x);
void launch_init_norms(const LaunchCtx& L, const double* r, int nrhs);
size_t local_solve_smem(int cmax, int ld, size_t tf_bytes, int depth);
int local_solve_depth(int cmax, int ld, size_t tf_bytes);
cudaError_t launch_local_solve(const LocalSolveArgs& a, int prec, const void* fac, const void* psi,
                               void* zf, void* rc);
void launch_coarse_gemm(const CoarseLaunch& c, int prec, int ld, const void* in, void* out);
cudaError_t launch_local_tma(const LocalTmaArgs& a, int prec, const void* psi, void* zf, void* rc);
// 8 to 32 right-hand sides: tile products as tensor-core MMAs (k_local_mma.cu)
cudaError_t launch_local_mma(const LocalTmaArgs& a, int prec, const void* psi, void* zf, void* rc);
size_t local_mma_smem(int cmax, int ld, int depth);
size_t local_tma_smem(int cmax, int ld, int depth);
// Shared memory the TMA local-solve launch for `a` needs at ring depth `depth`.
size_t local_tma_launch_smem(const LocalTmaArgs& a, int depth);
cudaError_t make_tile_map(void* base, int64_t rows, struct CUtensorMap_st* out);
void launch_band_pack_tiles(cudaStream_t s, int nwork, const SubInfo* subs, const int64_t* band_off,
                            const int2* work, const double* band, const int64_t* out_off, float* fwd, float* bwd,
                            float* piv);
struct ProlongArgs {
    const void* psi;
    const void* ec;          // coarse correction from a separate backward launch, or NULL
    const void* yc;          // forward coarse substitution output (NULL without a coarse space)
    const void* qmat;        // backward blocks of L_c^{-1} (NULL without a coarse space)
    const CoarseRef* cref;
    const int32_t* gat;
    const void* zf;
    double* r;
    const double* q;
    double* x;
    const double* p;
    void* z;                 // z in the apply precision (FP32 values are exact in FP64)
    int mmax;
    int flexible;
    int mode;                // 0 apply only, 1 first application, 2 CG iteration
};
void launch_prolong_update(const LaunchCtx& L, int prec, const ProlongArgs& a);

// multiplicative two-grid cycle (k_two_grid.cu); v_is_fp64: v holds doubles,
// else the apply precision's floats
void launch_tg_resid(const LaunchCtx& L, const void* v, int v_is_fp64, const ResidIn& in, double* w);
void launch_tg_scale(const LaunchCtx& L, int prec, void* zf, double omega, int64_t n);
// b = a rounded to FP32 (round to nearest even)
void launch_round_to_f32(cudaStream_t s, const double* a, int64_t n, float* b);
void launch_tg_combine(const LaunchCtx& L, int prec, void* zf, const void* x2, double omega, int64_t n);
void launch_tg_restrict(const LaunchCtx& L, int prec, const void* psi, const double* w, void* rc, int mmax);
// One power step for the cycle's damping: per system the sums x.y, y.z and
// z.z into out[3 s ..] (y = A x, z = the local solves of y in the apply
// precision), and x_next = z / ||z||.  sys_blk0: first kRowAlign-row block
// of each system (nsys + 1 entries); blk_sys: system of each block.
void launch_power_step(cudaStream_t s, int prec, const double* x, const double* y, const void* z, int64_t nrows,
                       const int64_t* sys_blk0, const int32_t* blk_sys, int nsys, double* part, double* out,
                       double* inv_norm, double* x_next);
// Condition of the device-resident iteration loop (a while node of a CUDA
// graph): continue while the solve is not done and fewer than `cap` bodies
// have run.
void launch_loop_cond(cudaStream_t s, cudaGraphConditionalHandle h, SolveState* st, int cap);
void launch_permute_in(cudaStream_t s, const double* f, int64_t n, int nrhs, int ld,
                       const int64_t* int_row, double* r, double* x);
void launch_permute_out(cudaStream_t s, const double* x, int64_t n, int nrhs, int ld,
                        const int64_t* int_row, double* u);
// the same from FP32 values (z in the reduced-precision modes), widened exactly
void launch_permute_out_f32(cudaStream_t s, const float* x, int64_t n, int nrhs, int ld,
                            const int64_t* int_row, double* u);
// u += u0 (caller order, single system) where the right-hand side is non-zero
void launch_add_initial_guess(cudaStream_t s, double* u, const double* u0, int64_t n, int nrhs,
                              const CgScalars* sc);
void launch_sddmm(cudaStream_t s, const int64_t* rowptr, const int32_t* colind, int64_t n, int nrhs,
                  const double* lam, const double* u, double* dvals);
void launch_zero(cudaStream_t s, double* a, int64_t n);
void launch_scatter_vals(cudaStream_t s, const double* vals, const int64_t* pos, int64_t nnz, double* sell_val);

// ---- setup kernels (k_setup.cu) ---------------------------------------------
struct BandArgs {
    cudaStream_t stream;
    int nsub;
    const SubInfo* subs;
    const int64_t* band_off;     // per subdomain: element offset of its band (32*nb rows x (32c+1))
    const int64_t* rowptr;       // internal CSR (renumbered, padded rows empty)
    const int32_t* colind;
    const double* vals;
};
// mode 0: A_i ; mode 1: \hat A_i + sigma S_i.  Also writes S (diag of \hat A
// with the zero-weight reading) and the \hat A diagonal when non-NULL.
void launch_band_assemble(const BandArgs& a, double* band, int mode, double sigma, double* S,
                          double* ahat_diag);
void launch_band_cholesky(const BandArgs& a, double* band, int32_t* status);

// eigensolver (shift-invert subspace iteration, FP64)
void launch_eig_init(cudaStream_t s, int nsub, const SubInfo* subs, int P, double* X);
void launch_eig_rr(cudaStream_t s, int nsub, const SubInfo* subs, int P, const int64_t* rowptr,
                   const int32_t* colind, const double* vals, const double* S, const double* ahat_diag,
                   const double* Y, double* AY, double* T, double* theta, int32_t* status,
                   int orth_only);
void launch_eig_update(cudaStream_t s, int64_t nrows_pad, int P, const int32_t* sub_of_row,
                       const SubInfo* subs, const double* Y, const double* T, double* X);
void launch_eig_resid(cudaStream_t s, int nsub, const SubInfo* subs, int P, const int64_t* rowptr,
                      const int32_t* colind, const double* vals, const double* S,
                      const double* ahat_diag, const double* X, const double* theta, int ncheck,
                      double* resid);
void launch_eig_finalize(cudaStream_t s, int nsub, const SubInfo* subs, int P, const double* X,
                         const double* S, double* psi64);
void launch_psi_round(cudaStream_t s, int64_t n, const double* psi64, int prec, double* psi_used,
                      float* psi32, __nv_bfloat16* psi16);

// Galerkin A_0 = R_0 A R_0^T into a dense (per system) row-major matrix
void launch_galerkin(cudaStream_t s, int nsub, const SubInfo* subs, const int64_t* rowptr,
                     const int32_t* colind, const double* vals, const int32_t* sub_of_row,
                     const double* psi, const int64_t* nbr_ptr, const int32_t* nbr, int max_nbr,
                     int mmax, double* Ac, int64_t ldA, int64_t coff0, int sub0);
void launch_extract_chunks(cudaStream_t s, int nchunks, const int64_t* desc, const int32_t* rng,
                           const double* Linv, int64_t ldL, double* out64, float* out32);
// Checking-build hooks of the translation units with index checks (no-ops
// in the release build; see kernels.cuh).
void debug_set_bounds_solve(int64_t n_rows, int64_t n_coarse);
void debug_set_bounds_coarse(int64_t n_rows, int64_t n_coarse);
void debug_set_bounds_local_mma(int64_t n_rows, int64_t n_coarse);
void debug_set_bounds_local_tma(int64_t n_rows, int64_t n_coarse);
int32_t debug_take_site_solve();
int32_t debug_take_site_coarse();
int32_t debug_take_site_local_mma();
int32_t debug_take_site_local_tma();
// launches a kernel that fails one check on purpose (site 99) without any
// memory access; the site then reads back from debug_take_site_solve()
void launch_debug_selftest(cudaStream_t s);

// Tile Cholesky factor of A_0 and its inverse (k_coarse_factor.cu).  The
// plan lists, per step, the kept 64 x 64 tiles of the nested-dissection
// pattern: row tiles of the TRSM of column k, (i, j) pairs of its update,
// (i, c | last << 31) pairs of row step k of the inversion.
struct CoarseTilePlan {
    int64_t nc = 0;
    int T = 0;                         // tiles per side
    int64_t kept_tiles = 0;            // kept tiles of the lower triangle
    double fma = 0.0;                  // tile multiply-adds of factor + inverse
    std::vector<int32_t> trsm;         // row tiles, by step
    std::vector<int64_t> trsm_ptr;     // T + 1
    std::vector<int32_t> upd;          // (i, j) pairs, by step
    std::vector<int64_t> upd_ptr;      // T + 1, in pairs
    std::vector<int32_t> inv;          // (i, c | last << 31) pairs, by step
    std::vector<int64_t> inv_ptr;      // T + 1, in pairs
};
void build_coarse_tile_plan(const std::vector<NDNode>& nodes, int64_t nc, CoarseTilePlan& P);
size_t coarse_tile_invd_elems(int T);
// A (N_c x N_c, column-major, lower triangle read) becomes L (lower
// triangle); X must be zero on entry and becomes L^{-1} (lower triangle);
// *bad (initially ~0) receives the first coarse row whose pivot is not
// positive.
void launch_coarse_tile_factor(cudaStream_t s, const CoarseTilePlan& P, const int32_t* d_trsm, const int2* d_upd,
                               const int2* d_inv, double* d_A, double* d_X, double* d_invd,
                               unsigned long long* d_bad);
void launch_band_pack_work(cudaStream_t s, int nwork, const SubInfo* subs, const int64_t* band_off,
                           const int2* work, const double* band, const int64_t* out_off, double* out64,
                           float* out32);

}  // namespace ams
