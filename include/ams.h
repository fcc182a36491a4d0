/*
 * ams.h — C ABI of the GB300 (sm_103a) solve-phase library for the two-grid
 * algebraic multiscale (AMS) preconditioner of arXiv 2606.04864
 * ("An algebraic multiscale preconditioner for large sparse SPD matrices").
 *
 * The library solves A u = f (Eq. matrix-form, Section 1) for a sparse SPD
 * matrix A by preconditioned conjugate gradients on one GPU.  The
 * preconditioner is the paper's two-level method (Section 3):
 *
 *   M^{-1} = sum_i R_i^T A_i^{-1} R_i  +  R_0^T A_0^{-1} R_0
 *
 * with non-overlapping subdomains Omega_i given by a partition vector
 * (Section 3.1), A_i = R_i A R_i^T (Section 3.2), R_0^T the zero-extended
 * eigenvectors of the m smallest eigenvalues of the local generalized
 * eigenproblems  \hat A_i psi = lambda S_i psi  (Eq. algebraic-eigenproblem),
 * and A_0 = R_0 A R_0^T (Section 3.1).  The fine-level sum over local solves
 * is this library's reading of the fine-level component the paper's
 * Theorem 2 assumes but does not spell out.
 *
 * Conventions shared by every call:
 *  - Every function returns an ams_status; none aborts, traps or exits.  On
 *    error the thread-local message from ams_last_error() says why.
 *  - Ownership: the caller owns every array it passes in or out; the library
 *    copies what it needs during ams_setup*, so the caller may free its
 *    inputs as soon as the call returns.  The handle owns all device memory
 *    it allocates and releases it in ams_destroy.
 *  - Pointer kind: when ams_options.device_ptrs is 0 every array argument is
 *    a host pointer (the library copies through its own staging buffers);
 *    when 1 every array argument is a device pointer on the current device.
 *  - Streams: all device work is enqueued on the stream given to ams_setup*
 *    (NULL = legacy default stream).  Calls return after that work is done.
 *  - A handle is not thread-safe: do not call into one handle from two
 *    threads at once.
 *  - Vectors with several right-hand sides are n x nrhs, column-major
 *    (right-hand side k starts at element k*n), in the caller's dof order.
 *  - Integer and index outputs are exact; floating-point results depend on
 *    the precision mode (see ams_options.precision).
 */
#ifndef AMS_H
#define AMS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ams_handle_s* ams_handle;

typedef enum {
    AMS_OK = 0,
    AMS_ERR_INVALID_ARG = 1,     /* bad size, pointer, CSR, partition or option */
    AMS_ERR_NOT_SPD = 2,         /* non-positive pivot in a local or coarse Cholesky */
    AMS_ERR_BREAKDOWN = 3,       /* p^T A p <= 0, r^T M^{-1} r <= 0 or a non-finite scalar in CG */
    AMS_ERR_NOT_CONVERGED = 4,   /* maxit reached; outputs hold the last iterate */
    AMS_ERR_DEVICE_TIMEOUT = 5,  /* a bounded device-side wait ran out */
    AMS_ERR_CUDA = 6,            /* a CUDA runtime call failed, or a checking-build index check fired */
    AMS_ERR_OOM = 7              /* device allocation failed */
} ams_status;

enum {
    AMS_PREC_FP64 = 0,           /* preconditioner in FP64 (reference path) */
    AMS_PREC_FP32 = 1,           /* local factors, basis and coarse inverse in FP32 */
    AMS_PREC_FP32_BF16 = 2       /* as FP32, basis blocks stored BF16 */
};

enum {
    AMS_CG_AUTO = -1,            /* PCG for FP64, flexible CG otherwise */
    AMS_CG_PCG = 0,
    AMS_CG_FCG = 1               /* beta_k = z_{k+1}^T (r_{k+1}-r_k) / (z_k^T r_k) */
};

typedef struct {
    int32_t precision;           /* AMS_PREC_*; default AMS_PREC_FP32_BF16 */
    int32_t cg_variant;          /* AMS_CG_*; default AMS_CG_AUTO */
    int32_t maxit;               /* outer iteration cap; default 10000 */
    int32_t device_ptrs;         /* 0 host pointers (default), 1 device pointers */
    int32_t autotune;            /* 1 (default): at the first solve with a given
                                    number of right-hand sides, time candidate
                                    launch shapes (blocks per SM of the SpMV and
                                    prolongation grids, local-solve ring depth,
                                    right-hand sides per warp of the several-RHS
                                    local solve, L2 priorities of the one-RHS
                                    local solve's tile copies) on that right-hand
                                    side and keep the fastest */
    int32_t coarse;              /* 1: two-level (default); 0: local solves only */
    double eig_shift;            /* shift sigma of the local eigensolver; 0 = default 1e-2 */
    int32_t eig_maxit;           /* local eigensolver iteration cap; 0 = default 300 */
    double eig_tol;              /* local eigenpair residual target; 0 = default 1e-13 */
    int64_t spin_budget_cycles;  /* budget of every bounded device-side wait
                                    (the local solves' mbarrier waits for
                                    their factor-tile copies), in SM clock
                                    cycles; 0 (default) = 2^30 (about half a
                                    second).  A wait that runs out ends the
                                    solve with AMS_ERR_DEVICE_TIMEOUT after
                                    the block has waited (about a second at
                                    most) for its own copies in flight; the
                                    CUDA context stays usable.  Negative:
                                    AMS_ERR_INVALID_ARG */
    double eig_threshold;        /* > 0: adaptive coarse space, m_i = the local
                                    eigenvalues below this threshold (at least
                                    1, at most m, grown across a cluster), so
                                    that lambda_{m_i+1} >= threshold wherever
                                    the cap m does not bind (mu_c of Section 4
                                    is then at least the threshold);
                                    0 (default) = m_i = min(m, n_i) */
    double two_grid_omega;       /* > 0: precondition with the multiplicative
                                    two-grid cycle of Section 3.2 (smoother
                                    omega sum_i R_i^T A_i^{-1} R_i before and
                                    after the coarse correction; SPD for
                                    0 < omega < 2 / lambda_max of the local
                                    solves times A); 0 (default) = the
                                    additive two-level preconditioner.
                                    With no coarse space (coarse = 0 or
                                    every m_i = 0) the cycle is the
                                    symmetrised smoother 2 omega S -
                                    omega^2 S A S.  An omega at or above
                                    2 / lambda_max makes the cycle
                                    indefinite: the solve then reports
                                    AMS_ERR_BREAKDOWN once r^T z <= 0 (or
                                    stalls); setup does not estimate
                                    lambda_max for a positive value.
                                    Negative (between -2 and 0): omega =
                                    -two_grid_omega / lambda_max, lambda_max
                                    estimated at setup by power steps on the
                                    local solves times A (a Rayleigh
                                    quotient, which approaches lambda_max
                                    from below; at most 300 steps, until it
                                    moves by less than 1e-7 relative);
                                    ams_get_info reports the omega and the
                                    estimate */
    int32_t timeout_probe;       /* test hook, 0 (default) = off.  1: every
                                    block of the local-solve kernels first
                                    waits, within spin_budget_cycles, on a
                                    barrier that nothing completes, so that
                                    the timeout path (status, drain of the
                                    copies in flight, clean exit) runs on
                                    purpose; every solve then returns
                                    AMS_ERR_DEVICE_TIMEOUT.  Applies to the
                                    reduced-precision modes (the FP64 local
                                    solves have no bounded waits) */
    int32_t warm_start;          /* 1: ams_solve reads u as the initial guess
                                    u_0 (same layout as the solution) and
                                    runs CG from it; the stopping rule stays
                                    ||r_k|| <= rtol ||f||, and a zero right-
                                    hand side still gives u = 0.  Single-
                                    system handles only.  0 (default): u_0 = 0
                                    and u is write-only */
} ams_options;

/* Fill *opt with the defaults listed above. */
void ams_options_default(ams_options* opt);

/*
 * ams_setup — build the preconditioner for one SPD matrix (Sections 3.1-3.2).
 *
 *  n        number of dofs (rows), 1 <= n < 2^31
 *  rowptr   CSR row pointer, n+1 entries, rowptr[0] = 0
 *  colind   CSR column indices, rowptr[n] entries, strictly ascending per row
 *  vals     CSR values (FP64); A must be symmetric (pattern and values equal
 *           to the last bit) with a positive diagonal
 *  part     subdomain id of each dof, in [0, nparts); no subdomain may be empty;
 *           NULL = the built-in partition of the pattern (ams_partition with
 *           the default imbalance and seed 0)
 *  nparts   number of subdomains N
 *  m        eigenvectors per subdomain; the library keeps m_i = min(m, n_i)
 *           and grows m_i while lambda_{m_i+1} equals lambda_{m_i} to a
 *           relative 1e-8 (a cluster split by the cut); m = 0 gives
 *           block-Jacobi PCG
 *  opt      options (NULL = defaults)
 *  stream   cudaStream_t as void* (NULL = default stream)
 *  out      receives the handle
 *
 * Errors: AMS_ERR_INVALID_ARG (CSR unsorted, out of range or unsymmetric,
 * part out of range, empty subdomain, band of a subdomain too wide for the
 * shared-memory staging), AMS_ERR_NOT_SPD (non-positive pivot), AMS_ERR_OOM,
 * AMS_ERR_CUDA.
 */
ams_status ams_setup(int64_t n, const int64_t* rowptr, const int32_t* colind,
                     const double* vals, const int32_t* part, int32_t nparts,
                     int32_t m, const ams_options* opt, void* stream,
                     ams_handle* out);

/*
 * ams_partition — split the dofs into nparts subdomains from the matrix
 * pattern alone.  The method takes a non-overlapping partition as given
 * (Section 3.1; the paper's experiments use METIS, Section 5); this
 * built-in one is a multilevel recursive bisection of the pattern's graph
 * (heavy-edge matching, region growing on the coarsest graph,
 * Fiduccia-Mattheyses refinement on every level, the best of three
 * bisections per split, a greedy k-way pass at the end) for callers with
 * no partitioner of their own.  Host code only: no GPU, no CUDA context.
 *
 *  n, rowptr, colind  CSR pattern as for ams_setup (host memory); diagonal
 *                     entries are ignored and the pattern is symmetrised
 *  nparts             1 <= nparts <= n
 *  imbalance          every part has at most about (1 + imbalance) n/nparts
 *                     dofs (one dof of rounding per bisection level);
 *                     0 = default 0.03
 *  seed               the result depends on the seed alone
 *  part               out, host, n entries in [0, nparts); every part is
 *                     non-empty; parts need not be connected
 *  edge_cut           out (NULL allowed): undirected pattern edges {i, j},
 *                     i != j, whose endpoints lie in different parts
 *
 * Errors: AMS_ERR_INVALID_ARG (NULL arrays, n out of range, nparts outside
 * [1, n], negative or non-finite imbalance, rowptr not starting at 0 or
 * decreasing, column index out of range).
 */
ams_status ams_partition(int64_t n, const int64_t* rowptr, const int32_t* colind, int32_t nparts,
                         double imbalance, uint64_t seed, int32_t* part, int64_t* edge_cut);

/* One independent system of a batch (same meaning as ams_setup's arguments). */
typedef struct {
    int64_t n;
    const int64_t* rowptr;
    const int32_t* colind;
    const double* vals;
    const int32_t* part;
    int32_t nparts;
    int32_t m;
} ams_system_desc;

/*
 * ams_setup_batched — one handle over nsys independent systems of uneven
 * size, solved together (one launch sequence per iteration covers every
 * system and right-hand side; each system converges on its own).  Each
 * system gets the preconditioner ams_setup builds (Sections 3.1-3.2) from
 * its own matrix, partition and m; the paper has no batched solve.  Errors
 * as for ams_setup, for the first system that fails.
 * Vectors passed to ams_solve on such a handle are the systems' n_s x nrhs
 * column-major blocks laid end to end in system order; iters/relres
 * have nsys*nrhs entries (system-major).
 */
ams_status ams_setup_batched(int32_t nsys, const ams_system_desc* systems,
                             const ams_options* opt, void* stream,
                             ams_handle* out);

/*
 * ams_solve — A u = f (Eq. matrix-form) by preconditioned CG (flexible CG
 * per the handle's options) with the two-level preconditioner of Section
 * 3.1 (or the cycle of Section 3.2), from u_0 = 0 (or from u with
 * ams_options.warm_start) for nrhs right-hand sides at once.  The paper
 * runs GMRES to 1e-6 (Section 5); CG is used here because A and the
 * preconditioner are SPD.  Each right-hand side stops at the first k >= 0
 * with ||r_k||_2 <= rtol ||f||_2 on the recurrence residual.  Pointers are
 * host or device per ams_options.device_ptrs, owned by the caller.
 *
 *  f        n x nrhs right-hand sides (read only)
 *  nrhs     1 <= nrhs <= 32
 *  rtol     relative residual target, > 0
 *  u        n x nrhs solution (written; with warm_start also read first as u_0)
 *  iters    nrhs (batched: nsys*nrhs) iteration counts, may be NULL (host)
 *  relres   same shape, final recurrence residual / ||f||, may be NULL (host)
 *
 * iters and relres are always host pointers.  Returns AMS_ERR_NOT_CONVERGED
 * when maxit is reached (u, iters, relres hold the last iterate) and
 * AMS_ERR_BREAKDOWN when p^T A p <= 0, r^T z <= 0 (the preconditioner is not
 * SPD, e.g. a two-grid omega at or above 2 / lambda_max) or a scalar is not
 * finite.
 */
ams_status ams_solve(ams_handle h, const double* f, int32_t nrhs, double rtol,
                     double* u, int32_t* iters, double* relres);

/*
 * ams_solve_adjoint — backward pass of u = A^{-1} f (Eq. matrix-form) for a
 * loss L(u); the paper has no adjoint, this is the adjoint of a linear
 * solve.  Solves A lambda = g with the same preconditioner (Section 3.1;
 * A is symmetric), then forms the sampled outer product on A's pattern:
 *
 *   dvals[e] = - sum_k lambda_k[row_e] * u_k[col_e]     (dL/dA, CSR order)
 *   lambda   = dL/df
 *
 *  g        dL/du, n x nrhs
 *  u        the forward solution, n x nrhs
 *  lambda   n x nrhs output
 *  dvals    nnz output in the caller's CSR entry order, may be NULL
 *  iters    nrhs host iteration counts, may be NULL
 *
 * Batched handles are not supported here (AMS_ERR_INVALID_ARG).
 */
ams_status ams_solve_adjoint(ams_handle h, const double* g, int32_t nrhs,
                             double rtol, const double* u, double* lambda,
                             double* dvals, int32_t* iters);

/*
 * ams_set_matrix_values — replace the values of A (same CSR pattern, caller
 * order, nnz entries; host or device per the handle's pointer mode) used by
 * the SpMV of later solves, keeping the preconditioner built at setup.  PCG
 * stays correct for any SPD matrix with this pattern (the preconditioner is
 * only an approximation of its inverse); it converges fastest while the new
 * matrix is close to the one the preconditioner was built from.  The values
 * are not validated (symmetry and definiteness are the caller's
 * responsibility).  Single-system handles only.
 */
ams_status ams_set_matrix_values(ams_handle h, const double* vals);

/* Release every resource of the handle.  NULL is accepted. */
ams_status ams_destroy(ams_handle h);

/* Static description of a status code. */
const char* ams_status_string(ams_status s);

/* Thread-local message describing the last error (empty if none). */
const char* ams_last_error(void);

/* ------------------------------------------------------------------ */
/* Inspection entry points (used by tests and benchmarks).             */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t n;                   /* total dofs (batched: sum over systems) */
    int64_t nnz;
    int32_t nparts;              /* total subdomains */
    int32_t nsys;
    int64_t ncoarse;             /* coarse dimension N_c = sum_i m_i */
    int32_t max_band_tiles;      /* widest local band, in 32-row tiles */
    int32_t precision;
    int32_t cg_variant;
    double setup_seconds;        /* wall time of ams_setup* */
    double eig_seconds;          /* of which: local eigensolves */
    double coarse_seconds;       /* of which: Galerkin product + coarse factor */
    int32_t eig_iterations;      /* subspace iterations the eigensolver used */
    double eig_max_residual;     /* largest ||\hat A psi - lambda S psi||_{S^-1} kept */
    int64_t local_factor_bytes;  /* bytes of the stored local factors */
    int64_t coarse_inverse_bytes;/* bytes of the stored coarse inverse blocks */
    int64_t basis_bytes;         /* bytes of the stored basis blocks */
    int32_t spmv_variant;        /* launch shape picked for the SpMV */
    int64_t kernel_launches;     /* CUDA kernels this handle has launched so far */
    double two_grid_omega;       /* damping of the multiplicative cycle in use
                                    (0: additive preconditioner) */
    double local_lambda_max;     /* estimated lambda_max of the local solves
                                    times A (two_grid_omega < 0 at setup), else 0 */
    double coarse_factor_seconds;/* of coarse_seconds: Cholesky factor of A_0
                                    and its inverse */
    double coarse_factor_gflop;  /* FP64 work of those on the kept tiles (2 flops
                                    per multiply-add) */
} ams_info;

/* Sizes, timings and launch counts of a handle (host output; the paper's
 * setup/solve split of Section 5 is setup_seconds against the solves). */
ams_status ams_get_info(ams_handle h, ams_info* info);

/*
 * Launch shapes of the solve kernels for solves with nrhs right-hand sides
 * (1 <= nrhs <= 32; shapes are kept per nrhs rounded up to a power of two).
 * shape[0]  blocks per SM of the element-layout grids (direction update, SpMV)
 * shape[1]  blocks per SM of the subdomain-layout grid (prolongation)
 * shape[2]  local-solve ring depth in band tiles; 0 = derived from the band width
 * shape[3]  right-hand sides per warp of the several-RHS local solve (2, 4 or 8
 *           below 8 right-hand sides; 8 or 16 from 8 on, where the tile
 *           products run on the tensor cores); 0 = default
 * shape[4]  L2 priorities of the one-RHS local solve's factor-tile copies:
 *           0 none (default); 1 evict-first on copies that read a block row
 *           for the last time; 2 as 1, plus evict-last on the kept copies
 * shape[5]  kept copies: the forward loads of this many block rows below
 *           the ones that stay in the staging ring (the rows the backward
 *           sweep reloads soonest) are not marked evict-first
 * shape[6]  (get only) 1 once the shapes are fixed, by the autotuner or by
 *           ams_set_launch_shape; 0 while they are the defaults
 * ams_get_launch_shape writes 7 entries to host memory.  ams_set_launch_shape
 * reads shape[0..5], fixes them (the autotuner then leaves this count alone)
 * and drops the iteration graph captured with the previous shapes; call it
 * between solves.  Errors: AMS_ERR_INVALID_ARG (NULL, nrhs out of range,
 * blocks per SM outside 1..8, depth outside 0..6, below 2 with TMA staging or
 * needing more than 200 KB of shared memory, right-hand sides per warp not
 * 0 or one of the values above, above the rounded count or leaving more
 * than 8 warps per block (4 from 8 right-hand sides on),
 * L2 mode outside 0..2, negative kept rows).
 */
ams_status ams_get_launch_shape(ams_handle h, int32_t nrhs, int32_t* shape);
ams_status ams_set_launch_shape(ams_handle h, int32_t nrhs, const int32_t* shape);

/*
 * Index maps (Section 3.1): perm[k] = global dof at position k of the
 * subdomain-major order (ascending global index inside each subdomain),
 * sub_ptr[i]..sub_ptr[i+1] = positions of subdomain i.  Host outputs of
 * n and nparts+1 entries.  Single-system handles only.
 */
ams_status ams_get_index_maps(ams_handle h, int64_t* perm, int64_t* sub_ptr);

/*
 * The coarse basis (Section 3.2): m_i (nparts entries), the kept local
 * eigenvalues (sum m_i entries, subdomain-major, ascending), and psi, the
 * FP64 basis blocks: for each subdomain in order an n_i x m_i column-major
 * block in the subdomain's local order.  Host outputs; NULL skips an output.
 * The blocks are the FP64 eigenvectors even when a lower-precision copy is
 * used in the solve.
 */
ams_status ams_get_coarse_basis(ams_handle h, int32_t* m_i, double* lambda,
                                double* psi);

/*
 * The Galerkin coarse matrix A_0 = R_0 A R_0^T (Section 3.1) as a dense
 * N_c x N_c row-major host array in the paper's order (subdomain-major,
 * mode-minor).  For precision modes with a BF16 basis it is the product of
 * the rounded basis.  Single-system handles only.
 */
ams_status ams_get_coarse_matrix(ams_handle h, double* A0);

/*
 * The inverse L_c^{-1} of the Cholesky factor of A_0 (A_0 = L_c L_c^T in
 * the nested-dissection order of the coarse dofs that the coarse solve
 * uses; Section 3.1 defines A_0, the order is this library's), as a dense
 * N_c x N_c row-major host array (lower triangular), and nd_paper[p], the
 * paper-order index (as in ams_get_coarse_matrix) of ND position p.
 * Either output may be NULL.  Single-system handles with N_c <= 4096 only.
 */
ams_status ams_get_coarse_factor_inverse(ams_handle h, int64_t* nd_paper, double* Linv);

/*
 * One application z = M^{-1} r of the two-level preconditioner (n x nrhs,
 * caller's order), in the handle's precision: M^{-1} = sum_i R_i^T A_i^{-1}
 * R_i + R_0^T A_0^{-1} R_0 (Section 3.1), or with two_grid_omega the cycle
 * of Section 3.2.  Pointers per ams_options.device_ptrs.
 */
ams_status ams_apply_preconditioner(ams_handle h, const double* r,
                                    int32_t nrhs, double* z);

/* y = A x with the handle's stored matrix A of Eq. matrix-form (n x nrhs,
 * caller's order; pointers per ams_options.device_ptrs). */
ams_status ams_spmv(ams_handle h, const double* x, int32_t nrhs, double* y);

/*
 * The kernels of one CG iteration, in launch order (indices of
 * ams_time_kernel and of the ams_profile_solve outputs):
 *   AMS_KERNEL_SPMV        direction p = z + beta p_old, then q = A p and
 *                          p.q (two launches, timed together)
 *   AMS_KERNEL_LOCAL       local solves sum_i R_i^T A_i^{-1} R_i r' and the
 *                          restriction R_0 r', with r' = r - alpha q
 *   AMS_KERNEL_COARSE      forward substitution y = L_c^{-1} r_c
 *                          (A_0 = L_c L_c^T); with more than four
 *                          right-hand sides also the backward substitution
 *                          e_c = L_c^{-T} y (a second launch)
 *   AMS_KERNEL_PROLONG     (up to four right-hand sides: the backward
 *                          substitution,) z = z_f + R_0^T e_c, r = r',
 *                          x += alpha p, dots, convergence test and beta
 * Without a coarse space (coarse = 0) AMS_KERNEL_COARSE does not run.
 */
enum {
    AMS_KERNEL_SPMV = 0,
    AMS_KERNEL_LOCAL = 1,
    AMS_KERNEL_COARSE = 2,
    AMS_KERNEL_PROLONG = 3,
    AMS_NUM_KERNELS = 4
};

/*
 * Time one kernel of the solve on the handle's current solve state (after
 * an ams_solve with nrhs right-hand sides): `reps` back-to-back launches on
 * the handle's stream between two CUDA events.  which: an AMS_KERNEL_*
 * index.  Outputs the mean launch time (ms) and the kernel's algorithmic
 * bytes per launch (each operand read once, each output written once).
 * The launches overwrite the handle's solve work vectors.
 */
ams_status ams_time_kernel(ams_handle h, int32_t which, int32_t reps,
                           double* avg_ms, double* bytes);

/*
 * One solve (same arguments and result as ams_solve, output discarded) with
 * a CUDA event pair recorded around every kernel on the handle's stream, so
 * each kernel's device time is measured inside a real solve (cold caches,
 * real data).  Outputs per kernel (AMS_KERNEL_* order), host arrays of
 * AMS_NUM_KERNELS entries: total milliseconds `ms`, launches `count`,
 * algorithmic bytes per launch `bytes`.  The solve runs without graph
 * capture.
 */
ams_status ams_profile_solve(ams_handle h, const double* f, int32_t nrhs,
                             double rtol, double* ms, double* bytes,
                             int64_t* count);

/*
 * Diagnostic.  The solve kernels convert between FP32 and FP64 with integer
 * instructions (FP64 instructions are scarce on this GPU).  This call
 * checks those conversions against the hardware conversions for n device
 * FP64 values x: *narrow_bad counts values whose FP64 -> FP32 result
 * differs bitwise (round to nearest even; NaNs compared as NaN), and
 * *widen_bad those whose FP32 -> FP64 widening of the hardware-rounded value
 * differs.  Both are 0 when the conversions agree.  Synchronous on the
 * current device's default stream; allocates 16 bytes of device memory.
 * Errors: AMS_ERR_INVALID_ARG (n < 0, NULL pointers), AMS_ERR_CUDA.
 */
ams_status ams_check_conversions(const double* x, int64_t n, int64_t* narrow_bad, int64_t* widen_bad);

/*
 * Checking build (libams_debug.so, compiled with -DAMS_DEBUG): the solve
 * kernels check the indices they gather through (matrix columns, coarse
 * gather lists, subdomain row ranges, the caller-order permutation); a
 * failed check records its site and skips the access, and the call that
 * launched it returns AMS_ERR_CUDA naming the site (ams_last_error).  This
 * entry point launches a kernel that fails one check on purpose, site 99,
 * without touching memory, and returns the recorded site in *site: 99 in
 * the checking build, 0 in the release build (checks compiled out).  Not a
 * method step (no section of the paper): a test hook of the library.
 */
ams_status ams_debug_selftest(int32_t* site);

/*
 * ams_csr_spmv_dot_noalloc — y = A x and *xy = x^T y for a CSR matrix, with
 * no handle and no device allocation.  The paper has no counterpart: this
 * is a service for callers that cannot allocate device memory at the
 * moment they need the product, e.g. code that runs while another library
 * captures a CUDA graph (allocation is not allowed during capture), hosts
 * whose device memory is handed out by their own fixed pool, or real-time
 * callers that forbid allocation after start-up.
 *
 *  n        rows (and columns) of A, 0 <= n <= 8,388,608 (larger n returns
 *           AMS_ERR_INVALID_ARG and does nothing)
 *  rowptr   device int64 CSR row pointer (n+1), colind device int32,
 *  vals     device FP64 values (any symmetric or unsymmetric CSR)
 *  x        device FP64 input (n), y device FP64 output (n)
 *  xy       device FP64 output scalar x^T y (summed in a fixed order)
 *  stream   cudaStream_t as void*; the call is asynchronous on it (unlike
 *           the other calls, it does not wait for the GPU)
 *
 * The dot product's per-block partial sums and arrival counter live in one
 * fixed 64 KB device array inside the library, held by every GPU that loads
 * it until the process exits.  The first call on a device looks up that
 * array's address on the current device; make that first call before any
 * stream capture.  All calls share the array (the counter is cleared at the
 * start of each call), so calls that overlap on the GPU race: order them on
 * one stream.
 */
ams_status ams_csr_spmv_dot_noalloc(int64_t n, const int64_t* rowptr,
                                    const int32_t* colind, const double* vals,
                                    const double* x, double* y, double* xy,
                                    void* stream);

#ifdef __cplusplus
}
#endif

#endif /* AMS_H */
