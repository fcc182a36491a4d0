// Internal declarations of the AMS solve library (not part of the C ABI).
//
// Internal dof order: the subdomain-major order of Section 3.1 (each
// subdomain's dofs in ascending global index), systems of a batch back to
// back, each system's row range padded with inert zero rows to a multiple
// of kRowAlign so that every reduction block lies inside one system.
// Vectors are node-major: element (row, rhs) at row*ld + rhs, with ld the
// number of right-hand sides rounded up to a power of two (<= 32).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "../../include/ams.h"

namespace ams {

constexpr int kTile = 32;              // rows per block row of a local factor
constexpr int kRowAlign = 2048;        // row padding of each system
constexpr int kRedThreads = 256;       // threads of the reduction kernels
constexpr int kRedElems = 256;         // elements per reduction block (one per thread)
constexpr int kRedGroup = 64;          // blocks summed per first-level group
constexpr int kRedDirect = 2048;       // at most this many blocks: one-stage sum
constexpr int kRedMaxNV = 4;           // values per right-hand side in one reduction
constexpr int kRedBlocksPerSM = 4;     // reduction-kernel grid: about this many blocks per SM
constexpr int kMaxLd = 32;             // right-hand sides per solve call
constexpr int kMaxM = 16;              // eigenvectors per subdomain (cap)
constexpr int kCoarseChunk = 512;      // node-matrix columns per coarse item
constexpr int64_t kDefaultSpinCycles = int64_t(1) << 30;   // bounded device waits: ~0.5 s at 2 GHz

// ---- per-subdomain descriptor (device array) ------------------------------
struct SubInfo {
    int64_t row0;      // first internal row
    int64_t fac_off;   // element offset of block row 0 of the local factor
    int64_t psi_off;   // element offset of row 0 of the basis block (stride m)
    int64_t coff;      // coarse index (ND order) of mode 0
    int32_t n;         // rows n_i
    int32_t nb;        // block rows ceil(n_i / 32)
    int32_t c;         // band width in tiles (>= 1)
    int32_t m;         // kept eigenvectors m_i
    int32_t seg;       // system index
    int32_t p;         // eigensolver block size for this subdomain
};

// Block row K of a local factor (c band tiles) holds, contiguously,
//   [ M tile | dense tiles 1..c-1 | 32 reciprocal pivots ]
// M[r][q] = L_{K,K-c}[r][q] for q >= r (upper triangle incl. diagonal) and
//           (L_KK^{-1})[r][q] for q < r (strict lower triangle);
// dense tile t = L_{K,K-c+t};  pivots[r] = 1 / L_KK[r][r].
// Tile element (r, q) sits at q*32 + (r ^ q): column-major with an XOR
// swizzle so that both row-wise (forward) and column-wise (backward)
// shared-memory reads are free of bank conflicts.
__host__ __device__ inline int64_t blockrow_elems(int c) { return (int64_t)c * 1024 + 32; }
__host__ __device__ inline int tile_idx(int r, int q) { return q * 32 + (r ^ q); }

// ---- coarse inverse GEMM items ---------------------------------------------
// out[out0 + r][:] = sum_k Mat[moff + (row_in_node + r)*ldm + k] * in[g(k)][:]
// over k in [k0, k1), where g maps a node-matrix column to an input row
// through the gather ranges rng[rng_off .. rng_off+nrng) (start, len).
struct CoarseItem {
    int64_t moff;
    int32_t K;
    int32_t ldm;           // row stride of the node matrix (K rounded up to 4)
    int32_t nrows;
    int32_t row_in_node;
    int32_t out0;
    int32_t k0, k1;
    int32_t rng_off, nrng;
    int32_t tile_id;       // (node, row tile) for the last-arriver reduction
    int32_t nchunks;       // chunks of this tile
    int32_t chunk;         // this item's chunk
    int32_t slot0;         // first partial slot of this tile
    int64_t gat_off;       // backward items: the node's column gather list (-1: one contiguous range)
};

// Backward coarse substitution, fused into the prolongation: the rows of
// L_c^{-T} that belong to one subdomain (m_i consecutive rows of its ND
// node's backward block) and the node's column gather list into y.
struct CoarseRef {
    int64_t q_off;         // first element of the subdomain's rows in the backward blocks
    int64_t gat_off;       // first entry of the node's gather list
    int32_t K;             // columns: the node's own coarse rows, then its ancestors'
    int32_t ldm;           // row stride (K rounded up to 4)
};

// ---- per (system, rhs) CG scalars -----------------------------------------
struct CgScalars {
    double fnorm2;     // ||f||^2
    double rho;        // r.z (or z.r for the flexible variant)
    double pq;         // p.Ap
    double rr;         // r.r
    double zq;         // z.q (flexible variant)
    double alpha, beta;
    int32_t active;    // 1 while not converged
    int32_t iters;     // completed iterations
    int32_t xpend;     // x += alpha p of the last iteration still to apply (the
                       // next direction update, or the flush after the loop)
};

struct SolveState {    // device-resident control block
    int32_t it;        // completed iterations of the current solve
    int32_t done;      // all (system, rhs) converged
    int32_t status;    // ams_status set by device-side checks
    int32_t nactive;
    int32_t maxit;     // iteration cap of the current solve
    int32_t bodies;    // loop bodies (two iterations each) the device-resident loop has run
    int32_t xdone_it;  // value of `it` when a direction update last ran (it applied the
                       // pending x updates of iteration it - 1)
    double rtol2;      // squared relative residual target
    double worst;      // max over active (system, rhs) of ||r||^2 / ||f||^2
};

// ---- error bookkeeping ------------------------------------------------------
void set_error(const std::string& msg);

// Multilevel recursive bisection of the matrix pattern's graph into nparts
// parts (partition.cpp; behind ams_partition).
ams_status partition_graph(int64_t n, const int64_t* rowptr, const int32_t* colind, int32_t nparts,
                           double imbalance, uint64_t seed, int32_t* part, int64_t* edge_cut);

#define AMS_CUDA_TRY(expr)                                                     \
    do {                                                                       \
        cudaError_t _e = (expr);                                               \
        if (_e != cudaSuccess) {                                               \
            ::ams::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e)); \
            return (_e == cudaErrorMemoryAllocation) ? AMS_ERR_OOM : AMS_ERR_CUDA; \
        }                                                                      \
    } while (0)

// ---- host-side graph work (host_graph.cpp) --------------------------------
struct HostCSR {
    int64_t n = 0;
    std::vector<int64_t> rowptr;
    std::vector<int32_t> colind;
    std::vector<double> vals;
};

// Validate a CSR + partition (sorted, in range, symmetric to the last bit,
// positive diagonal, partition ids in range, no empty subdomain).
ams_status validate_system(const HostCSR& A, const int32_t* part, int32_t nparts);

// Subdomain-major order (Section 3.1): perm[k] = global dof, iperm inverse.
void build_index_maps(int64_t n, const int32_t* part, int32_t nparts,
                      std::vector<int64_t>& perm, std::vector<int64_t>& iperm,
                      std::vector<int64_t>& sub_ptr);

// Nested-dissection tree of the coarse (subdomain) graph.
struct NDNode {
    std::vector<int32_t> subs;   // subdomains of this node, in coarse order
    int32_t parent = -1;
    int64_t a = 0;               // first coarse row of the node
    int64_t k = 0;               // coarse rows of the node
    int64_t cstart = 0;          // first coarse row of the node's subtree
};
// adjacency: CSR over subdomains (no self loops); weight = m_i.
void nested_dissection(int32_t N, const std::vector<int64_t>& adj_ptr,
                       const std::vector<int32_t>& adj, const std::vector<int32_t>& weight,
                       int32_t leaf_weight, std::vector<NDNode>& nodes);

// ---- launchers (k_solve.cu) -------------------------------------------------
struct SolveBuffers;   // defined in ams_api.cu

}  // namespace ams
