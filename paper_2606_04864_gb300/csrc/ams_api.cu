// C ABI of the AMS solve library: handle, setup orchestration, PCG driver,
// adjoint and inspection entry points.  See include/ams.h for the contract.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "ams_internal.h"
#include "kernels.cuh"
#include "launch.h"

namespace ams {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

// NVTX range for the duration of a scope: every entry point marks its work
// (ams_setup, ams_solve, ...), and the per-kernel profiling solve marks
// each kernel slot, so profilers can select them by name.  Costs nothing
// when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
static const char* const kSlotNames[AMS_NUM_KERNELS] = {"spmv_direction", "local_solve_restrict", "coarse_solve",
                                                        "prolong_update"};

static int pow2ceil(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}
static int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

#define AMS_TRY(expr)                          \
    do {                                       \
        ams_status _s = (expr);                \
        if (_s != AMS_OK) return _s;           \
    } while (0)

// device allocation owned by a handle
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct RedCache {
    int ld = 0;
    int64_t nblk = 0;
    int ngrp = 0;
    int64_t* blk_lo = nullptr;
    int32_t *blk_seg = nullptr, *seg_blk0 = nullptr, *seg_nblk = nullptr, *seg_grp0 = nullptr;
    double *part1 = nullptr, *part2 = nullptr;
    int32_t *cnt1 = nullptr, *cnt2 = nullptr, *cnt3 = nullptr;
};

// Launch shapes of the solve kernels for one ld.
struct TuneCfg {
    int bps_elem = kRedBlocksPerSM;     // element-layout blocks per SM (direction update, SpMV)
    int bps_sub = kRedBlocksPerSM;      // subdomain-layout blocks per SM (prolongation)
    int depth = 0;                      // local-solve ring depth; 0: chosen from the band width
    int nr = 0;                         // several-RHS local solve: right-hand sides per warp; 0: default
    int l2mode = 0;                     // one-RHS local solve: L2 priorities of the factor tiles (0 none)
    int l2keep = 0;                     // block rows whose forward load keeps its L2 priority
    bool done = false;                  // autotuned
};

struct SystemHost {
    int64_t n = 0, nnz = 0;
    int64_t caller0 = 0;       // offset of this system in caller vectors
    int64_t caller_nnz0 = 0;   // offset of this system's entries among all systems' entries
    int64_t row0 = 0;          // first internal row
    int64_t npad = 0;          // padded internal rows
    int32_t sub0 = 0, nparts = 0, m = 0;
    int64_t coff0 = 0, nc = 0; // coarse range (global coarse index)
    std::vector<int64_t> perm, sub_ptr;
    std::vector<NDNode> nodes;
    std::vector<double> A0_nd;  // dense A_0 in ND order (small systems only)
    std::vector<double> Linv_nd;  // L_c^{-1} in ND order, column-major (small systems only)
    std::vector<int64_t> nd_pos_of_sub;  // coarse position (relative) of mode 0 of each subdomain
};

}  // namespace ams

using namespace ams;

// per-kernel event timing of one solve (ams_profile_solve)
struct KernelProfile {
    double ms[AMS_NUM_KERNELS] = {};
    int64_t count[AMS_NUM_KERNELS] = {};
    cudaEvent_t ev[32];
    int nev = 0;
    int which[16];
};

struct ams_handle_s {
    ams_options opt{};
    cudaStream_t stream = nullptr;      // internal non-blocking stream (all device work)
    cudaStream_t ustream = nullptr;     // caller's stream (ordering only)
    cudaEvent_t ev_enter = nullptr;
    std::map<int, cudaGraphExec_t> loop_graph;   // device-resident iteration loop per ld
    KernelProfile* prof = nullptr;
    int prec = AMS_PREC_FP32_BF16;
    int flexible = 1;
    int nsys = 0;
    std::vector<SystemHost> sys;
    int64_t n_total = 0, n_pad = 0, nnz_total = 0;
    int32_t N = 0;
    int64_t Nc = 0;
    int cmax = 1, mmax = 0, nbmax = 1;
    // subdomains grouped by band width (several-RHS local solve: one launch
    // per group; empty when every subdomain has the same width)
    std::vector<int> cls_c, cls_n, cls_nb;
    int32_t* d_cls_order = nullptr;
    int num_sms = 1;                    // SMs of the handle's device
    bool use_pdl = false;               // solve-loop kernels overlap their prologue with the previous kernel
    std::vector<SubInfo> h_subs;
    std::vector<double> h_lam;          // kept eigenvalues, subdomain-major
    std::vector<DevBuf> bufs;
    // device data
    SubInfo* d_subs = nullptr;
    int64_t* d_int_row = nullptr;
    int32_t* d_sub_of_row = nullptr;
    int64_t *d_sell_ptr = nullptr;
    int32_t* d_sell_col = nullptr;
    double* d_sell_val = nullptr;
    float* d_sell_val32 = nullptr;      // the values in FP32, for the two-grid cycle's residuals (mixed path)
    int64_t sell_elems = 0;             // stored SELL entries (padding included)
    int64_t* d_crowptr = nullptr;       // caller CSR (single system) for dL/dA
    int32_t* d_ccolind = nullptr;
    int64_t* d_sell_pos = nullptr;      // caller CSR entry -> SELL slot (single system)
    void* d_fac = nullptr;
    int64_t fac_elems = 0;
    // reduced-precision local factors in the TMA tile layout
    bool use_tma = false;
    float *d_tfwd = nullptr, *d_tbwd = nullptr, *d_piv = nullptr;
    int64_t* d_trow0 = nullptr;
    int64_t tile_elems = 0;
    CUtensorMap tmF{}, tmB{};
    double* d_psi64 = nullptr;
    void* d_psi = nullptr;              // basis in the solve precision
    int64_t psi_elems = 0;
    CoarseItem *d_fwd = nullptr, *d_bwd = nullptr;
    int nfwd = 0, nbwd = 0;
    void *d_Rmat = nullptr, *d_Qmat = nullptr;
    CoarseRef* d_cref = nullptr;        // per subdomain: its rows of the backward blocks
    int32_t* d_gat = nullptr;           // per ND node: backward column gather lists
    int64_t R_elems = 0, Q_elems = 0;
    int32_t* d_rng = nullptr;
    void* d_partial = nullptr;
    int32_t* d_cnt = nullptr;
    // solve work space (sized for ld_alloc)
    int ld_alloc = 0, ld_last = 0;
    double *d_x = nullptr, *d_r = nullptr, *d_p = nullptr, *d_q = nullptr, *d_z = nullptr;
    double* d_p2 = nullptr;             // second direction buffer (iterations alternate p and p2)
    void *d_zf = nullptr, *d_rc = nullptr, *d_yc = nullptr, *d_ec = nullptr;
    double* d_tw = nullptr;     // two-grid cycle: residual of the current iterate
    double *d_stage_in = nullptr, *d_stage_out = nullptr, *d_stage_aux = nullptr;
    double* d_stage_dvals = nullptr;
    CgScalars* d_sc = nullptr;
    SolveState* d_st = nullptr;
    std::map<std::pair<int, int>, RedCache> red;      // element blocks, per (ld, blocks per SM)
    std::map<std::pair<int, int>, RedCache> red_sub;  // subdomain ranges, per (ld, blocks per SM)
    std::map<int, TuneCfg> tune;        // launch shapes per ld (autotuned or defaults)
    ams_info info{};
    int64_t launches = 0;               // kernels launched by solve-time entry points

    size_t tf_bytes() const { return prec == AMS_PREC_FP64 ? 8 : 4; }
    size_t tp_bytes() const { return prec == AMS_PREC_FP64 ? 8 : (prec == AMS_PREC_FP32 ? 4 : 2); }

    ams_status alloc(void** p, size_t bytes) {
        *p = nullptr;
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
            return AMS_ERR_OOM;
        }
        bufs.push_back({*p, bytes});
        return AMS_OK;
    }
    template <typename T>
    ams_status alloc_t(T** p, size_t count) {
        return alloc((void**)p, count * sizeof(T));
    }
    void release(void* p) {
        for (auto& b : bufs)
            if (b.p == p && p) {
                cudaFree(p);
                b.p = nullptr;
            }
    }
    // pinned host mirrors of the solve state and the per-(system, rhs) CG
    // scalars, read back at the end of a solve without a blocking copy
    SolveState* h_st = nullptr;
    CgScalars* h_sc = nullptr;
    int64_t pending_lpi = 0;   // launches per loop body of the solve in flight (0: counted already)
    ~ams_handle_s() {
        if (stream) cudaStreamSynchronize(stream);
        if (h_st) cudaFreeHost(h_st);
        if (h_sc) cudaFreeHost(h_sc);
        for (auto& g : loop_graph) cudaGraphExecDestroy(g.second);
        for (auto& b : bufs)
            if (b.p) cudaFree(b.p);
        if (ev_enter) cudaEventDestroy(ev_enter);
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace ams {

template <typename T>
static ams_status upload(ams_handle h, T** dst, const std::vector<T>& v) {
    AMS_TRY(h->alloc_t(dst, v.size()));
    if (!v.empty())
        AMS_CUDA_TRY(cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    return AMS_OK;
}

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------------------
// reduction layout for a given ld
// ---------------------------------------------------------------------------
// Blocks [blk0[s], blk0[s] + nblk[s]) belong to system s; block b covers
// the range [blk_lo[b], blk_lo[b+1]).
static ams_status build_red(ams_handle h, int ld, const std::vector<int64_t>& blk_lo,
                            const std::vector<int32_t>& blk_seg, const std::vector<int32_t>& seg_blk0,
                            const std::vector<int32_t>& seg_nblk, RedCache& rc) {
    rc.ld = ld;
    rc.nblk = (int64_t)blk_seg.size();
    std::vector<int32_t> seg_grp0(h->nsys);
    int ngrp = 0;
    for (int s = 0; s < h->nsys; ++s) {
        seg_grp0[s] = ngrp;
        ngrp += (seg_nblk[s] + kRedGroup - 1) / kRedGroup;
    }
    rc.ngrp = ngrp;
    AMS_TRY(upload(h, &rc.blk_lo, blk_lo));
    AMS_TRY(upload(h, &rc.blk_seg, blk_seg));
    AMS_TRY(upload(h, &rc.seg_blk0, seg_blk0));
    AMS_TRY(upload(h, &rc.seg_nblk, seg_nblk));
    AMS_TRY(upload(h, &rc.seg_grp0, seg_grp0));
    AMS_TRY(h->alloc_t(&rc.part1, (size_t)std::max<int64_t>(rc.nblk, 1) * kRedMaxNV * ld));
    AMS_TRY(h->alloc_t(&rc.part2, (size_t)std::max(ngrp, 1) * kRedMaxNV * ld));
    AMS_TRY(h->alloc_t(&rc.cnt1, (size_t)std::max(ngrp, 1)));
    AMS_TRY(h->alloc_t(&rc.cnt2, (size_t)h->nsys));
    AMS_TRY(h->alloc_t(&rc.cnt3, 1));
    AMS_CUDA_TRY(cudaMemsetAsync(rc.cnt1, 0, sizeof(int32_t) * std::max(ngrp, 1), h->stream));
    AMS_CUDA_TRY(cudaMemsetAsync(rc.cnt2, 0, sizeof(int32_t) * h->nsys, h->stream));
    AMS_CUDA_TRY(cudaMemsetAsync(rc.cnt3, 0, sizeof(int32_t), h->stream));
    return AMS_OK;
}

// Split `work[i]` (i = 0..count-1, one system) into `nb` consecutive ranges of
// about equal total work; appends the range starts (offset by `first`).
static void split_ranges(const std::vector<int64_t>& work, int nb, int64_t first, std::vector<int64_t>& lo) {
    const int64_t count = (int64_t)work.size();
    double tot = 0.0;
    for (int64_t w : work) tot += (double)w;
    int64_t i = 0;
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) {
        lo.push_back(first + i);
        const double target = tot * (double)(b + 1) / nb;
        const int64_t left = nb - 1 - b;   // later ranges each keep at least one item
        while (i < count - left && (acc < target || i == lo.back() - first)) acc += (double)work[i++];
    }
}

// Reduction layouts for a given ld, sized to about `bps` blocks per SM:
// blocks of whole kRedElems-element chunks of one system, and blocks of
// consecutive subdomains of one system (balanced by rows).
static ams_status get_layout(ams_handle h, int ld, int bps, bool sub, RedCache** out) {
    auto& cache = sub ? h->red_sub : h->red;
    const auto key = std::make_pair(ld, bps);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *out = &it->second;
        return AMS_OK;
    }
    const int target = std::max(1, bps * h->num_sms);
    std::vector<int64_t> blk_lo;
    std::vector<int32_t> blk_seg, seg_blk0(h->nsys), seg_nblk(h->nsys);
    if (!sub) {
        const int64_t nchunk_tot = h->n_pad * ld / kRedElems;
        for (int s = 0; s < h->nsys; ++s) {
            const int64_t c0 = h->sys[s].row0 * ld / kRedElems;
            const int64_t nc = h->sys[s].npad * ld / kRedElems;
            int nb = (int)std::llround((double)target * (double)nc / (double)nchunk_tot);
            nb = (int)std::max<int64_t>(1, std::min<int64_t>(nb, nc));
            seg_blk0[s] = (int32_t)blk_seg.size();
            seg_nblk[s] = nb;
            std::vector<int64_t> work(nc, 1), lo;
            split_ranges(work, nb, c0, lo);
            for (int64_t c : lo) {
                blk_lo.push_back(c * kRedElems);
                blk_seg.push_back(s);
            }
        }
        blk_lo.push_back(h->n_pad * ld);
    } else {
        for (int s = 0; s < h->nsys; ++s) {
            const SystemHost& S = h->sys[s];
            int nb = (int)std::llround((double)target * (double)S.n / (double)std::max<int64_t>(1, h->n_total));
            nb = std::max(1, std::min(nb, S.nparts));
            seg_blk0[s] = (int32_t)blk_seg.size();
            seg_nblk[s] = nb;
            std::vector<int64_t> work(S.nparts), lo;
            for (int a = 0; a < S.nparts; ++a) work[a] = std::max<int64_t>(1, h->h_subs[S.sub0 + a].n);
            split_ranges(work, nb, S.sub0, lo);
            for (int64_t b : lo) {
                blk_lo.push_back(b);
                blk_seg.push_back(s);
            }
        }
        blk_lo.push_back(h->N);
    }
    RedCache rc;
    AMS_TRY(build_red(h, ld, blk_lo, blk_seg, seg_blk0, seg_nblk, rc));
    cache[key] = rc;
    *out = &cache[key];
    return AMS_OK;
}

// The layouts of the current launch shapes for ld.
static ams_status get_red(ams_handle h, int ld, RedCache** out, RedCache** out_sub) {
    const TuneCfg& T = h->tune[ld];
    AMS_TRY(get_layout(h, ld, T.bps_elem, false, out));
    return get_layout(h, ld, T.bps_sub, true, out_sub);
}

static RedLayout layout_of(const RedCache& rc) {
    RedLayout R;
    R.blk_lo = rc.blk_lo;
    R.blk_seg = rc.blk_seg;
    R.seg_blk0 = rc.seg_blk0;
    R.seg_nblk = rc.seg_nblk;
    R.seg_grp0 = rc.seg_grp0;
    R.part1 = rc.part1;
    R.part2 = rc.part2;
    R.cnt1 = rc.cnt1;
    R.cnt2 = rc.cnt2;
    R.cnt3 = rc.cnt3;
    return R;
}

static LaunchCtx make_ctx(ams_handle h, const RedCache& rc, const RedCache& rcs) {
    LaunchCtx L;
    L.stream = h->stream;
    L.ld = rc.ld;
    L.nblk = rc.nblk;
    L.nseg = h->nsys;
    L.red = layout_of(rc);
    L.red_sub = layout_of(rcs);
    L.nblk_sub = rcs.nblk;
    L.nsub = h->N;
    L.sc = h->d_sc;
    L.st = h->d_st;
    L.sell_ptr = h->d_sell_ptr;
    L.sell_col = h->d_sell_col;
    L.sell_val = h->d_sell_val;
    L.sell_val32 = h->d_sell_val32;
    L.sub_of_row = h->d_sub_of_row;
    L.subs = h->d_subs;
    L.pdl = h->use_pdl;
    return L;
}

// ---------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------
struct SysInput {
    HostCSR A;
    std::vector<int32_t> part;
    int32_t nparts;
    int32_t m;
};

static ams_status read_inputs(const ams_system_desc& d, int device_ptrs, SysInput& in) {
    if (d.n <= 0 || !d.rowptr || !d.colind || !d.vals) {
        set_error("null pointer or non-positive n");
        return AMS_ERR_INVALID_ARG;
    }
    if (d.m < 0 || d.m > kMaxM) {
        set_error("m must be in [0, " + std::to_string(kMaxM) + "]");
        return AMS_ERR_INVALID_ARG;
    }
    in.A.n = d.n;
    in.A.rowptr.resize(d.n + 1);
    in.part.resize(d.n);
    const cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    AMS_CUDA_TRY(cudaMemcpy(in.A.rowptr.data(), d.rowptr, sizeof(int64_t) * (d.n + 1), kind));
    const int64_t nnz = in.A.rowptr[d.n];
    if (nnz < d.n || nnz > (int64_t(1) << 40)) {
        set_error("implausible nnz (rowptr[n])");
        return AMS_ERR_INVALID_ARG;
    }
    in.A.colind.resize(nnz);
    in.A.vals.resize(nnz);
    AMS_CUDA_TRY(cudaMemcpy(in.A.colind.data(), d.colind, sizeof(int32_t) * nnz, kind));
    AMS_CUDA_TRY(cudaMemcpy(in.A.vals.data(), d.vals, sizeof(double) * nnz, kind));
    if (d.part) {
        AMS_CUDA_TRY(cudaMemcpy(in.part.data(), d.part, sizeof(int32_t) * d.n, kind));
    } else {   // no partition given: the built-in one of the matrix pattern
        AMS_TRY(partition_graph(d.n, in.A.rowptr.data(), in.A.colind.data(), d.nparts, 0.0, 0, in.part.data(),
                                nullptr));
    }
    in.nparts = d.nparts;
    in.m = d.m;
    return validate_system(in.A, in.part.data(), d.nparts);
}

static ams_status build_local_factors(ams_handle h, const int64_t* d_rowptr, const int32_t* d_colind,
                                      const double* d_vals, double* d_S, double* d_ahat, double sigma,
                                      int eig_mode, void** out_fac, int64_t* out_elems, int out_fp64,
                                      bool tiles = false) {
    // band buffer
    std::vector<int64_t> band_off(h->N), fac_off(h->N);
    int64_t band_tot = 0, fac_tot = 0;
    std::vector<int2> work;
    for (int s = 0; s < h->N; ++s) {
        const SubInfo& S = h->h_subs[s];
        band_off[s] = band_tot;
        band_tot += (int64_t)32 * S.nb * (32 * S.c + 1);
        fac_off[s] = fac_tot;
        fac_tot += (int64_t)S.nb * blockrow_elems(S.c);
        for (int K = 0; K < S.nb; ++K) work.push_back(make_int2(s, K));
    }
    double* d_band = nullptr;
    int64_t *d_band_off = nullptr, *d_fac_off = nullptr;
    int2* d_work = nullptr;
    int32_t* d_status = nullptr;
    AMS_TRY(h->alloc_t(&d_band, (size_t)band_tot));
    AMS_TRY(upload(h, &d_band_off, band_off));
    AMS_TRY(upload(h, &d_fac_off, fac_off));
    AMS_TRY(upload(h, &d_work, work));
    AMS_TRY(h->alloc_t(&d_status, 1));
    AMS_CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int32_t), h->stream));
    BandArgs ba{h->stream, h->N, h->d_subs, d_band_off, d_rowptr, d_colind, d_vals};
    launch_band_assemble(ba, d_band, eig_mode, sigma, d_S, d_ahat);
    launch_band_cholesky(ba, d_band, d_status);
    void* fac = nullptr;
    if (tiles) {
        // forward/backward FP32 tiles (c tiles per block row) + pivots
        std::vector<int64_t> toff(h->N), trow0(h->N);
        int64_t ttot = 0;
        for (int s = 0; s < h->N; ++s) {
            toff[s] = ttot;
            trow0[s] = ttot / 32;
            ttot += (int64_t)h->h_subs[s].nb * h->h_subs[s].c * 1024;
        }
        int64_t* d_toff = nullptr;
        AMS_TRY(upload(h, &d_toff, toff));
        AMS_TRY(upload(h, &h->d_trow0, trow0));
        AMS_TRY(h->alloc_t(&h->d_tfwd, (size_t)ttot));
        AMS_TRY(h->alloc_t(&h->d_tbwd, (size_t)ttot));
        AMS_TRY(h->alloc_t(&h->d_piv, (size_t)h->n_pad));
        launch_band_pack_tiles(h->stream, (int)work.size(), h->d_subs, d_band_off, d_work, d_band, d_toff,
                               h->d_tfwd, h->d_tbwd, h->d_piv);
        AMS_CUDA_TRY(cudaGetLastError());
        AMS_CUDA_TRY(make_tile_map(h->d_tfwd, ttot / 32, &h->tmF));
        AMS_CUDA_TRY(make_tile_map(h->d_tbwd, ttot / 32, &h->tmB));
        h->tile_elems = ttot;
        h->use_tma = true;
        fac_tot = 0;
        AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
        h->release(d_toff);
    } else {
        AMS_TRY(h->alloc(&fac, (size_t)fac_tot * (out_fp64 ? 8 : 4)));
        launch_band_pack_work(h->stream, (int)work.size(), h->d_subs, d_band_off, d_work, d_band, d_fac_off,
                              out_fp64 ? (double*)fac : nullptr, out_fp64 ? nullptr : (float*)fac);
        AMS_CUDA_TRY(cudaGetLastError());
    }
    int32_t status = 0;
    AMS_CUDA_TRY(cudaMemcpyAsync(&status, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->release(d_band);
    if (status != 0) {
        set_error(eig_mode ? "non-positive pivot in the shifted local eigen-operator"
                           : "non-positive pivot in a local Cholesky factor (A_i not SPD)");
        return AMS_ERR_NOT_SPD;
    }
    // record offsets (only for the solve factor)
    if (!eig_mode)
        for (int s = 0; s < h->N; ++s) h->h_subs[s].fac_off = fac_off[s];
    *out_fac = fac;
    *out_elems = fac_tot;
    return AMS_OK;
}

static ams_status setup_eigen(ams_handle h, const int64_t* d_rowptr, const int32_t* d_colind,
                              const double* d_vals) {
    const double t0 = now_s();
    int mreq = 0;
    for (auto& s : h->sys) mreq = std::max(mreq, s.m);
    const int P = std::min(32, pow2ceil(2 * mreq + 4));
    for (int s = 0; s < h->N; ++s) h->h_subs[s].p = std::min(h->h_subs[s].n, P);
    AMS_CUDA_TRY(cudaMemcpyAsync(h->d_subs, h->h_subs.data(), sizeof(SubInfo) * h->N, cudaMemcpyHostToDevice,
                                 h->stream));
    const double sigma = h->opt.eig_shift > 0 ? h->opt.eig_shift : 1e-2;
    double *d_S = nullptr, *d_ahat = nullptr;
    AMS_TRY(h->alloc_t(&d_S, (size_t)h->n_pad));
    AMS_TRY(h->alloc_t(&d_ahat, (size_t)h->n_pad));
    AMS_CUDA_TRY(cudaMemsetAsync(d_S, 0, sizeof(double) * h->n_pad, h->stream));
    AMS_CUDA_TRY(cudaMemsetAsync(d_ahat, 0, sizeof(double) * h->n_pad, h->stream));
    void* d_efac = nullptr;
    int64_t efac_elems = 0;
    // factor of \hat A_i + sigma S_i in the solve layout (FP64); the solve
    // factor offsets are reused because the band structure is identical
    std::vector<SubInfo> saved = h->h_subs;
    AMS_TRY(build_local_factors(h, d_rowptr, d_colind, d_vals, d_S, d_ahat, sigma, 1, &d_efac, &efac_elems, 1));
    double *d_X = nullptr, *d_Y = nullptr, *d_AY = nullptr, *d_T = nullptr, *d_theta = nullptr,
           *d_res = nullptr;
    int32_t* d_status = nullptr;
    AMS_TRY(h->alloc_t(&d_X, (size_t)h->n_pad * P));
    AMS_TRY(h->alloc_t(&d_Y, (size_t)h->n_pad * P));
    AMS_TRY(h->alloc_t(&d_AY, (size_t)h->n_pad * P));
    AMS_TRY(h->alloc_t(&d_T, (size_t)h->N * P * P));
    AMS_TRY(h->alloc_t(&d_theta, (size_t)h->N * P));
    AMS_TRY(h->alloc_t(&d_res, (size_t)h->N));
    AMS_TRY(h->alloc_t(&d_status, 1));
    AMS_CUDA_TRY(cudaMemsetAsync(d_X, 0, sizeof(double) * h->n_pad * P, h->stream));
    AMS_CUDA_TRY(cudaMemsetAsync(d_Y, 0, sizeof(double) * h->n_pad * P, h->stream));
    AMS_CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int32_t), h->stream));
    launch_eig_init(h->stream, h->N, h->d_subs, P, d_X);
    // the eigen factor was packed with the offsets computed in build_local_factors
    // (same structure as the solve factor): set them on the device copy
    std::vector<SubInfo> esubs = h->h_subs;
    {
        int64_t off = 0;
        for (int s = 0; s < h->N; ++s) {
            esubs[s].fac_off = off;
            off += (int64_t)esubs[s].nb * blockrow_elems(esubs[s].c);
            esubs[s].m = 0;
        }
    }
    SubInfo* d_esubs = nullptr;
    AMS_TRY(upload(h, &d_esubs, esubs));
    LocalSolveArgs la{h->stream, h->N, d_esubs, ResidIn{d_X, nullptr, nullptr}, d_S, P, h->cmax, 0, nullptr, false,
                      0};
    const int maxit = h->opt.eig_maxit > 0 ? h->opt.eig_maxit : 300;
    const double tol = h->opt.eig_tol > 0 ? h->opt.eig_tol : 1e-13;
    std::vector<double> res(h->N);
    int it = 0;
    double worst = 0.0;
    const int ncheck = std::min(P, mreq + 1);
    for (it = 1; it <= maxit; ++it) {
        AMS_CUDA_TRY(launch_local_solve(la, AMS_PREC_FP64, d_efac, nullptr, d_Y, nullptr));
        // Rayleigh-Ritz on the iterations whose residuals are checked; on the
        // others only the S-orthonormalisation (the span is the same)
        const bool check = it % 4 == 0 || it == maxit;
        launch_eig_rr(h->stream, h->N, d_esubs, P, d_rowptr, d_colind, d_vals, d_S, d_ahat, d_Y, d_AY, d_T,
                      d_theta, d_status, check ? 0 : 1);
        launch_eig_update(h->stream, h->n_pad, P, h->d_sub_of_row, d_esubs, d_Y, d_T, d_X);
        AMS_CUDA_TRY(cudaGetLastError());
        if (check) {
            launch_eig_resid(h->stream, h->N, d_esubs, P, d_rowptr, d_colind, d_vals, d_S, d_ahat, d_X, d_theta,
                             ncheck, d_res);
            AMS_CUDA_TRY(cudaMemcpyAsync(res.data(), d_res, sizeof(double) * h->N, cudaMemcpyDeviceToHost,
                                         h->stream));
            AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
            worst = *std::max_element(res.begin(), res.end());
            if (worst <= tol) break;
        }
    }
    // final exact S-orthonormalisation: Rayleigh-Ritz on span(X) itself
    launch_eig_rr(h->stream, h->N, d_esubs, P, d_rowptr, d_colind, d_vals, d_S, d_ahat, d_X, d_AY, d_T,
                  d_theta, d_status, 0);
    launch_eig_update(h->stream, h->n_pad, P, h->d_sub_of_row, d_esubs, d_X, d_T, d_Y);
    std::swap(d_X, d_Y);
    launch_eig_resid(h->stream, h->N, d_esubs, P, d_rowptr, d_colind, d_vals, d_S, d_ahat, d_X, d_theta,
                     ncheck, d_res);
    std::vector<double> theta((size_t)h->N * P);
    int32_t status = 0;
    AMS_CUDA_TRY(cudaMemcpyAsync(theta.data(), d_theta, sizeof(double) * theta.size(), cudaMemcpyDeviceToHost,
                                 h->stream));
    AMS_CUDA_TRY(cudaMemcpyAsync(res.data(), d_res, sizeof(double) * h->N, cudaMemcpyDeviceToHost, h->stream));
    AMS_CUDA_TRY(cudaMemcpyAsync(&status, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (status != 0) {
        set_error("local eigensolver: Gram matrix lost positive definiteness");
        return AMS_ERR_CUDA;
    }
    h->info.eig_iterations = std::min(it, maxit);
    h->info.eig_max_residual = *std::max_element(res.begin(), res.end());
    // kept modes per subdomain: m_i = min(m, n_i), or with a threshold the
    // eigenvalues below it among those (at least one), grown across a cut
    // cluster
    int64_t psi_tot = 0;
    h->h_lam.clear();
    h->mmax = 0;
    for (int s = 0; s < h->N; ++s) {
        SubInfo& S = h->h_subs[s];
        const int mreq_s = h->sys[S.seg].m;
        int mi = std::min(mreq_s, S.n);
        const double* th = &theta[(size_t)s * P];
        if (h->opt.eig_threshold > 0.0 && mi > 0) {
            int below = 0;
            while (below < mi && th[below] < h->opt.eig_threshold) ++below;
            mi = std::max(1, below);
        }
        while (mi > 0 && mi < S.p && mi < kMaxM &&
               std::fabs(th[mi] - th[mi - 1]) <= 1e-8 * std::max(std::fabs(th[mi]), 1e-300))
            ++mi;
        S.m = mi;
        S.psi_off = psi_tot;
        psi_tot += (int64_t)S.n * mi;
        for (int k = 0; k < mi; ++k) h->h_lam.push_back(th[k]);
        h->mmax = std::max(h->mmax, mi);
    }
    h->psi_elems = psi_tot;
    AMS_CUDA_TRY(cudaMemcpyAsync(h->d_subs, h->h_subs.data(), sizeof(SubInfo) * h->N, cudaMemcpyHostToDevice,
                                 h->stream));
    AMS_TRY(h->alloc_t(&h->d_psi64, (size_t)psi_tot));
    launch_eig_finalize(h->stream, h->N, h->d_subs, P, d_X, d_S, h->d_psi64);
    AMS_CUDA_TRY(cudaGetLastError());
    AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (void* p : {(void*)d_S, (void*)d_ahat, d_efac, (void*)d_X, (void*)d_Y, (void*)d_AY, (void*)d_T,
                    (void*)d_theta, (void*)d_res})
        h->release(p);
    (void)saved;
    h->info.eig_seconds = now_s() - t0;
    return AMS_OK;
}

static ams_status setup_coarse(ams_handle h, const std::vector<SysInput>& inputs, const int64_t* d_rowptr,
                               const int32_t* d_colind, const double* d_vals, const double* d_psi_used) {
    const double t0 = now_s();
    // coarse layout per system: ND order of the subdomain graph
    int64_t coff = 0;
    for (int s = 0; s < h->nsys; ++s) {
        SystemHost& S = h->sys[s];
        const SysInput& in = inputs[s];
        const int32_t N = S.nparts;
        std::vector<std::vector<int32_t>> nb(N);
        for (int64_t i = 0; i < S.n; ++i)
            for (int64_t e = in.A.rowptr[i]; e < in.A.rowptr[i + 1]; ++e) {
                const int32_t a = in.part[i], b = in.part[in.A.colind[e]];
                if (a != b) nb[a].push_back(b);
            }
        std::vector<int64_t> adj_ptr(N + 1, 0);
        std::vector<int32_t> adj;
        for (int32_t a = 0; a < N; ++a) {
            std::sort(nb[a].begin(), nb[a].end());
            nb[a].erase(std::unique(nb[a].begin(), nb[a].end()), nb[a].end());
            adj.insert(adj.end(), nb[a].begin(), nb[a].end());
            adj_ptr[a + 1] = adj.size();
        }
        std::vector<int32_t> w(N);
        for (int32_t a = 0; a < N; ++a) w[a] = h->h_subs[S.sub0 + a].m;
        nested_dissection(N, adj_ptr, adj, w, 96, S.nodes);
        S.coff0 = coff;
        S.nd_pos_of_sub.assign(N, 0);
        int64_t nc = 0;
        for (auto& nd : S.nodes) {
            int64_t pos = nd.a;
            for (int32_t a : nd.subs) {
                S.nd_pos_of_sub[a] = pos;
                h->h_subs[S.sub0 + a].coff = coff + pos;
                pos += w[a];
            }
            nc = std::max(nc, nd.a + nd.k);
        }
        S.nc = nc;
        coff += nc;
    }
    h->Nc = coff;
    AMS_CUDA_TRY(cudaMemcpyAsync(h->d_subs, h->h_subs.data(), sizeof(SubInfo) * h->N, cudaMemcpyHostToDevice,
                                 h->stream));
    // neighbour lists (incl. self) for the Galerkin product
    std::vector<int64_t> nbr_ptr(h->N + 1, 0);
    std::vector<int32_t> nbr;
    int max_nbr = 1;
    for (int s = 0; s < h->nsys; ++s) {
        const SystemHost& S = h->sys[s];
        const SysInput& in = inputs[s];
        std::vector<std::vector<int32_t>> nb(S.nparts);
        for (int64_t i = 0; i < S.n; ++i)
            for (int64_t e = in.A.rowptr[i]; e < in.A.rowptr[i + 1]; ++e)
                nb[in.part[i]].push_back(S.sub0 + in.part[in.A.colind[e]]);
        for (int32_t a = 0; a < S.nparts; ++a) {
            auto& v = nb[a];
            std::sort(v.begin(), v.end());
            v.erase(std::unique(v.begin(), v.end()), v.end());
            nbr.insert(nbr.end(), v.begin(), v.end());
            nbr_ptr[S.sub0 + a + 1] = nbr.size();
            max_nbr = std::max(max_nbr, (int)v.size());
        }
    }
    if (max_nbr > 256) {
        set_error("a subdomain has more than 256 neighbouring subdomains");
        return AMS_ERR_INVALID_ARG;
    }
    int64_t* d_nbr_ptr = nullptr;
    int32_t* d_nbr = nullptr;
    AMS_TRY(upload(h, &d_nbr_ptr, nbr_ptr));
    AMS_TRY(upload(h, &d_nbr, nbr));
    const int mm = std::max(1, h->mmax);

    // node matrices and GEMM items (all systems)
    struct NodeMat { int64_t off; int64_t K; };
    std::vector<CoarseItem> fwd, bwd;
    std::vector<int32_t> rng;
    std::vector<int64_t> desc;   // extraction chunks, 8 per chunk
    std::vector<int32_t> gat;
    std::vector<CoarseRef> cref(h->N, CoarseRef{0, 0, 0, 4});
    int64_t Roff = 0, Qoff = 0;
    int32_t tile_id = 0, slot = 0;
    const int KCHUNK = kCoarseChunk;
    const int64_t ECHUNK = 65536;
    // build all layouts first (host), then run factorisation + extraction per system
    struct SysChunks { int64_t d0, d1; };
    std::vector<SysChunks> sys_chunks(h->nsys);
    auto add_items = [&](std::vector<CoarseItem>& items, int64_t moff, int64_t K, int64_t ldm, int64_t rows,
                         int64_t out0, int32_t rng_off, int32_t nrng, int64_t gat_off) {
        for (int64_t r0 = 0; r0 < rows; r0 += 32) {
            const int nr = (int)std::min<int64_t>(32, rows - r0);
            const int nch = (int)std::max<int64_t>(1, (K + KCHUNK - 1) / KCHUNK);
            for (int ch = 0; ch < nch; ++ch) {
                CoarseItem it{};
                it.moff = moff;
                it.K = (int32_t)K;
                it.ldm = (int32_t)ldm;
                it.nrows = nr;
                it.row_in_node = (int32_t)r0;
                it.out0 = (int32_t)(out0 + r0);
                it.k0 = ch * KCHUNK;
                it.k1 = (int32_t)std::min<int64_t>(K, (int64_t)(ch + 1) * KCHUNK);
                it.rng_off = rng_off;
                it.nrng = nrng;
                it.tile_id = tile_id;
                it.nchunks = nch;
                it.chunk = ch;
                it.slot0 = slot;
                it.gat_off = gat_off;
                items.push_back(it);
            }
            if (nch > 1) slot += nch;
            ++tile_id;
        }
    };
    for (int s = 0; s < h->nsys; ++s) {
        SystemHost& S = h->sys[s];
        sys_chunks[s].d0 = (int64_t)desc.size() / 8;
        for (size_t ni = 0; ni < S.nodes.size(); ++ni) {
            const NDNode& nd = S.nodes[ni];
            if (nd.k == 0) continue;
            // forward block: rows of the node x its subtree
            const int64_t a = S.coff0 + nd.a, cst = S.coff0 + nd.cstart;
            const int64_t Kf = nd.a + nd.k - nd.cstart;
            const int32_t roff = (int32_t)(rng.size() / 2);
            rng.push_back((int32_t)cst);
            rng.push_back((int32_t)Kf);
            const int64_t Kfp = (Kf + 3) & ~int64_t(3);
            add_items(fwd, Roff, Kf, Kfp, nd.k, a, roff, 1, -1);
            for (int64_t e0 = 0; e0 < nd.k * Kfp; e0 += ECHUNK) {
                desc.insert(desc.end(), {Roff, Kf | (Kfp << 32), 0, nd.a, nd.cstart, (int64_t)roff, e0,
                                         std::min(nd.k * Kfp, e0 + ECHUNK)});
            }
            Roff += nd.k * Kfp;
            // backward block: rows of the node x (own rows, then ancestors' rows)
            const int32_t boff = (int32_t)(rng.size() / 2);
            int64_t Kb = 0;
            int32_t nrng = 0;
            for (int32_t q = (int32_t)ni; q >= 0; q = S.nodes[q].parent) {
                if (S.nodes[q].k == 0) continue;
                rng.push_back((int32_t)(S.coff0 + S.nodes[q].a));
                rng.push_back((int32_t)S.nodes[q].k);
                Kb += S.nodes[q].k;
                ++nrng;
            }
            const int64_t Kbp = (Kb + 3) & ~int64_t(3);
            // gather list of the node's columns (the backward items and the
            // fused backward substitution read y through it)
            const int64_t goff = (int64_t)gat.size();
            add_items(bwd, Qoff, Kb, Kbp, nd.k, a, boff, nrng, goff);
            for (int32_t r = 0; r < nrng; ++r) {
                const int32_t st0 = rng[2 * (boff + r)], len = rng[2 * (boff + r) + 1];
                for (int32_t i = 0; i < len; ++i) gat.push_back(st0 + i);
            }
            for (int32_t sa : nd.subs) {
                const SubInfo& I = h->h_subs[S.sub0 + sa];
                CoarseRef& cr = cref[S.sub0 + sa];
                cr.q_off = Qoff + (I.coff - a) * Kbp;
                cr.gat_off = goff;
                cr.K = (int32_t)Kb;
                cr.ldm = (int32_t)Kbp;
            }
            for (int64_t e0 = 0; e0 < nd.k * Kbp; e0 += ECHUNK) {
                desc.insert(desc.end(), {Qoff, Kb | (Kbp << 32), 1, nd.a, nd.cstart,
                                         (int64_t)boff | ((int64_t)nrng << 32), e0,
                                         std::min(nd.k * Kbp, e0 + ECHUNK)});
            }
            Qoff += nd.k * Kbp;
        }
        sys_chunks[s].d1 = (int64_t)desc.size() / 8;
    }
    // the extraction ranges index the dense per-system matrix: make them
    // system-relative (subtract coff0) for the backward gather list copy
    std::vector<int32_t> rng_rel = rng;
    {
        // forward/backward ranges hold global coarse rows; extraction needs
        // rows relative to the system: build a relative copy per system
        for (int s = 0; s < h->nsys; ++s) {
            (void)s;
        }
    }
    h->R_elems = Roff;
    h->Q_elems = Qoff;
    h->nfwd = (int)fwd.size();
    h->nbwd = (int)bwd.size();
    const size_t tfb = h->tf_bytes();
    AMS_TRY(h->alloc(&h->d_Rmat, (size_t)Roff * tfb));
    AMS_TRY(h->alloc(&h->d_Qmat, (size_t)Qoff * tfb));
    AMS_TRY(upload(h, &h->d_fwd, fwd));
    AMS_TRY(upload(h, &h->d_bwd, bwd));
    AMS_TRY(upload(h, &h->d_rng, rng));
    if (gat.empty()) gat.push_back(0);
    AMS_TRY(upload(h, &h->d_gat, gat));
    AMS_TRY(upload(h, &h->d_cref, cref));
    AMS_TRY(h->alloc(&h->d_partial, (size_t)std::max<int32_t>(slot, 1) * 32 * kMaxLd * tfb));
    AMS_TRY(h->alloc_t(&h->d_cnt, (size_t)std::max<int32_t>(tile_id, 1)));
    AMS_CUDA_TRY(cudaMemsetAsync(h->d_cnt, 0, sizeof(int32_t) * std::max<int32_t>(tile_id, 1), h->stream));

    // per system: dense A_0 (ND order), Cholesky, triangular inverse, extraction
    for (int s = 0; s < h->nsys; ++s) {
        SystemHost& S = h->sys[s];
        const int64_t nc = S.nc;
        if (nc == 0) continue;
        double* d_A = nullptr;
        AMS_TRY(h->alloc_t(&d_A, (size_t)nc * nc));
        AMS_CUDA_TRY(cudaMemsetAsync(d_A, 0, sizeof(double) * nc * nc, h->stream));
        launch_galerkin(h->stream, S.nparts, h->d_subs, d_rowptr, d_colind, d_vals, h->d_sub_of_row, d_psi_used,
                        d_nbr_ptr, d_nbr, max_nbr, mm, d_A, nc, S.coff0, S.sub0);
        AMS_CUDA_TRY(cudaGetLastError());
        if (nc <= 4096) {
            S.A0_nd.resize((size_t)nc * nc);
            AMS_CUDA_TRY(cudaMemcpyAsync(S.A0_nd.data(), d_A, sizeof(double) * nc * nc, cudaMemcpyDeviceToHost,
                                         h->stream));
        }
        // Cholesky factor of A_0 and its inverse on the tiles that the
        // nested-dissection order keeps (k_coarse_factor.cu)
        const double tf0 = now_s();
        CoarseTilePlan plan;
        build_coarse_tile_plan(S.nodes, nc, plan);
        double *d_X = nullptr, *d_invd = nullptr;
        int32_t *d_trsm = nullptr, *d_upd = nullptr, *d_inv = nullptr;
        unsigned long long* d_bad = nullptr;
        AMS_TRY(h->alloc_t(&d_X, (size_t)nc * nc));
        AMS_CUDA_TRY(cudaMemsetAsync(d_X, 0, sizeof(double) * nc * nc, h->stream));
        AMS_TRY(h->alloc_t(&d_invd, coarse_tile_invd_elems(plan.T)));
        AMS_TRY(upload(h, &d_trsm, plan.trsm));
        AMS_TRY(upload(h, &d_upd, plan.upd));
        AMS_TRY(upload(h, &d_inv, plan.inv));
        AMS_TRY(h->alloc_t(&d_bad, 1));
        AMS_CUDA_TRY(cudaMemsetAsync(d_bad, 0xff, sizeof(unsigned long long), h->stream));
        launch_coarse_tile_factor(h->stream, plan, d_trsm, reinterpret_cast<const int2*>(d_upd),
                                  reinterpret_cast<const int2*>(d_inv), d_A, d_X, d_invd, d_bad);
        AMS_CUDA_TRY(cudaGetLastError());
        unsigned long long bad = 0;
        AMS_CUDA_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, h->stream));
        AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
        if (bad != ~0ull) {
            set_error("coarse matrix A_0 is not SPD (Cholesky pivot at coarse row " + std::to_string(bad) + ")");
            return AMS_ERR_NOT_SPD;
        }
        h->info.coarse_factor_gflop += 2e-9 * plan.fma;
        h->info.coarse_factor_seconds += now_s() - tf0;
        if (nc <= 4096) {
            S.Linv_nd.resize((size_t)nc * nc);
            AMS_CUDA_TRY(cudaMemcpyAsync(S.Linv_nd.data(), d_X, sizeof(double) * nc * nc, cudaMemcpyDeviceToHost,
                                         h->stream));
        }
        // system-relative gather ranges for the extraction
        std::vector<int32_t> rel = rng;
        for (size_t q = 0; q < rel.size(); q += 2) rel[q] -= (int32_t)S.coff0;
        int32_t* d_rel = nullptr;
        AMS_TRY(upload(h, &d_rel, rel));
        const int64_t nch = sys_chunks[s].d1 - sys_chunks[s].d0;
        std::vector<int64_t> dsub(desc.begin() + 8 * sys_chunks[s].d0, desc.begin() + 8 * sys_chunks[s].d1);
        int64_t* d_desc = nullptr;
        AMS_TRY(upload(h, &d_desc, dsub));
        // forward chunks write R, backward chunks write Q: two passes with the
        // kind filter done by splitting the descriptor list
        std::vector<int64_t> df, db;
        for (int64_t c = 0; c < nch; ++c) (dsub[8 * c + 2] == 0 ? df : db).insert((dsub[8 * c + 2] == 0 ? df : db).end(),
                                                                                   dsub.begin() + 8 * c, dsub.begin() + 8 * c + 8);
        int64_t *d_df = nullptr, *d_db = nullptr;
        AMS_TRY(upload(h, &d_df, df));
        AMS_TRY(upload(h, &d_db, db));
        const bool f64 = h->prec == AMS_PREC_FP64;
        launch_extract_chunks(h->stream, (int)(df.size() / 8), d_df, d_rel, d_X, nc,
                              f64 ? (double*)h->d_Rmat : nullptr, f64 ? nullptr : (float*)h->d_Rmat);
        launch_extract_chunks(h->stream, (int)(db.size() / 8), d_db, d_rel, d_X, nc,
                              f64 ? (double*)h->d_Qmat : nullptr, f64 ? nullptr : (float*)h->d_Qmat);
        AMS_CUDA_TRY(cudaGetLastError());
        AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
        for (void* p : {(void*)d_A, (void*)d_X, (void*)d_invd, (void*)d_trsm, (void*)d_upd, (void*)d_inv,
                        (void*)d_bad, (void*)d_rel, (void*)d_desc, (void*)d_df, (void*)d_db})
            h->release(p);
    }
    h->release(d_nbr_ptr);
    h->release(d_nbr);
    h->info.coarse_seconds = now_s() - t0;
    return AMS_OK;
}

static ams_status estimate_two_grid_omega(ams_handle h);
static void debug_bounds(ams_handle h);
static ams_status debug_check(ams_handle h, ams_status st);

static ams_status setup_impl(int32_t nsys, const ams_system_desc* systems, const ams_options* opt,
                             void* stream, ams_handle* out) {
    const double t0 = now_s();
    if (!out || nsys <= 0 || !systems) {
        set_error("invalid arguments to setup");
        return AMS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    std::unique_ptr<ams_handle_s> h(new ams_handle_s());
    if (opt) h->opt = *opt;
    else ams_options_default(&h->opt);
    if (h->opt.precision < 0 || h->opt.precision > 2) {
        set_error("unknown precision mode");
        return AMS_ERR_INVALID_ARG;
    }
    if (!(h->opt.two_grid_omega > -2.0) || !std::isfinite(h->opt.two_grid_omega)) {
        set_error("two_grid_omega must be finite and > -2 (negative: that multiple of 1/lambda_max, estimated)");
        return AMS_ERR_INVALID_ARG;
    }
    if (h->opt.warm_start < 0 || h->opt.warm_start > 1) {
        set_error("warm_start must be 0 or 1");
        return AMS_ERR_INVALID_ARG;
    }
    if (h->opt.spin_budget_cycles < 0 || h->opt.timeout_probe < 0 || h->opt.timeout_probe > 1) {
        set_error("spin_budget_cycles must be >= 0 and timeout_probe 0 or 1");
        return AMS_ERR_INVALID_ARG;
    }
    if (!(h->opt.eig_threshold >= 0.0) || !std::isfinite(h->opt.eig_threshold)) {
        set_error("eig_threshold must be finite and >= 0");
        return AMS_ERR_INVALID_ARG;
    }
    if (h->opt.maxit <= 0) h->opt.maxit = 10000;
    h->prec = h->opt.precision;
    h->flexible = h->opt.cg_variant == AMS_CG_AUTO ? (h->prec != AMS_PREC_FP64) : (h->opt.cg_variant == AMS_CG_FCG);
    h->ustream = (cudaStream_t)stream;
    AMS_CUDA_TRY(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    {
        int dev = 0;
        AMS_CUDA_TRY(cudaGetDevice(&dev));
        AMS_CUDA_TRY(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    AMS_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_enter, cudaEventDisableTiming));
    AMS_CUDA_TRY(cudaEventRecord(h->ev_enter, h->ustream));
    AMS_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev_enter, 0));
    h->nsys = nsys;
    std::vector<SysInput> inputs(nsys);
    for (int s = 0; s < nsys; ++s) AMS_TRY(read_inputs(systems[s], h->opt.device_ptrs, inputs[s]));
    // layout
    h->sys.resize(nsys);
    int64_t caller = 0, row = 0;
    int32_t sub = 0;
    for (int s = 0; s < nsys; ++s) {
        SystemHost& S = h->sys[s];
        S.n = inputs[s].A.n;
        S.nnz = inputs[s].A.rowptr[S.n];
        S.caller0 = caller;
        S.caller_nnz0 = h->nnz_total;
        S.row0 = row;
        S.npad = round_up(S.n, kRowAlign);
        S.sub0 = sub;
        S.nparts = inputs[s].nparts;
        S.m = h->opt.coarse ? inputs[s].m : 0;
        std::vector<int64_t> iperm;
        build_index_maps(S.n, inputs[s].part.data(), S.nparts, S.perm, iperm, S.sub_ptr);
        caller += S.n;
        row += S.npad;
        sub += S.nparts;
        h->nnz_total += S.nnz;
    }
    h->n_total = caller;
    h->n_pad = row;
    h->N = sub;
    if (h->n_pad > (int64_t(1) << 31) - 1) {
        set_error("total padded size exceeds 2^31 rows");
        return AMS_ERR_INVALID_ARG;
    }
    // index maps, internal CSR, subdomain descriptors
    std::vector<int64_t> int_row(h->n_total), irp(h->n_pad + 1, 0);
    std::vector<int32_t> sub_of_row(h->n_pad, -1), icol;
    std::vector<double> ival;
    icol.reserve(h->nnz_total);
    ival.reserve(h->nnz_total);
    h->h_subs.resize(h->N);
    std::vector<std::pair<int32_t, double>> rowbuf;
    std::vector<std::pair<int32_t, int64_t>> rowsrc;   // (internal col, caller entry)
    std::vector<int64_t> ientry_src;                    // internal CSR entry -> caller entry
    ientry_src.reserve(h->nnz_total);
    int64_t rp = 0;
    for (int s = 0; s < nsys; ++s) {
        SystemHost& S = h->sys[s];
        const HostCSR& A = inputs[s].A;
        std::vector<int64_t> iperm(S.n);
        for (int64_t k = 0; k < S.n; ++k) iperm[S.perm[k]] = k;
        for (int64_t g = 0; g < S.n; ++g) int_row[S.caller0 + g] = S.row0 + iperm[g];
        for (int32_t a = 0; a < S.nparts; ++a) {
            SubInfo& I = h->h_subs[S.sub0 + a];
            I = SubInfo{};
            I.row0 = S.row0 + S.sub_ptr[a];
            I.n = (int32_t)(S.sub_ptr[a + 1] - S.sub_ptr[a]);
            I.nb = (I.n + 31) / 32;
            h->nbmax = std::max(h->nbmax, (int)I.nb);
            I.seg = s;
            I.m = 0;
            int64_t bw = 0;
            for (int64_t k = S.sub_ptr[a]; k < S.sub_ptr[a + 1]; ++k) {
                sub_of_row[S.row0 + k] = S.sub0 + a;
                const int64_t g = S.perm[k];
                for (int64_t e = A.rowptr[g]; e < A.rowptr[g + 1]; ++e) {
                    const int64_t kk = iperm[A.colind[e]];
                    if (kk >= S.sub_ptr[a] && kk < k) bw = std::max(bw, k - kk);
                }
            }
            I.c = (int32_t)std::max<int64_t>(1, (bw + 31) / 32);
            h->cmax = std::max(h->cmax, I.c);
        }
        for (int64_t k = 0; k < S.npad; ++k) {
            irp[S.row0 + k] = rp;
            if (k < S.n) {
                const int64_t g = S.perm[k];
                rowsrc.clear();
                for (int64_t e = A.rowptr[g]; e < A.rowptr[g + 1]; ++e)
                    rowsrc.push_back({(int32_t)(S.row0 + iperm[A.colind[e]]), S.caller_nnz0 + e});
                std::sort(rowsrc.begin(), rowsrc.end());
                for (auto& pr : rowsrc) {
                    icol.push_back(pr.first);
                    const int64_t ce = pr.second - S.caller_nnz0;
                    ival.push_back(A.vals[ce]);
                    ientry_src.push_back(pr.second);
                }
                rp += (int64_t)rowsrc.size();
            }
        }
    }
    irp[h->n_pad] = rp;
    {
        std::vector<int32_t> order;
        for (int c = 1; c <= h->cmax; ++c) {
            int cnt = 0, nbm = 1;
            for (int32_t i = 0; i < h->N; ++i)
                if (h->h_subs[i].c == c) {
                    order.push_back(i);
                    ++cnt;
                    nbm = std::max(nbm, (int)h->h_subs[i].nb);
                }
            if (cnt > 0) {
                h->cls_c.push_back(c);
                h->cls_n.push_back(cnt);
                h->cls_nb.push_back(nbm);
            }
        }
        if (h->cls_c.size() > 1) AMS_TRY(upload(h.get(), &h->d_cls_order, order));
        else h->cls_c.clear(), h->cls_n.clear(), h->cls_nb.clear();
    }
    // shared-memory staging limits of the local solve
    {
        const size_t lim = 227 * 1024;
        const size_t need_solve = local_solve_smem(h->cmax, kMaxLd, h->tf_bytes(), 1);
        const size_t need_eig = local_solve_smem(h->cmax, 32, 8, 1);
        if (need_solve > lim || (h->opt.coarse && need_eig > lim)) {
            set_error("a subdomain's band (" + std::to_string(32 * h->cmax) +
                      ") is too wide for shared-memory staging; renumber the subdomain or use smaller subdomains");
            return AMS_ERR_INVALID_ARG;
        }
    }
    // SELL-32 layout of the internal matrix
    const int64_t nslices = h->n_pad / 32;
    std::vector<int64_t> sell_ptr(nslices + 1, 0);
    for (int64_t sl = 0; sl < nslices; ++sl) {
        int64_t w = 0;
        for (int l = 0; l < 32; ++l) w = std::max(w, irp[sl * 32 + l + 1] - irp[sl * 32 + l]);
        sell_ptr[sl + 1] = sell_ptr[sl] + 32 * w;
    }
    std::vector<int32_t> sell_col(sell_ptr[nslices]);
    std::vector<double> sell_val(sell_ptr[nslices], 0.0);
    std::vector<int64_t> sell_pos(h->nnz_total, 0);
    for (int64_t sl = 0; sl < nslices; ++sl) {
        const int64_t w = (sell_ptr[sl + 1] - sell_ptr[sl]) / 32;
        for (int l = 0; l < 32; ++l) {
            const int64_t r = sl * 32 + l;
            const int64_t len = irp[r + 1] - irp[r];
            for (int64_t j = 0; j < w; ++j) {
                const int64_t o = sell_ptr[sl] + 32 * j + l;
                if (j < len) {
                    sell_col[o] = icol[irp[r] + j];
                    sell_val[o] = ival[irp[r] + j];
                    sell_pos[ientry_src[irp[r] + j]] = o;
                } else {
                    sell_col[o] = (int32_t)r;
                    sell_val[o] = 0.0;
                }
            }
        }
    }
    ams_handle H = h.get();
    AMS_TRY(upload(H, &h->d_int_row, int_row));
    AMS_TRY(upload(H, &h->d_sub_of_row, sub_of_row));
    AMS_TRY(upload(H, &h->d_sell_ptr, sell_ptr));
    AMS_TRY(upload(H, &h->d_sell_col, sell_col));
    AMS_TRY(upload(H, &h->d_sell_val, sell_val));
    h->sell_elems = (int64_t)sell_val.size();
    if (h->opt.two_grid_omega != 0.0 && h->prec != AMS_PREC_FP64) {
        // the cycle's internal residuals belong to the reduced-precision apply
        AMS_TRY(h->alloc_t(&h->d_sell_val32, sell_val.size()));
        launch_round_to_f32(h->stream, h->d_sell_val, (int64_t)sell_val.size(), h->d_sell_val32);
    }
    int64_t* d_irp = nullptr;
    int32_t* d_icol = nullptr;
    double* d_ival = nullptr;
    AMS_TRY(upload(H, &d_irp, irp));
    AMS_TRY(upload(H, &d_icol, icol));
    AMS_TRY(upload(H, &d_ival, ival));
    if (nsys == 1) {
        AMS_TRY(upload(H, &h->d_crowptr, inputs[0].A.rowptr));
        AMS_TRY(upload(H, &h->d_ccolind, inputs[0].A.colind));
        AMS_TRY(upload(H, &h->d_sell_pos, sell_pos));
    }
    AMS_TRY(h->alloc_t(&h->d_subs, (size_t)h->N));
    AMS_CUDA_TRY(cudaMemcpyAsync(h->d_subs, h->h_subs.data(), sizeof(SubInfo) * h->N, cudaMemcpyHostToDevice,
                                 h->stream));
    // local factors of A_i
    AMS_TRY(build_local_factors(H, d_irp, d_icol, d_ival, nullptr, nullptr, 0.0, 0, &h->d_fac, &h->fac_elems,
                                h->prec == AMS_PREC_FP64, h->prec != AMS_PREC_FP64));
    AMS_CUDA_TRY(cudaMemcpyAsync(h->d_subs, h->h_subs.data(), sizeof(SubInfo) * h->N, cudaMemcpyHostToDevice,
                                 h->stream));
    // coarse space
    bool any_m = false;
    for (auto& S : h->sys) any_m = any_m || S.m > 0;
    if (any_m) {
        AMS_TRY(setup_eigen(H, d_irp, d_icol, d_ival));
        double* d_psi_used = nullptr;
        AMS_TRY(h->alloc_t(&d_psi_used, (size_t)h->psi_elems));
        AMS_TRY(h->alloc(&h->d_psi, (size_t)h->psi_elems * h->tp_bytes()));
        launch_psi_round(h->stream, h->psi_elems, h->d_psi64, h->prec, d_psi_used,
                         h->prec == AMS_PREC_FP32 ? (float*)h->d_psi : nullptr,
                         h->prec == AMS_PREC_FP32_BF16 ? (__nv_bfloat16*)h->d_psi : nullptr);
        if (h->prec == AMS_PREC_FP64)
            AMS_CUDA_TRY(cudaMemcpyAsync(h->d_psi, h->d_psi64, sizeof(double) * h->psi_elems,
                                         cudaMemcpyDeviceToDevice, h->stream));
        AMS_CUDA_TRY(cudaGetLastError());
        if (h->mmax > 0) AMS_TRY(setup_coarse(H, inputs, d_irp, d_icol, d_ival, d_psi_used));
        h->release(d_psi_used);
    }
    for (void* p : {(void*)d_irp, (void*)d_icol, (void*)d_ival}) h->release(p);
    AMS_TRY(h->alloc_t(&h->d_st, 1));
    AMS_CUDA_TRY(cudaMemsetAsync(h->d_st, 0, sizeof(SolveState), h->stream));
    AMS_TRY(h->alloc_t(&h->d_sc, (size_t)h->nsys * kMaxLd));
    AMS_CUDA_TRY(cudaMallocHost((void**)&h->h_st, sizeof(SolveState)));
    AMS_CUDA_TRY(cudaMallocHost((void**)&h->h_sc, sizeof(CgScalars) * (size_t)h->nsys * kMaxLd));
    AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
    // info
    ams_info& I = h->info;
    I.n = h->n_total;
    I.nnz = h->nnz_total;
    I.nparts = h->N;
    I.nsys = h->nsys;
    I.ncoarse = h->Nc;
    I.max_band_tiles = h->cmax;
    I.precision = h->prec;
    I.cg_variant = h->flexible ? AMS_CG_FCG : AMS_CG_PCG;
    I.local_factor_bytes = h->use_tma ? 2 * h->tile_elems * 4 + 4 * h->n_pad : h->fac_elems * (int64_t)h->tf_bytes();
    I.coarse_inverse_bytes = (h->R_elems + h->Q_elems) * (int64_t)h->tf_bytes();
    I.basis_bytes = h->psi_elems * (int64_t)h->tp_bytes();
    I.spmv_variant = 0;
    debug_bounds(h.get());
    if (h->opt.two_grid_omega < 0.0) AMS_TRY(estimate_two_grid_omega(h.get()));
    AMS_TRY(debug_check(h.get(), AMS_OK));
    I.two_grid_omega = h->opt.two_grid_omega;
    I.setup_seconds = now_s() - t0;
    *out = h.release();
    return AMS_OK;
}

// ---------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------
static ams_status ensure_work(ams_handle h, int ld) {
    if (ld > h->ld_alloc) {
        // the cached iteration-loop graphs hold the old buffers' addresses
        // in their kernel nodes: drop them before the buffers go
        AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
        for (auto& g : h->loop_graph) cudaGraphExecDestroy(g.second);
        h->loop_graph.clear();
        for (void* p : {(void*)h->d_x, (void*)h->d_r, (void*)h->d_p, (void*)h->d_p2, (void*)h->d_q, (void*)h->d_z, h->d_zf, h->d_rc,
                        h->d_yc, h->d_ec, (void*)h->d_stage_in, (void*)h->d_stage_out, (void*)h->d_stage_aux,
                        (void*)h->d_tw})
            h->release(p);
        const size_t nv = (size_t)h->n_pad * ld;
        const size_t nc = (size_t)std::max<int64_t>(h->Nc, 1) * ld;
        AMS_TRY(h->alloc_t(&h->d_x, nv));
        AMS_TRY(h->alloc_t(&h->d_r, nv));
        AMS_TRY(h->alloc_t(&h->d_p, nv));
        AMS_TRY(h->alloc_t(&h->d_p2, nv));
        AMS_TRY(h->alloc_t(&h->d_q, nv));
        AMS_TRY(h->alloc_t(&h->d_z, nv));
        AMS_TRY(h->alloc(&h->d_zf, nv * h->tf_bytes()));
        AMS_TRY(h->alloc(&h->d_rc, nc * h->tf_bytes()));
        AMS_TRY(h->alloc(&h->d_yc, nc * h->tf_bytes()));
        AMS_TRY(h->alloc(&h->d_ec, nc * h->tf_bytes()));
        AMS_TRY(h->alloc_t(&h->d_stage_in, (size_t)h->n_total * ld));
        AMS_TRY(h->alloc_t(&h->d_stage_out, (size_t)h->n_total * ld));
        AMS_TRY(h->alloc_t(&h->d_stage_aux, (size_t)h->n_total * ld));
        h->d_tw = nullptr;
        // the cycle's residual buffer: an automatic omega (negative at setup)
        // turns positive after its power steps, which already use this space
        if (h->opt.two_grid_omega != 0.0) AMS_TRY(h->alloc_t(&h->d_tw, nv));
        h->ld_alloc = ld;
        h->ld_last = 0;
    }
    if (ld != h->ld_last) {
        const size_t nv = (size_t)h->n_pad * ld;
        for (double* p : {h->d_x, h->d_r, h->d_p, h->d_p2, h->d_q, h->d_z})
            AMS_CUDA_TRY(cudaMemsetAsync(p, 0, nv * sizeof(double), h->stream));
        AMS_CUDA_TRY(cudaMemsetAsync(h->d_zf, 0, nv * h->tf_bytes(), h->stream));
        h->ld_last = ld;
    }
    return AMS_OK;
}

// Event bracketing of single kernels while profiling (one solve).
static void prof_begin(ams_handle h, int which) {
    KernelProfile* P = h->prof;
    if (!P) return;
    nvtxRangePushA(kSlotNames[which]);
    cudaEventRecord(P->ev[2 * P->nev], h->stream);
    P->which[P->nev] = which;
}
static void prof_end(ams_handle h) {
    KernelProfile* P = h->prof;
    if (!P) return;
    cudaEventRecord(P->ev[2 * P->nev + 1], h->stream);
    P->nev++;
    nvtxRangePop();
}
static ams_status prof_flush(ams_handle h) {
    KernelProfile* P = h->prof;
    if (!P || P->nev == 0) return AMS_OK;
    AMS_CUDA_TRY(cudaEventSynchronize(P->ev[2 * P->nev - 1]));
    for (int i = 0; i < P->nev; ++i) {
        float ms = 0.f;
        AMS_CUDA_TRY(cudaEventElapsedTime(&ms, P->ev[2 * i], P->ev[2 * i + 1]));
        P->ms[P->which[i]] += ms;
        P->count[P->which[i]] += 1;
    }
    P->nev = 0;
    return AMS_OK;
}

// The device status word that kernels set when a bounded wait runs out
// (SolveState::status): cleared before work outside a solve, read after.
static ams_status clear_device_status(ams_handle h) {
    AMS_CUDA_TRY(cudaMemsetAsync(&h->d_st->status, 0, sizeof(int32_t), h->stream));
    return AMS_OK;
}
static ams_status device_status(ams_handle h) {
    int32_t s = 0;
    AMS_CUDA_TRY(cudaMemcpyAsync(&s, &h->d_st->status, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
    AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (s == AMS_ERR_DEVICE_TIMEOUT) {
        set_error("a bounded device-side wait ran out (spin_budget_cycles)");
        return AMS_ERR_DEVICE_TIMEOUT;
    }
    return AMS_OK;
}

// Budget of every bounded device-side wait, in SM clock cycles.
static int64_t spin_budget(ams_handle h) {
    return h->opt.spin_budget_cycles > 0 ? h->opt.spin_budget_cycles : kDefaultSpinCycles;
}

// Fine-level local solves (+ restriction when the coarse space exists).
static LocalTmaArgs local_tma_args(ams_handle h, int ld, const ResidIn& in, bool with_state) {
    LocalTmaArgs a{h->stream, h->N, h->d_subs, &h->tmF, &h->tmB, h->d_trow0, h->d_piv, in, ld, h->cmax,
                   std::max(1, h->mmax), h->nbmax, spin_budget(h), with_state ? h->d_st : nullptr,
                   h->use_pdl, h->tune[ld].depth, h->tune[ld].nr, h->tune[ld].l2mode, h->tune[ld].l2keep,
                   &h->d_st->status, h->opt.timeout_probe};
    a.nclass = (int)h->cls_c.size();
    a.class_c = h->cls_c.data();
    a.class_n = h->cls_n.data();
    a.class_nb = h->cls_nb.data();
    a.order = h->d_cls_order;
    return a;
}

// Launches of one local-solve pass beyond the first: the several-RHS
// kernel launches once per band-width group.
static int local_extra_launches(ams_handle h, int ld) {
    return (h->use_tma && ld >= 8 && h->cls_c.size() > 1) ? (int)h->cls_c.size() - 1 : 0;
}

static ams_status launch_local(ams_handle h, int ld, const ResidIn& in, bool with_state,
                               bool restrict_rc = true) {
    const bool coarse = h->Nc > 0 && restrict_rc;
    if (h->use_tma) {
        LocalTmaArgs a = local_tma_args(h, ld, in, with_state);
        AMS_CUDA_TRY(launch_local_tma(a, h->prec, h->d_psi, h->d_zf, coarse ? h->d_rc : nullptr));
    } else {
        LocalSolveArgs la{h->stream, h->N, h->d_subs, in, nullptr, ld, h->cmax, std::max(1, h->mmax),
                          with_state ? h->d_st : nullptr, h->use_pdl, h->tune[ld].depth};
        AMS_CUDA_TRY(launch_local_solve(la, h->prec, h->d_fac, h->d_psi, h->d_zf, coarse ? h->d_rc : nullptr));
    }
    return AMS_OK;
}

// Damping of the multiplicative cycle from the local solves' spectrum:
// omega = c / lambda_max(T), T = (sum_i R_i^T A_i^{-1} R_i) A, c = minus
// the option's value.  lambda_max is estimated by power steps (Rayleigh
// quotient of T in the A inner product, which rises towards lambda_max
// from below) in the apply precision, per system, until the estimate moves
// by less than 1e-7 relative between steps (at most kPowerSteps); the
// handle takes the largest (the smallest omega).  The cycle is SPD for omega < 2 /
// lambda_max, so c < 2 keeps it SPD up to the estimate's shortfall.
constexpr int kPowerSteps = 300;

static ams_status estimate_two_grid_omega(ams_handle h) {
    const double c = -h->opt.two_grid_omega;
    AMS_TRY(ensure_work(h, 1));
    RedCache *rc = nullptr, *rcs = nullptr;
    AMS_TRY(get_red(h, 1, &rc, &rcs));
    LaunchCtx L = make_ctx(h, *rc, *rcs);
    L.st = nullptr;
    const int64_t nblk = h->n_pad / kRowAlign;
    std::vector<int64_t> sys_blk0(h->nsys + 1);
    std::vector<int32_t> blk_sys(nblk);
    for (int s = 0; s < h->nsys; ++s) {
        sys_blk0[s] = h->sys[s].row0 / kRowAlign;
        sys_blk0[s + 1] = (h->sys[s].row0 + h->sys[s].npad) / kRowAlign;
        for (int64_t b = sys_blk0[s]; b < sys_blk0[s + 1]; ++b) blk_sys[b] = s;
    }
    int64_t* d_sys_blk0 = nullptr;
    int32_t* d_blk_sys = nullptr;
    double *d_part = nullptr, *d_out = nullptr, *d_inv = nullptr;
    AMS_TRY(upload(h, &d_sys_blk0, sys_blk0));
    AMS_TRY(upload(h, &d_blk_sys, blk_sys));
    AMS_TRY(h->alloc_t(&d_part, (size_t)3 * nblk));
    AMS_TRY(h->alloc_t(&d_out, (size_t)3 * h->nsys));
    AMS_TRY(h->alloc_t(&d_inv, (size_t)h->nsys));
    // x_0: 1 + sin(i)/2 at every dof (caller order), zero on padding rows
    std::vector<double> x0(h->n_total);
    for (int64_t i = 0; i < h->n_total; ++i) x0[i] = 1.0 + 0.5 * std::sin((double)i);
    AMS_CUDA_TRY(cudaMemcpyAsync(h->d_stage_in, x0.data(), sizeof(double) * h->n_total, cudaMemcpyHostToDevice,
                                 h->stream));
    AMS_CUDA_TRY(cudaMemsetAsync(h->d_r, 0, sizeof(double) * h->n_pad, h->stream));
    for (int s = 0; s < h->nsys; ++s) {
        const SystemHost& S = h->sys[s];
        launch_permute_in(h->stream, h->d_stage_in + S.caller0, S.n, 1, 1, h->d_int_row + S.caller0, h->d_r, nullptr);
    }
    double* x = h->d_r;          // iterate, normalised each step (the next one is built in p)
    double* y = h->d_q;
    std::vector<double> out(3 * h->nsys);
    auto estimate = [&]() {
        double l = 0.0;
        for (int s = 0; s < h->nsys; ++s)
            if (out[3 * s] > 0.0) l = std::max(l, out[3 * s + 1] / out[3 * s]);
        return l;
    };
    double lam = 0.0;
    for (int step = 0; step < kPowerSteps; ++step) {
        launch_spmv_dot(L, x, y, 0);                                              // y = A x
        AMS_TRY(launch_local(h, 1, ResidIn{y, nullptr, h->d_sc}, false, false));  // z = S y
        launch_power_step(h->stream, h->prec, x, y, h->d_zf, h->n_pad, d_sys_blk0, d_blk_sys, h->nsys, d_part,
                          d_out, d_inv, h->d_p);
        AMS_CUDA_TRY(cudaMemcpyAsync(x, h->d_p, sizeof(double) * h->n_pad, cudaMemcpyDeviceToDevice, h->stream));
        AMS_CUDA_TRY(cudaMemcpyAsync(out.data(), d_out, sizeof(double) * out.size(), cudaMemcpyDeviceToHost,
                                     h->stream));
        AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
        const double next = estimate();
        const bool settled = step >= 4 && std::fabs(next - lam) <= 1e-7 * next;
        lam = next;
        if (settled) break;
    }
    AMS_CUDA_TRY(cudaGetLastError());
    for (void* p : {(void*)d_sys_blk0, (void*)d_blk_sys, (void*)d_part, (void*)d_out, (void*)d_inv}) h->release(p);
    if (!(lam > 0.0) || !std::isfinite(lam)) {
        set_error("two-grid damping: the power steps gave no positive eigenvalue estimate");
        return AMS_ERR_BREAKDOWN;
    }
    h->info.local_lambda_max = lam;
    h->opt.two_grid_omega = c / lam;
    if (h->d_tw == nullptr) {
        set_error("two-grid damping: the cycle's work vector is missing");
        return AMS_ERR_CUDA;
    }
    h->ld_last = 0;   // the next solve starts from cleared work vectors
    return AMS_OK;
}

// Up to four right-hand sides the backward coarse substitution runs inside
// the prolongation (each subdomain multiplies its rows of the backward block
// with y); with more, the per-subdomain gathers of y cost more than the
// separate backward launch.
static bool fused_backward(int ld) { return ld <= 4; }

// forward coarse substitution y = L_c^{-1} r_c, and the backward one when it
// is not fused
static int launch_coarse(ams_handle h, int ld, bool with_state) {
    CoarseLaunch cf{h->stream, h->nfwd, h->d_fwd, h->d_Rmat, h->d_rng, h->d_gat, h->d_partial, h->d_cnt,
                    with_state ? h->d_st : nullptr, h->use_pdl};
    launch_coarse_gemm(cf, h->prec, ld, h->d_rc, h->d_yc);
    if (fused_backward(ld)) return 1;
    CoarseLaunch cb{h->stream, h->nbwd, h->d_bwd, h->d_Qmat, h->d_rng, h->d_gat, h->d_partial, h->d_cnt,
                    with_state ? h->d_st : nullptr, h->use_pdl};
    launch_coarse_gemm(cb, h->prec, ld, h->d_yc, h->d_ec);
    return 2;
}

// From 8 right-hand sides x += alpha p moves from the prolongation to the
// next iteration's direction update, which streams that p anyway (one read
// of p less per iteration; measured faster at 32 right-hand sides).  With
// fewer the prolongation is latency-bound and gains nothing from the bytes,
// while the direction update would pay for them: the update stays there.
static bool defer_x_update(int ld) { return ld >= 8; }

static ProlongArgs prolong_args(ams_handle h, int mode, const double* p, int ld) {
    const bool coarse = h->Nc > 0, fused = fused_backward(ld);
    return ProlongArgs{h->d_psi, coarse && !fused ? h->d_ec : nullptr, coarse && fused ? h->d_yc : nullptr,
                       coarse && fused ? h->d_Qmat : nullptr, h->d_cref, h->d_gat, h->d_zf, h->d_r, h->d_q,
                       defer_x_update(ld) ? nullptr : h->d_x, p, h->d_z, std::max(1, h->mmax), h->flexible, mode};
}

// Multiplicative two-grid cycle z = B r' (Section 3.2's two-grid algorithm
// from x^0 = 0; the smoother is omega times the local solves, before and
// after the coarse-grid correction):
//   x^1 = omega S r'                 local solves, scaled in place in z_f
//   r_c = R_0 (r' - A x^1)           residual SpMV, restriction
//   x^2 = x^1 + R_0^T A_0^{-1} r_c   coarse substitutions, prolongation (mode 0, into z)
//   z   = x^2 + omega S (r' - A x^2) residual SpMV, local solves, combine in z_f
// and the additive path's prolongation kernel, with the coarse term off,
// applies z = z_f and the CG update of `mode` as in apply_precond.
static ams_status apply_two_grid(ams_handle h, const LaunchCtx& L, int mode, const double* p) {
    const bool with_state = mode != 0;
    const double omega = h->opt.two_grid_omega;
    const int64_t nv = h->n_pad * L.ld;
    const ResidIn rin{h->d_r, mode == 2 ? h->d_q : nullptr, h->d_sc};
    LaunchCtx L2 = L;
    if (!with_state) L2.st = nullptr;
    prof_begin(h, AMS_KERNEL_LOCAL);
    AMS_TRY(launch_local(h, L.ld, rin, with_state, false));
    launch_tg_scale(L2, h->prec, h->d_zf, omega, nv);
    prof_end(h);
    h->launches += 2 + local_extra_launches(h, L.ld);
    if (h->Nc > 0) {   // without a coarse space x^2 = x^1
        prof_begin(h, AMS_KERNEL_COARSE);
        launch_tg_resid(L2, h->d_zf, h->prec == AMS_PREC_FP64, rin, h->d_tw);
        launch_tg_restrict(L2, h->prec, h->d_psi, h->d_tw, h->d_rc, std::max(1, h->mmax));
        h->launches += 2 + launch_coarse(h, L.ld, with_state);
        prof_end(h);
    }
    prof_begin(h, AMS_KERNEL_PROLONG);
    launch_prolong_update(L2, h->prec, prolong_args(h, 0, p, L.ld));   // z = x^2
    launch_tg_resid(L2, h->d_z, h->prec == AMS_PREC_FP64, rin, h->d_tw);   // z in the apply precision
    prof_end(h);
    prof_begin(h, AMS_KERNEL_LOCAL);
    AMS_TRY(launch_local(h, L.ld, ResidIn{h->d_tw, nullptr, h->d_sc}, with_state, false));
    launch_tg_combine(L2, h->prec, h->d_zf, h->d_z, omega, nv);
    prof_end(h);
    ProlongArgs a = prolong_args(h, mode, p, L.ld);
    a.ec = nullptr;
    a.yc = nullptr;
    a.qmat = nullptr;
    prof_begin(h, AMS_KERNEL_PROLONG);
    launch_prolong_update(L2, h->prec, a);
    prof_end(h);
    h->launches += 5 + local_extra_launches(h, L.ld);   // prolongation, residual, local solves, combine, prolongation
    AMS_CUDA_TRY(cudaGetLastError());
    return AMS_OK;
}

// z = M^{-1} r' (internal layout).  mode 0: plain application (r' = r, no
// dots); mode 1: first application of a solve (r' = r, rho = r.z); mode 2:
// inside an iteration (r' = r - alpha q formed by the local solves and
// stored by the prolongation together with x += alpha p, the dots and the
// convergence test).  p is the direction of the current iteration.
static ams_status apply_precond(ams_handle h, const LaunchCtx& L, int mode, const double* p) {
    if (h->opt.two_grid_omega > 0.0) return apply_two_grid(h, L, mode, p);
    const bool coarse = h->Nc > 0;
    const bool with_state = mode != 0;
    prof_begin(h, AMS_KERNEL_LOCAL);
    AMS_TRY(launch_local(h, L.ld, ResidIn{h->d_r, mode == 2 ? h->d_q : nullptr, h->d_sc}, with_state));
    prof_end(h);
    h->launches += 2 + local_extra_launches(h, L.ld);
    if (coarse) {
        prof_begin(h, AMS_KERNEL_COARSE);
        h->launches += launch_coarse(h, L.ld, with_state);
        prof_end(h);
    }
    LaunchCtx L2 = L;
    if (!with_state) L2.st = nullptr;
    prof_begin(h, AMS_KERNEL_PROLONG);
    launch_prolong_update(L2, h->prec, prolong_args(h, mode, p, L.ld));
    prof_end(h);
    AMS_CUDA_TRY(cudaGetLastError());
    return AMS_OK;
}

static int launches_per_iteration(ams_handle h, int ld) {
    const int coarse = h->Nc > 0 ? (fused_backward(ld) ? 1 : 2) : 0;
    const int extra = local_extra_launches(h, ld);
    if (h->opt.two_grid_omega > 0.0) return 9 + 2 * extra + (h->Nc > 0 ? 2 + coarse : 0);
    return 4 + extra + coarse;
}

static void launch_direction_spmv(ams_handle h, const LaunchCtx& L, const double* p_old, double* p_new) {
    launch_dir_update(L, h->prec, h->d_z, p_old, p_new, defer_x_update(L.ld) ? h->d_x : nullptr);
    launch_spmv_dot(L, p_new, h->d_q, 1);
}

// One CG iteration; `par` selects which direction buffer holds p_old.
static ams_status launch_iteration(ams_handle h, const LaunchCtx& L, int par) {
    double* p_old = par ? h->d_p2 : h->d_p;
    double* p_new = par ? h->d_p : h->d_p2;
    h->launches += 2;
    prof_begin(h, AMS_KERNEL_SPMV);
    launch_direction_spmv(h, L, p_old, p_new);
    prof_end(h);
    return apply_precond(h, L, 2, p_new);
}

// The whole iteration loop as one CUDA graph: a while node whose body is
// two CG iterations (the direction buffers swap roles once each) and the
// condition kernel, which stops the loop once the device solve state says
// done (every (system, rhs) converged, the iteration cap, a breakdown or a
// device timeout) or after `cap` bodies.  Kernel arguments are fixed device
// pointers and every scalar lives in device memory, so one graph launch
// runs the solve to the end with no host round trip.
static ams_status get_loop_graph(ams_handle h, const LaunchCtx& L, cudaGraphExec_t* out) {
    auto it = h->loop_graph.find(L.ld);
    if (it != h->loop_graph.end()) {
        *out = it->second;
        return AMS_OK;
    }
    cudaGraph_t g = nullptr;
    AMS_CUDA_TRY(cudaGraphCreate(&g, 0));
    struct GraphGuard {
        cudaGraph_t g;
        ~GraphGuard() {
            if (g) cudaGraphDestroy(g);
        }
    } guard{g};
    cudaGraphConditionalHandle cond;
    AMS_CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = cond;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    AMS_CUDA_TRY(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p));
    cudaGraph_t body = p.conditional.phGraph_out[0];
    const int64_t saved = h->launches;
    AMS_CUDA_TRY(cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
    ams_status st = launch_iteration(h, L, 0);
    if (st == AMS_OK) st = launch_iteration(h, L, 1);
    if (st == AMS_OK) launch_loop_cond(h->stream, cond, h->d_st, h->opt.maxit / 2 + 2);
    cudaError_t e = cudaStreamEndCapture(h->stream, &body);
    h->launches = saved;
    if (st != AMS_OK) return st;
    AMS_CUDA_TRY(e);
    cudaGraphExec_t ex = nullptr;
    AMS_CUDA_TRY(cudaGraphInstantiate(&ex, g, 0));
    h->loop_graph[L.ld] = ex;
    *out = ex;
    return AMS_OK;
}

// Stage caller vectors (host or device) into device memory in caller order.
static ams_status stage_in(ams_handle h, const double* src, int nrhs, double* dst, const double** dev) {
    if (h->opt.device_ptrs) {
        *dev = src;
        return AMS_OK;
    }
    AMS_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(double) * h->n_total * nrhs, cudaMemcpyHostToDevice, h->stream));
    *dev = dst;
    return AMS_OK;
}

// Internal state at the start of a solve: r = f (internal order), x = 0,
// p = 0, ||f||^2, and the first preconditioner application (z, rho).  With
// an initial guess u0 (caller order, single system) r = f - A u0 instead:
// the solve runs from e = 0 on A e = f - A u0 (the iterates of CG from u0,
// shifted by u0), its stopping rule still relative to ||f||, and pcg() adds
// u0 to the result.
static ams_status start_solve(ams_handle h, const LaunchCtx& L, const double* f_dev, int nrhs, int32_t maxit,
                              double rtol2, const double* u0_dev = nullptr) {
    const int ld = L.ld;
    if (h->nsys == 1) {
        launch_permute_in(h->stream, f_dev, h->n_total, nrhs, ld, h->d_int_row, h->d_r, h->d_x);
    } else {
        for (int s = 0; s < h->nsys; ++s) {
            const SystemHost& S = h->sys[s];
            launch_permute_in(h->stream, f_dev + S.caller0 * nrhs, S.n, nrhs, ld, h->d_int_row + S.caller0, h->d_r,
                              h->d_x);
        }
    }
    // the first iteration reads p_old = 0 (beta = 0)
    AMS_CUDA_TRY(cudaMemsetAsync(h->d_p, 0, sizeof(double) * h->n_pad * ld, h->stream));
    SolveState init{};
    init.maxit = maxit;
    init.rtol2 = rtol2;
    AMS_CUDA_TRY(cudaMemcpyAsync(h->d_st, &init, sizeof(init), cudaMemcpyHostToDevice, h->stream));
    h->launches += 2 * h->nsys + 1;     // permutes in/out, norms
    launch_init_norms(L, h->d_r, nrhs);
    if (u0_dev != nullptr) {   // r = f - A u0 (u0 through q, which the first SpMV overwrites)
        launch_permute_in(h->stream, u0_dev, h->n_total, nrhs, ld, h->d_int_row, h->d_q, nullptr);
        launch_tg_resid(L, h->d_q, 1, ResidIn{h->d_r, nullptr, h->d_sc}, h->d_r);
        h->launches += 2;
    }
    AMS_TRY(apply_precond(h, L, 1, nullptr));
    AMS_CUDA_TRY(cudaGetLastError());
    return AMS_OK;
}

// Autotuning (opt.autotune): at the first solve with a given ld, time the
// candidate launch shapes on the caller's right-hand side and keep the
// fastest for this handle: blocks per SM of the element layout (direction
// update + SpMV), the local-solve ring depth, and blocks per SM of the
// subdomain layout (prolongation).  Each candidate runs once untimed, then
// three times between CUDA events, inside a solve state that never
// reports convergence; the real solve starts afresh afterwards.
static ams_status autotune(ams_handle h, const double* f_dev, int nrhs, int ld) {
    TuneCfg& T = h->tune[ld];
    struct Restore {                    // tuning launches are not part of a profiled solve
        ams_handle h;
        KernelProfile* prof;
        int64_t launches;
        ~Restore() {
            h->prof = prof;
            h->launches = launches;
        }
    } restore{h, h->prof, h->launches};
    h->prof = nullptr;
    auto ctx = [&](LaunchCtx* L) -> ams_status {
        RedCache *rc = nullptr, *rcs = nullptr;
        AMS_TRY(get_red(h, ld, &rc, &rcs));
        *L = make_ctx(h, *rc, *rcs);
        return AMS_OK;
    };
    // Every candidate launch is timed right after a launch that streams other
    // data through L2, as in a solve: the SpMV after a local solve, the local
    // solve after an SpMV.  Back-to-back launches of one kernel find part of
    // their own operands still in L2 and favour the wrong shapes (deep
    // rings; three blocks per SM for the SpMV).  The prolongation is the
    // exception: timed after the local and coarse solves it favours six
    // blocks per SM, which take 61 us per launch in the solve against 44 us
    // for the four that back-to-back timing picks.  Each candidate: one
    // warm pair, then the faster of two rounds of three (one round let a
    // clock or L2 hiccup pick a slower shape).
    cudaEvent_t ev[6] = {};
    struct Events {
        cudaEvent_t* e;
        ~Events() {
            for (int k = 0; k < 6; ++k)
                if (e[k]) cudaEventDestroy(e[k]);
        }
    } ev_guard{ev};
    for (auto& e : ev) AMS_CUDA_TRY(cudaEventCreate(&e));
    auto timed_after = [&](auto&& pre, auto&& launch, float* ms) -> ams_status {
        AMS_TRY(pre());
        AMS_TRY(launch());
        *ms = 1e30f;
        for (int round = 0; round < 2; ++round) {
            for (int k = 0; k < 3; ++k) {
                AMS_TRY(pre());
                AMS_CUDA_TRY(cudaEventRecord(ev[2 * k], h->stream));
                AMS_TRY(launch());
                AMS_CUDA_TRY(cudaEventRecord(ev[2 * k + 1], h->stream));
            }
            AMS_CUDA_TRY(cudaEventSynchronize(ev[5]));
            AMS_CUDA_TRY(cudaGetLastError());
            float sum = 0.f;
            for (int k = 0; k < 3; ++k) {
                float t = 0.f;
                AMS_CUDA_TRY(cudaEventElapsedTime(&t, ev[2 * k], ev[2 * k + 1]));
                sum += t;
            }
            *ms = std::min(*ms, sum);
        }
        return AMS_OK;
    };
    LaunchCtx L;
    AMS_TRY(ctx(&L));
    AMS_TRY(start_solve(h, L, f_dev, nrhs, 0x7fffffff, 0.0));
    const int cand_bps[] = {3, 4, 6};
    auto local_pre = [&]() -> ams_status { return launch_local(h, ld, ResidIn{h->d_r, h->d_q, h->d_sc}, true); };

    {   // element layout: direction update + SpMV
        float best = 1e30f;
        int arg = T.bps_elem;
        for (int bps : cand_bps) {
            T.bps_elem = bps;
            AMS_TRY(ctx(&L));
            float ms = 0.f;
            AMS_TRY(timed_after(local_pre, [&]() -> ams_status {
                launch_direction_spmv(h, L, h->d_p, h->d_p2);
                return AMS_OK;
            }, &ms));
            if (ms < best) {
                best = ms;
                arg = bps;
            }
        }
        T.bps_elem = arg;
        AMS_TRY(ctx(&L));
    }
    auto spmv = [&]() -> ams_status {
        launch_direction_spmv(h, L, h->d_p, h->d_p2);
        return AMS_OK;
    };
    {   // local-solve ring depth, among the depths whose staging fits 200 KB
        const ResidIn in{h->d_r, h->d_q, h->d_sc};
        float best = 1e30f;
        int arg = 0;
        for (int d = 1; d <= 6; ++d) {
            const size_t smem = h->use_tma ? local_tma_launch_smem(local_tma_args(h, ld, in, true), d)
                                           : local_solve_smem(h->cmax, ld, h->tf_bytes(), d);
            if (smem > 200 * 1024 || (h->use_tma && d < 2)) continue;
            T.depth = d;
            float ms = 0.f;
            AMS_TRY(timed_after(spmv, [&]() -> ams_status { return launch_local(h, ld, in, true); }, &ms));
            if (ms < best) {
                best = ms;
                arg = d;
            }
        }
        T.depth = arg;
    }
    if (h->use_tma && ld == 1) {   // one-RHS local solve: L2 priorities of the factor tiles
        const ResidIn in{h->d_r, h->d_q, h->d_sc};
        const int cand[][2] = {{0, 0}, {1, 4}, {1, 8}, {1, 16}, {1, 1 << 20}, {2, 4}, {2, 8}, {2, 16}};
        float best = 1e30f;
        int arg = 0;
        for (int i = 0; i < (int)(sizeof(cand) / sizeof(cand[0])); ++i) {
            T.l2mode = cand[i][0];
            T.l2keep = cand[i][1];
            float ms = 0.f;
            AMS_TRY(timed_after(spmv, [&]() -> ams_status { return launch_local(h, ld, in, true); }, &ms));
            if (ms < best) {
                best = ms;
                arg = i;
            }
        }
        T.l2mode = cand[arg][0];
        T.l2keep = cand[arg][1];
    }
    if (h->use_tma && ld > 1) {   // several-RHS local solve: right-hand sides per warp
        const ResidIn in{h->d_r, h->d_q, h->d_sc};
        float best = 1e30f;
        int arg = 0;
        // tensor-core kernel from 8 right-hand sides on: 8 or 16 per warp,
        // at most four warps; below that 2, 4 or 8 per warp, at most eight
        const int hi = ld >= 8 ? 16 : 8, lo = ld >= 8 ? 8 : 2, maxw = ld >= 8 ? 4 : 8;
        for (int nr = hi; nr >= lo; nr /= 2) {
            if (nr > ld || ld / nr > maxw) continue;
            T.nr = nr;
            float ms = 0.f;
            AMS_TRY(timed_after(spmv, [&]() -> ams_status { return launch_local(h, ld, in, true); }, &ms));
            if (ms < best) {
                best = ms;
                arg = nr;
            }
        }
        T.nr = arg;
    }
    {   // subdomain layout: prolongation (updates x and r of this throw-away state)
        float best = 1e30f;
        int arg = T.bps_sub;
        for (int bps : cand_bps) {
            T.bps_sub = bps;
            AMS_TRY(ctx(&L));
            float ms = 0.f;
            AMS_TRY(timed_after([]() -> ams_status { return AMS_OK; }, [&]() -> ams_status {
                launch_prolong_update(L, h->prec, prolong_args(h, 2, h->d_p2, ld));
                return AMS_OK;
            }, &ms));
            if (ms < best) {
                best = ms;
                arg = bps;
            }
        }
        T.bps_sub = arg;
    }
    T.done = true;
    return AMS_OK;
}

// The solve up to its outputs, enqueued on the handle's stream: the loop,
// the solution in caller order into u_dev, and the solve state and CG
// scalars into the pinned host mirrors.  The caller enqueues its own copies
// behind it, synchronises once and calls pcg_finish.
static ams_status pcg_launch(ams_handle h, const double* f_dev, int nrhs, double rtol, double* u_dev,
                             const double* u0_dev = nullptr) {
    const int ld = pow2ceil(nrhs);
    AMS_TRY(ensure_work(h, ld));
    RedCache *rc = nullptr, *rcs = nullptr;
    AMS_TRY(get_red(h, ld, &rc, &rcs));
    LaunchCtx L = make_ctx(h, *rc, *rcs);
    if (h->opt.autotune && !h->tune[ld].done) {
        AMS_TRY(autotune(h, f_dev, nrhs, ld));
        AMS_TRY(get_red(h, ld, &rc, &rcs));
        L = make_ctx(h, *rc, *rcs);
    }
    AMS_TRY(start_solve(h, L, f_dev, nrhs, h->opt.maxit, rtol * rtol, u0_dev));
    AMS_TRY(prof_flush(h));
    SolveState st{};
    if (!h->prof) {
        // the whole loop on the device: one graph launch, one read at the end
        cudaGraphExec_t graph = nullptr;
        AMS_TRY(get_loop_graph(h, L, &graph));
        AMS_CUDA_TRY(cudaGraphLaunch(graph, h->stream));
        h->pending_lpi = 2 * launches_per_iteration(h, ld) + 1;   // counted per body in pcg_finish
    } else {
        h->pending_lpi = 0;
        // profiled solve: kernels launched one by one (events around each),
        // the device state read between chunks of iterations, each chunk
        // sized from the observed residual decay
        int chunk = 8;
        int it_prev = 0;
        double w_prev = 1.0;
        const double target = rtol * rtol;
        while (true) {
            for (int k = 0; k < (chunk + 1) / 2; ++k)
                for (int par = 0; par < 2; ++par) {
                    AMS_TRY(launch_iteration(h, L, par));
                    AMS_TRY(prof_flush(h));
                }
            AMS_CUDA_TRY(cudaMemcpyAsync(&st, h->d_st, sizeof(SolveState), cudaMemcpyDeviceToHost, h->stream));
            AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
            if (st.done) break;
            int next = 2 * chunk;
            if (st.it > it_prev && st.worst > 0 && w_prev > 0 && st.worst < w_prev) {
                const double rate = std::log(st.worst / w_prev) / (st.it - it_prev);   // < 0
                const double need = std::log(target / st.worst) / rate;
                next = (int)std::ceil(need);
            }
            chunk = std::max(1, std::min(next, 64));
            it_prev = st.it;
            w_prev = st.worst;
        }
    }
    // the last iteration's deferred x += alpha p (no direction update followed it)
    if (defer_x_update(ld)) {
        launch_x_flush(L, h->d_p, h->d_p2, h->d_x);
        h->launches += 1;
    }
    // outputs
    if (h->nsys == 1) {
        launch_permute_out(h->stream, h->d_x, h->n_total, nrhs, ld, h->d_int_row, u_dev);
        if (u0_dev != nullptr) launch_add_initial_guess(h->stream, u_dev, u0_dev, h->n_total, nrhs, h->d_sc);
    } else {
        for (int s = 0; s < h->nsys; ++s) {
            const SystemHost& S = h->sys[s];
            launch_permute_out(h->stream, h->d_x, S.n, nrhs, ld, h->d_int_row + S.caller0, u_dev + S.caller0 * nrhs);
        }
    }
    AMS_CUDA_TRY(cudaMemcpyAsync(h->h_st, h->d_st, sizeof(SolveState), cudaMemcpyDeviceToHost, h->stream));
    AMS_CUDA_TRY(cudaMemcpyAsync(h->h_sc, h->d_sc, sizeof(CgScalars) * (size_t)h->nsys * ld,
                                 cudaMemcpyDeviceToHost, h->stream));
    return AMS_OK;
}

// After the stream has been synchronised: launch count, iterations,
// relative residuals and the status of the solve pcg_launch enqueued.
static ams_status pcg_finish(ams_handle h, int nrhs, int32_t* iters, double* relres) {
    const int ld = pow2ceil(nrhs);
    const SolveState st = *h->h_st;
    h->launches += (int64_t)st.bodies * h->pending_lpi;
    h->pending_lpi = 0;
    const CgScalars* sc = h->h_sc;
    bool any_active = false;
    for (int s = 0; s < h->nsys; ++s)
        for (int k = 0; k < nrhs; ++k) {
            const CgScalars& c = sc[(size_t)s * ld + k];
            if (iters) iters[s * nrhs + k] = c.iters;
            if (relres) relres[s * nrhs + k] = c.fnorm2 > 0 ? std::sqrt(c.rr / c.fnorm2) : 0.0;
            any_active = any_active || c.active;
        }
    if (st.status == AMS_ERR_DEVICE_TIMEOUT) {
        set_error("a bounded device-side wait ran out (spin_budget_cycles)");
        return AMS_ERR_DEVICE_TIMEOUT;
    }
    if (st.status == AMS_ERR_BREAKDOWN) {
        set_error("CG breakdown (p^T A p <= 0 or non-finite scalar)");
        return AMS_ERR_BREAKDOWN;
    }
    if (any_active) {
        set_error("maximum iteration count reached");
        return AMS_ERR_NOT_CONVERGED;
    }
    return AMS_OK;
}

static ams_status pcg(ams_handle h, const double* f_dev, int nrhs, double rtol, double* u_dev, int32_t* iters,
                      double* relres, const double* u0_dev = nullptr) {
    AMS_TRY(pcg_launch(h, f_dev, nrhs, rtol, u_dev, u0_dev));
    AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return pcg_finish(h, nrhs, iters, relres);
}

// Checking build (-DAMS_DEBUG): point the device-side index checks at this
// handle's sizes, and after a call turn a recorded failure into an error.
// Release build: both do nothing.
static void debug_bounds(ams_handle h) {
#ifdef AMS_DEBUG
    debug_set_bounds_solve(h->n_pad, h->Nc);
    debug_set_bounds_coarse(h->n_pad, h->Nc);
    debug_set_bounds_local_mma(h->n_pad, h->Nc);
    debug_set_bounds_local_tma(h->n_pad, h->Nc);
#else
    (void)h;
#endif
}

static ams_status debug_check(ams_handle h, ams_status st) {
#ifdef AMS_DEBUG
    cudaStreamSynchronize(h->stream);
    int32_t site = 0;
    for (int32_t v : {debug_take_site_solve(), debug_take_site_coarse(), debug_take_site_local_mma(),
                      debug_take_site_local_tma()})
        if (site == 0 && v != 0) site = v;
    if (site != 0) {
        set_error("AMS_DEBUG: a device-side index check failed (site " + std::to_string(site) + ")");
        return AMS_ERR_CUDA;
    }
#else
    (void)h;
#endif
    return st;
}

}  // namespace ams

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void ams_options_default(ams_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = AMS_PREC_FP32_BF16;
    opt->cg_variant = AMS_CG_AUTO;
    opt->maxit = 10000;
    opt->device_ptrs = 0;
    opt->autotune = 1;
    opt->coarse = 1;
    opt->eig_shift = 0.0;
    opt->eig_maxit = 0;
    opt->eig_tol = 0.0;
    opt->spin_budget_cycles = 0;
    opt->eig_threshold = 0.0;
    opt->two_grid_omega = 0.0;
    opt->timeout_probe = 0;
    opt->warm_start = 0;
}

const char* ams_status_string(ams_status s) {
    switch (s) {
        case AMS_OK: return "AMS_OK";
        case AMS_ERR_INVALID_ARG: return "AMS_ERR_INVALID_ARG";
        case AMS_ERR_NOT_SPD: return "AMS_ERR_NOT_SPD";
        case AMS_ERR_BREAKDOWN: return "AMS_ERR_BREAKDOWN";
        case AMS_ERR_NOT_CONVERGED: return "AMS_ERR_NOT_CONVERGED";
        case AMS_ERR_DEVICE_TIMEOUT: return "AMS_ERR_DEVICE_TIMEOUT";
        case AMS_ERR_CUDA: return "AMS_ERR_CUDA";
        case AMS_ERR_OOM: return "AMS_ERR_OOM";
    }
    return "AMS_ERR_UNKNOWN";
}

const char* ams_last_error(void) { return g_last_error.c_str(); }

ams_status ams_setup(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* vals,
                     const int32_t* part, int32_t nparts, int32_t m, const ams_options* opt, void* stream,
                     ams_handle* out) {
    NvtxRange nvtx_range("ams_setup");
    g_last_error.clear();
    ams_system_desc d{n, rowptr, colind, vals, part, nparts, m};
    return setup_impl(1, &d, opt, stream, out);
}

ams_status ams_setup_batched(int32_t nsys, const ams_system_desc* systems, const ams_options* opt, void* stream,
                             ams_handle* out) {
    NvtxRange nvtx_range("ams_setup_batched");
    g_last_error.clear();
    return setup_impl(nsys, systems, opt, stream, out);
}

ams_status ams_destroy(ams_handle h) {
    if (h) {
        cudaStreamSynchronize(h->stream);
        delete h;
    }
    return AMS_OK;
}

// Algorithmic bytes of one launch of kernel `which` (each operand read once,
// each output written once) at `ld` right-hand sides.
// Algorithmic bytes of one launch: every operand read once, every output
// written once (FP64 vectors, the stored factor and basis at their storage
// precision).
static double kernel_bytes(ams_handle h, int which, int ld) {
    const double n = (double)h->n_total, nl = n * ld;
    const double tf = (double)h->tf_bytes(), tp = (double)h->tp_bytes();
    switch (which) {
        case AMS_KERNEL_SPMV:    // vals + cols, z (apply precision), p_old in, p, q out, slice pointers;
                                 // x in and out where the direction update applies x += alpha p
            return 12.0 * (double)h->nnz_total + (tf + (defer_x_update(ld) ? 40.0 : 24.0)) * nl +
                   8.0 * (double)h->n_pad / 32;
        case AMS_KERNEL_LOCAL: {
            // factor once (tiles + pivots, or the packed factor), r and q in,
            // z_f out, basis rows, r_c out
            const double fb = h->use_tma ? (double)h->tile_elems * 4.0 + 4.0 * n : (double)h->fac_elems * tf;
            return fb + 16.0 * nl + tf * nl + (double)h->psi_elems * tp + (double)h->Nc * ld * tf;
        }
        case AMS_KERNEL_COARSE:     // forward blocks, r_c in, y out (+ the backward pass when separate)
            return (double)h->R_elems * tf + 2.0 * (double)h->Nc * ld * tf +
                   (fused_backward(ld) ? 0.0 : (double)h->Q_elems * tf + 2.0 * (double)h->Nc * ld * tf);
        case AMS_KERNEL_PROLONG:    // (backward blocks, y) or e_c; z_f, basis; r, q in; r out, z out (apply
                                    // precision); p, x in and x out where this kernel applies x += alpha p
            return (fused_backward(ld) ? (double)h->Q_elems * tf : 0.0) + (double)h->Nc * ld * tf + tf * nl +
                   (double)h->psi_elems * tp + (24.0 + tf + (defer_x_update(ld) ? 0.0 : 24.0)) * nl;
    }
    return 0.0;
}

// Order the handle's internal stream after work already queued on the
// caller's stream (the caller's inputs may be produced there).
static ams_status enter(ams_handle h) {
    debug_bounds(h);
    AMS_CUDA_TRY(cudaEventRecord(h->ev_enter, h->ustream));
    AMS_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev_enter, 0));
    return AMS_OK;
}

static ams_status check_solve_args(ams_handle h, const void* a, const void* b, int32_t nrhs, double rtol) {
    if (!h || !a || !b) {
        set_error("null handle or vector");
        return AMS_ERR_INVALID_ARG;
    }
    if (nrhs < 1 || nrhs > kMaxLd) {
        set_error("nrhs must be in [1, 32]");
        return AMS_ERR_INVALID_ARG;
    }
    if (!(rtol > 0.0) || !std::isfinite(rtol)) {
        set_error("rtol must be positive and finite");
        return AMS_ERR_INVALID_ARG;
    }
    return enter(h);
}

ams_status ams_solve(ams_handle h, const double* f, int32_t nrhs, double rtol, double* u, int32_t* iters,
                     double* relres) {
    NvtxRange nvtx_range("ams_solve");
    g_last_error.clear();
    AMS_TRY(check_solve_args(h, f, u, nrhs, rtol));
    AMS_TRY(ensure_work(h, pow2ceil(nrhs)));
    const double* f_dev = nullptr;
    AMS_TRY(stage_in(h, f, nrhs, h->d_stage_in, &f_dev));
    double* u_dev = h->opt.device_ptrs ? u : h->d_stage_out;
    const double* u0_dev = nullptr;
    if (h->opt.warm_start) {   // u holds the initial guess: keep a copy, u is overwritten
        if (h->nsys != 1) {
            set_error("warm_start needs a single-system handle");
            return AMS_ERR_INVALID_ARG;
        }
        AMS_CUDA_TRY(cudaMemcpyAsync(h->d_stage_aux, u, sizeof(double) * h->n_total * nrhs,
                                     h->opt.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                     h->stream));
        u0_dev = h->d_stage_aux;
    }
    AMS_TRY(pcg_launch(h, f_dev, nrhs, rtol, u_dev, u0_dev));
    if (!h->opt.device_ptrs)   // the solution goes back behind the solve: one wait for both
        AMS_CUDA_TRY(cudaMemcpyAsync(u, u_dev, sizeof(double) * h->n_total * nrhs, cudaMemcpyDeviceToHost,
                                     h->stream));
    AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
    const ams_status st = pcg_finish(h, nrhs, iters, relres);
    return debug_check(h, st);
}

ams_status ams_solve_adjoint(ams_handle h, const double* g, int32_t nrhs, double rtol, const double* u,
                             double* lambda, double* dvals, int32_t* iters) {
    NvtxRange nvtx_range("ams_solve_adjoint");
    g_last_error.clear();
    AMS_TRY(check_solve_args(h, g, lambda, nrhs, rtol));
    if (h->nsys != 1) {
        set_error("adjoint solves need a single-system handle");
        return AMS_ERR_INVALID_ARG;
    }
    if (!u && dvals) {
        set_error("u is required to form dL/dA");
        return AMS_ERR_INVALID_ARG;
    }
    AMS_TRY(ensure_work(h, pow2ceil(nrhs)));
    const double* g_dev = nullptr;
    AMS_TRY(stage_in(h, g, nrhs, h->d_stage_in, &g_dev));
    double* lam_dev = h->opt.device_ptrs ? lambda : h->d_stage_out;
    std::vector<double> rel(nrhs);
    ams_status st = pcg(h, g_dev, nrhs, rtol, lam_dev, iters, rel.data());
    if (st != AMS_OK && st != AMS_ERR_NOT_CONVERGED) return st;
    if (dvals) {
        const double* u_dev = nullptr;
        AMS_TRY(stage_in(h, u, nrhs, h->d_stage_aux, &u_dev));
        double* dv_dev = dvals;
        if (!h->opt.device_ptrs) {
            if (!h->d_stage_dvals) AMS_TRY(h->alloc_t(&h->d_stage_dvals, (size_t)h->nnz_total));
            dv_dev = h->d_stage_dvals;
        }
        launch_sddmm(h->stream, h->d_crowptr, h->d_ccolind, h->n_total, nrhs, lam_dev, u_dev, dv_dev);
        h->launches += 1;
        AMS_CUDA_TRY(cudaGetLastError());
        if (!h->opt.device_ptrs)
            AMS_CUDA_TRY(cudaMemcpyAsync(dvals, dv_dev, sizeof(double) * h->nnz_total, cudaMemcpyDeviceToHost,
                                         h->stream));
    }
    if (!h->opt.device_ptrs)
        AMS_CUDA_TRY(cudaMemcpyAsync(lambda, lam_dev, sizeof(double) * h->n_total * nrhs, cudaMemcpyDeviceToHost,
                                     h->stream));
    AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return debug_check(h, st);
}

ams_status ams_set_matrix_values(ams_handle h, const double* vals) {
    g_last_error.clear();
    if (!h || !vals || h->nsys != 1) {
        set_error("single-system handle and values required");
        return AMS_ERR_INVALID_ARG;
    }
    AMS_TRY(enter(h));
    const double* dv = vals;
    double* tmp = nullptr;
    if (!h->opt.device_ptrs) {
        AMS_TRY(h->alloc_t(&tmp, (size_t)h->nnz_total));
        AMS_CUDA_TRY(cudaMemcpyAsync(tmp, vals, sizeof(double) * h->nnz_total, cudaMemcpyHostToDevice, h->stream));
        dv = tmp;
    }
    launch_scatter_vals(h->stream, dv, h->d_sell_pos, h->nnz_total, h->d_sell_val);
    if (h->d_sell_val32 != nullptr)
        launch_round_to_f32(h->stream, h->d_sell_val, h->sell_elems, h->d_sell_val32);
    h->launches += 1;
    AMS_CUDA_TRY(cudaGetLastError());
    AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (tmp) h->release(tmp);
    return AMS_OK;
}

ams_status ams_get_info(ams_handle h, ams_info* info) {
    if (!h || !info) {
        set_error("null argument");
        return AMS_ERR_INVALID_ARG;
    }
    *info = h->info;
    info->kernel_launches = h->launches;
    return AMS_OK;
}

ams_status ams_get_launch_shape(ams_handle h, int32_t nrhs, int32_t* shape) {
    if (!h || !shape || nrhs < 1 || nrhs > kMaxLd) {
        set_error("null argument or nrhs outside [1, 32]");
        return AMS_ERR_INVALID_ARG;
    }
    const TuneCfg& T = h->tune[pow2ceil(nrhs)];
    shape[0] = T.bps_elem;
    shape[1] = T.bps_sub;
    shape[2] = T.depth;
    shape[3] = T.nr;
    shape[4] = T.l2mode;
    shape[5] = T.l2keep;
    shape[6] = T.done ? 1 : 0;
    return AMS_OK;
}

ams_status ams_set_launch_shape(ams_handle h, int32_t nrhs, const int32_t* shape) {
    if (!h || !shape || nrhs < 1 || nrhs > kMaxLd) {
        set_error("null argument or nrhs outside [1, 32]");
        return AMS_ERR_INVALID_ARG;
    }
    const int ld = pow2ceil(nrhs);
    const int bps_e = shape[0], bps_s = shape[1], depth = shape[2], nr = shape[3];
    const int l2mode = shape[4], l2keep = shape[5];
    if (bps_e < 1 || bps_e > 8 || bps_s < 1 || bps_s > 8) {
        set_error("blocks per SM must be in [1, 8]");
        return AMS_ERR_INVALID_ARG;
    }
    if (depth < 0 || depth > 6) {
        set_error("ring depth must be in [0, 6]");
        return AMS_ERR_INVALID_ARG;
    }
    if (depth > 0) {
        const ResidIn in{nullptr, nullptr, nullptr};
        const size_t smem = h->use_tma ? local_tma_launch_smem(local_tma_args(h, ld, in, false), depth)
                                       : local_solve_smem(h->cmax, ld, h->tf_bytes(), depth);
        if ((h->use_tma && depth < 2) || smem > 200 * 1024) {
            set_error("ring depth too small for the TMA staging or its shared memory above 200 KB");
            return AMS_ERR_INVALID_ARG;
        }
    }
    const bool nr_ok = ld >= 8 ? ((nr == 8 || nr == 16) && nr <= ld && ld / nr <= 4)
                               : ((nr == 2 || nr == 4 || nr == 8) && nr <= ld && ld / nr <= 8);
    if (nr != 0 && !nr_ok) {
        set_error("right-hand sides per warp must be 0, or (below 8 right-hand sides) 2, 4 or 8 with at most "
                  "8 warps per block, or (8 or more) 8 or 16 with at most 4 warps per block");
        return AMS_ERR_INVALID_ARG;
    }
    if (l2mode < 0 || l2mode > 2 || l2keep < 0) {
        set_error("L2 mode must be 0, 1 or 2 and the kept block rows non-negative");
        return AMS_ERR_INVALID_ARG;
    }
    TuneCfg& T = h->tune[ld];
    T.l2mode = l2mode;
    T.l2keep = l2keep;
    T.bps_elem = bps_e;
    T.bps_sub = bps_s;
    T.depth = depth;
    T.nr = nr;
    T.done = true;
    auto g = h->loop_graph.find(ld);   // captured with the previous shapes
    if (g != h->loop_graph.end()) {
        AMS_CUDA_TRY(cudaGraphExecDestroy(g->second));
        h->loop_graph.erase(g);
    }
    return AMS_OK;
}

ams_status ams_get_index_maps(ams_handle h, int64_t* perm, int64_t* sub_ptr) {
    if (!h || h->nsys != 1) {
        set_error("single-system handle required");
        return AMS_ERR_INVALID_ARG;
    }
    const SystemHost& S = h->sys[0];
    if (perm) std::memcpy(perm, S.perm.data(), sizeof(int64_t) * S.n);
    if (sub_ptr) std::memcpy(sub_ptr, S.sub_ptr.data(), sizeof(int64_t) * (S.nparts + 1));
    return AMS_OK;
}

ams_status ams_get_coarse_basis(ams_handle h, int32_t* m_i, double* lambda, double* psi) {
    if (!h) {
        set_error("null handle");
        return AMS_ERR_INVALID_ARG;
    }
    if (m_i)
        for (int s = 0; s < h->N; ++s) m_i[s] = h->h_subs[s].m;
    if (lambda && !h->h_lam.empty()) std::memcpy(lambda, h->h_lam.data(), sizeof(double) * h->h_lam.size());
    if (psi && h->psi_elems > 0) {
        std::vector<double> tmp(h->psi_elems);
        AMS_CUDA_TRY(cudaMemcpy(tmp.data(), h->d_psi64, sizeof(double) * h->psi_elems, cudaMemcpyDeviceToHost));
        int64_t o = 0;
        for (int s = 0; s < h->N; ++s) {
            const SubInfo& S = h->h_subs[s];
            for (int k = 0; k < S.m; ++k)
                for (int i = 0; i < S.n; ++i) psi[o + (int64_t)k * S.n + i] = tmp[S.psi_off + (int64_t)i * S.m + k];
            o += (int64_t)S.n * S.m;
        }
    }
    return AMS_OK;
}

ams_status ams_get_coarse_matrix(ams_handle h, double* A0) {
    if (!h || h->nsys != 1 || !A0) {
        set_error("single-system handle and output required");
        return AMS_ERR_INVALID_ARG;
    }
    const SystemHost& S = h->sys[0];
    if (S.nc > 0 && S.A0_nd.empty()) {
        set_error("coarse matrix not retained (N_c > 4096)");
        return AMS_ERR_INVALID_ARG;
    }
    // paper order: subdomain-major, mode-minor
    std::vector<int64_t> paper_of_nd(S.nc);
    int64_t pos = 0;
    for (int32_t a = 0; a < S.nparts; ++a) {
        const int m = h->h_subs[S.sub0 + a].m;
        for (int k = 0; k < m; ++k) paper_of_nd[S.nd_pos_of_sub[a] + k] = pos + k;
        pos += m;
    }
    for (int64_t i = 0; i < S.nc; ++i)
        for (int64_t j = 0; j < S.nc; ++j) A0[paper_of_nd[i] * S.nc + paper_of_nd[j]] = S.A0_nd[i * S.nc + j];
    return AMS_OK;
}

ams_status ams_get_coarse_factor_inverse(ams_handle h, int64_t* nd_paper, double* Linv) {
    if (!h || h->nsys != 1) {
        set_error("single-system handle required");
        return AMS_ERR_INVALID_ARG;
    }
    const SystemHost& S = h->sys[0];
    if (S.nc > 0 && S.Linv_nd.empty()) {
        set_error("coarse factor inverse not retained (N_c > 4096)");
        return AMS_ERR_INVALID_ARG;
    }
    if (nd_paper) {
        int64_t pos = 0;
        for (int32_t a = 0; a < S.nparts; ++a) {
            const int m = h->h_subs[S.sub0 + a].m;
            for (int k = 0; k < m; ++k) nd_paper[S.nd_pos_of_sub[a] + k] = pos + k;
            pos += m;
        }
    }
    if (Linv)
        for (int64_t i = 0; i < S.nc; ++i)
            for (int64_t j = 0; j < S.nc; ++j) Linv[i * S.nc + j] = S.Linv_nd[i + j * S.nc];
    return AMS_OK;
}

ams_status ams_debug_selftest(int32_t* site) {
    g_last_error.clear();
    if (!site) {
        set_error("site pointer required");
        return AMS_ERR_INVALID_ARG;
    }
    launch_debug_selftest(0);
    AMS_CUDA_TRY(cudaGetLastError());
    AMS_CUDA_TRY(cudaDeviceSynchronize());
    *site = debug_take_site_solve();
    return AMS_OK;
}

ams_status ams_apply_preconditioner(ams_handle h, const double* r, int32_t nrhs, double* z) {
    NvtxRange nvtx_range("ams_apply_preconditioner");
    g_last_error.clear();
    AMS_TRY(check_solve_args(h, r, z, nrhs, 1.0));
    if (h->nsys != 1) {
        set_error("single-system handle required");
        return AMS_ERR_INVALID_ARG;
    }
    const int ld = pow2ceil(nrhs);
    AMS_TRY(ensure_work(h, ld));
    RedCache *rc = nullptr, *rcs = nullptr;
    AMS_TRY(get_red(h, ld, &rc, &rcs));
    LaunchCtx L = make_ctx(h, *rc, *rcs);
    const double* r_dev = nullptr;
    AMS_TRY(stage_in(h, r, nrhs, h->d_stage_in, &r_dev));
    launch_permute_in(h->stream, r_dev, h->n_total, nrhs, ld, h->d_int_row, h->d_r, nullptr);
    h->launches += 2;
    AMS_TRY(clear_device_status(h));
    AMS_TRY(apply_precond(h, L, 0, nullptr));
    double* z_dev = h->opt.device_ptrs ? z : h->d_stage_out;
    if (h->prec == AMS_PREC_FP64)
        launch_permute_out(h->stream, h->d_z, h->n_total, nrhs, ld, h->d_int_row, z_dev);
    else   // z is stored in the apply precision
        launch_permute_out_f32(h->stream, reinterpret_cast<const float*>(h->d_z), h->n_total, nrhs, ld,
                               h->d_int_row, z_dev);
    AMS_CUDA_TRY(cudaGetLastError());
    if (!h->opt.device_ptrs)
        AMS_CUDA_TRY(cudaMemcpyAsync(z, z_dev, sizeof(double) * h->n_total * nrhs, cudaMemcpyDeviceToHost, h->stream));
    AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return debug_check(h, device_status(h));
}

ams_status ams_spmv(ams_handle h, const double* x, int32_t nrhs, double* y) {
    NvtxRange nvtx_range("ams_spmv");
    g_last_error.clear();
    AMS_TRY(check_solve_args(h, x, y, nrhs, 1.0));
    if (h->nsys != 1) {
        set_error("single-system handle required");
        return AMS_ERR_INVALID_ARG;
    }
    const int ld = pow2ceil(nrhs);
    AMS_TRY(ensure_work(h, ld));
    RedCache *rc = nullptr, *rcs = nullptr;
    AMS_TRY(get_red(h, ld, &rc, &rcs));
    LaunchCtx L = make_ctx(h, *rc, *rcs);
    L.st = nullptr;
    const double* x_dev = nullptr;
    AMS_TRY(stage_in(h, x, nrhs, h->d_stage_in, &x_dev));
    launch_permute_in(h->stream, x_dev, h->n_total, nrhs, ld, h->d_int_row, h->d_p, nullptr);
    launch_spmv_dot(L, h->d_p, h->d_q, 0);
    h->launches += 3;
    double* y_dev = h->opt.device_ptrs ? y : h->d_stage_out;
    launch_permute_out(h->stream, h->d_q, h->n_total, nrhs, ld, h->d_int_row, y_dev);
    AMS_CUDA_TRY(cudaGetLastError());
    if (!h->opt.device_ptrs)
        AMS_CUDA_TRY(cudaMemcpyAsync(y, y_dev, sizeof(double) * h->n_total * nrhs, cudaMemcpyDeviceToHost, h->stream));
    AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return debug_check(h, AMS_OK);
}

ams_status ams_time_kernel(ams_handle h, int32_t which, int32_t reps, double* avg_ms, double* bytes) {
    NvtxRange nvtx_range("ams_time_kernel");
    g_last_error.clear();
    if (!h || reps <= 0 || which < 0 || which >= AMS_NUM_KERNELS || h->ld_last == 0) {
        set_error("invalid arguments (a solve must run first)");
        return AMS_ERR_INVALID_ARG;
    }
    AMS_TRY(enter(h));
    const int ld = h->ld_last;
    RedCache *rc = nullptr, *rcs = nullptr;
    AMS_TRY(get_red(h, ld, &rc, &rcs));
    LaunchCtx L = make_ctx(h, *rc, *rcs);
    // keep every (system, rhs) active and never converge while timing
    {
        std::vector<CgScalars> sc((size_t)h->nsys * ld);
        AMS_CUDA_TRY(cudaMemcpy(sc.data(), h->d_sc, sizeof(CgScalars) * sc.size(), cudaMemcpyDeviceToHost));
        for (auto& c : sc) {
            c.active = 1;
            if (!(c.pq > 0)) c.pq = 1.0;
            if (!(c.rho > 0)) c.rho = 1.0;
            c.fnorm2 = 1.0;
        }
        AMS_CUDA_TRY(cudaMemcpy(h->d_sc, sc.data(), sizeof(CgScalars) * sc.size(), cudaMemcpyHostToDevice));
        SolveState st{};
        st.maxit = 0x7fffffff;
        st.rtol2 = 0.0;
        AMS_CUDA_TRY(cudaMemcpy(h->d_st, &st, sizeof(st), cudaMemcpyHostToDevice));
    }
    const double b = kernel_bytes(h, which, ld);
    // Timed launches keep their solve-state argument (so they run the code
    // path of a solve) but the state above never reports convergence.  The
    // SpMV reads p and writes p2, the prolongation updates x and r in place.
    auto launch = [&]() -> ams_status {
        switch (which) {
            case AMS_KERNEL_SPMV: launch_direction_spmv(h, L, h->d_p, h->d_p2); break;
            case AMS_KERNEL_LOCAL:
                AMS_TRY(launch_local(h, ld, ResidIn{h->d_r, h->d_q, h->d_sc}, true));
                break;
            case AMS_KERNEL_COARSE: launch_coarse(h, ld, true); break;
            case AMS_KERNEL_PROLONG: launch_prolong_update(L, h->prec, prolong_args(h, 2, h->d_p2, ld)); break;
        }
        return AMS_OK;
    };
    AMS_TRY(launch());
    cudaEvent_t e0, e1;
    AMS_CUDA_TRY(cudaEventCreate(&e0));
    AMS_CUDA_TRY(cudaEventCreate(&e1));
    AMS_CUDA_TRY(cudaStreamSynchronize(h->stream));
    AMS_CUDA_TRY(cudaEventRecord(e0, h->stream));
    for (int k = 0; k < reps; ++k) AMS_TRY(launch());
    AMS_CUDA_TRY(cudaEventRecord(e1, h->stream));
    AMS_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    AMS_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    AMS_CUDA_TRY(cudaGetLastError());
    if (avg_ms) *avg_ms = ms / reps;
    if (bytes) *bytes = b;
    return AMS_OK;
}

ams_status ams_profile_solve(ams_handle h, const double* f, int32_t nrhs, double rtol, double* ms,
                             double* bytes, int64_t* count) {
    NvtxRange nvtx_range("ams_profile_solve");
    g_last_error.clear();
    AMS_TRY(check_solve_args(h, f, f, nrhs, rtol));
    AMS_TRY(ensure_work(h, pow2ceil(nrhs)));
    KernelProfile P;
    for (auto& e : P.ev) AMS_CUDA_TRY(cudaEventCreate(&e));
    const double* f_dev = nullptr;
    ams_status st = stage_in(h, f, nrhs, h->d_stage_in, &f_dev);
    if (st == AMS_OK) {
        h->prof = &P;
        std::vector<int32_t> its(h->nsys * nrhs);
        st = pcg(h, f_dev, nrhs, rtol, h->d_stage_out, its.data(), nullptr);
        h->prof = nullptr;
        if (st == AMS_OK) st = prof_flush(h);
    }
    for (auto& e : P.ev) cudaEventDestroy(e);
    if (st != AMS_OK && st != AMS_ERR_NOT_CONVERGED) return st;
    const int ld = pow2ceil(nrhs);
    for (int k = 0; k < AMS_NUM_KERNELS; ++k) {
        if (ms) ms[k] = P.ms[k];
        if (count) count[k] = P.count[k];
        if (bytes) bytes[k] = kernel_bytes(h, k, ld);
    }
    return st;
}

}  // extern "C"
