// Coarse solve of the AMS preconditioner (a5): y = L_c^{-1} r_c and
// e_c = L_c^{-T} y as products of the nested-dissection blocks of L_c^{-1}
// (A_0 = L_c L_c^T, Section 3.1) with gathered inputs.  FP64 items
// (k_coarse_gemm), few right-hand sides (k_coarse_rows) and, in the
// reduced-precision apply with 8-32 right-hand sides, TF32-split tensor-core
// MMAs (k_coarse_mma).
#include <cstdint>
#include <cstdio>
#include <type_traits>

#include "ams_internal.h"
#include "kernels.cuh"
#include "launch.h"
#include "mma_tf32.cuh"

namespace ams {

// ===========================================================================
// a5: coarse solve by blocks of L_c^{-1} (nested-dissection layout).
// Each item multiplies a <=32-row tile of one node matrix by a gathered
// chunk of the input; several chunks of one tile are summed in chunk order
// by the last item to finish (deterministic split-K).
// ===========================================================================
template <typename TF, int LD>
__global__ void __launch_bounds__(256)
k_coarse_gemm(const CoarseItem* __restrict__ items, const TF* __restrict__ mat,
              const int32_t* __restrict__ rng, const int32_t* __restrict__ gat, const TF* __restrict__ in,
              TF* __restrict__ out, TF* __restrict__ partial, int32_t* __restrict__ cnt, const SolveState* st) {
    // Many right-hand sides (LD >= 8): thread (h = t % LD, row group t / LD)
    // accumulates RPT consecutive rows of the 32-row tile for right-hand side
    // h.  Per stage of KC columns the tile (transposed, so one aligned load
    // gives a thread its RPT rows at one column) and the gathered input go
    // through shared memory; the next stage's global loads are issued into
    // registers before the current stage is computed.
    pdl_wait();
    if (st != nullptr && st->done) return;
    pdl_trigger();
    using A = typename Acc<TF>::type;
    using V4 = typename std::conditional<sizeof(TF) == 4, float4, double4>::type;
    static_assert(LD >= 8 && LD <= 32, "k_coarse_gemm serves 8 to 32 right-hand sides");
    constexpr int KC = 64;                                   // columns per stage
    constexpr int OUT = 32 * LD;                             // outputs of a tile
    constexpr int NRG = 256 / LD;                            // row groups
    constexpr int RPT = 32 / NRG;                            // rows per thread (1, 2 or 4)
    constexpr int TP = 32 + 4;                               // padded transposed row
    constexpr int MV = 32 * KC / 4 / 256;                    // 4-column tile pieces per thread (2)
    constexpr int XV = KC * LD / 256;                        // input values per thread
    __shared__ __align__(32) TF sMT[KC][TP];
    __shared__ TF sX[KC][LD];
    __shared__ int s_last;
    const CoarseItem it = items[blockIdx.x];
    const int t = threadIdx.x;
    const int h = t % LD, r0 = (t / LD) * RPT;
    const TF* M0 = mat + it.moff + (int64_t)it.row_in_node * it.ldm;
    const int g0 = (it.gat_off < 0) ? rng[2 * it.rng_off] : 0;
    const int32_t* G = gat + (it.gat_off < 0 ? 0 : it.gat_off);
    V4 mreg[MV];
    TF xreg[XV];
    auto load_stage = [&](int kb) {
        const int kn = min(KC, it.k1 - kb);
#pragma unroll
        for (int u = 0; u < MV; ++u) {
            const int i = t + 256 * u;
            const int r = i / (KC / 4), c4 = i % (KC / 4);
            mreg[u] = V4{};
            if (r < it.nrows && 4 * c4 < kn)
                mreg[u] = *reinterpret_cast<const V4*>(M0 + (int64_t)r * it.ldm + kb + 4 * c4);
        }
#pragma unroll
        for (int u = 0; u < XV; ++u) {
            const int i = t + 256 * u;
            const int kk = i / LD, hh = i % LD;
            xreg[u] = TF(0);
            if (kk < kn) {
                const int k = kb + kk;
                const int g = (it.gat_off < 0) ? g0 + k : __ldg(G + k);
                if (AMS_COARSE_OK(g, 3)) xreg[u] = in[(int64_t)g * LD + hh];
            }
        }
    };
    auto store_stage = [&]() {
#pragma unroll
        for (int u = 0; u < MV; ++u) {
            const int i = t + 256 * u;
            const int r = i / (KC / 4), c4 = i % (KC / 4);
            sMT[4 * c4 + 0][r] = mreg[u].x;
            sMT[4 * c4 + 1][r] = mreg[u].y;
            sMT[4 * c4 + 2][r] = mreg[u].z;
            sMT[4 * c4 + 3][r] = mreg[u].w;
        }
#pragma unroll
        for (int u = 0; u < XV; ++u) {
            const int i = t + 256 * u;
            sX[i / LD][i % LD] = xreg[u];
        }
    };
    A acc[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) acc[i] = A(0);
    load_stage(it.k0);
    for (int kb = it.k0; kb < it.k1; kb += KC) {
        __syncthreads();                     // the previous stage is no longer read
        store_stage();
        __syncthreads();
        if (kb + KC < it.k1) load_stage(kb + KC);
#pragma unroll 8
        for (int kk = 0; kk < KC; ++kk) {
            const A x = (A)sX[kk][h];
            if (RPT == 4) {
                const V4 m = *reinterpret_cast<const V4*>(&sMT[kk][r0]);
                acc[0] += (A)m.x * x;
                acc[RPT > 1 ? 1 : 0] += (A)m.y * x;
                acc[RPT > 2 ? 2 : 0] += (A)m.z * x;
                acc[RPT > 3 ? 3 : 0] += (A)m.w * x;
            } else {
#pragma unroll
                for (int i = 0; i < RPT; ++i) acc[i] += (A)sMT[kk][r0 + i] * x;
            }
        }
    }
    if (it.nchunks == 1) {
#pragma unroll
        for (int i = 0; i < RPT; ++i)
            if (r0 + i < it.nrows) out[(int64_t)(it.out0 + r0 + i) * LD + h] = (TF)acc[i];
        return;
    }
    TF* P = partial + (int64_t)(it.slot0 + it.chunk) * OUT;
#pragma unroll
    for (int i = 0; i < RPT; ++i) P[(r0 + i) * LD + h] = (TF)acc[i];

    __syncthreads();
    if (t == 0) {
        __threadfence();
        s_last = (atomicAdd(cnt + it.tile_id, 1) == it.nchunks - 1);
        if (s_last) __threadfence();
    }
    __syncthreads();
    if (!s_last) return;
    for (int o = t; o < OUT; o += 256) {
        A s = A(0);
        for (int ch = 0; ch < it.nchunks; ++ch) s += (A)__ldcg(partial + (int64_t)(it.slot0 + ch) * OUT + o);
        const int rr = o / LD, hh = o % LD;
        if (rr < it.nrows) out[(int64_t)(it.out0 + rr) * LD + hh] = (TF)s;
    }
    if (t == 0) cnt[it.tile_id] = 0;
}

// Many right-hand sides (LD >= 8) in the reduced-precision apply: the same
// items as k_coarse_gemm, with the 32-row tile times the gathered input
// computed by warp-level tensor-core MMAs (m16n8k8, TF32 head/tail split
// of both operands, FP32 accumulation: FP32 accuracy).  Every warp computes
// the whole 32 x LD output tile over its own k-steps of each stage (warp w
// takes k-steps w, w + NW, ..; NW = LD/4 warps), so each staged element is
// split into its TF32 head and tail exactly once; the warps' partial tiles
// are summed in warp order through shared memory at the end.  Stages of 64 columns of the tile (row-major, rows padded to 68 floats so
// that the A-fragment loads are conflict-free) and of the gathered input
// (rows padded to 8 mod 32 words for the B fragments) stream through a ring
// of kCoarseStages shared-memory slots with 16-byte cp.async copies (zero
// fill past the tile's rows and columns), so that two stages are in flight
// while one is multiplied; the gather indices of a stage are read one stage
// before its copies are issued.  Split-K chunks reduce as in k_coarse_gemm.
constexpr int kCoarseStages = 3;
template <int LD>
constexpr size_t coarse_mma_smem() {
    return (size_t)kCoarseStages * (32 * 68 + 64 * (LD >= 16 ? LD + 8 : 24)) * sizeof(float);
}
template <int LD>
__global__ void __launch_bounds__(LD * 8, 4)
k_coarse_mma(const CoarseItem* __restrict__ items, const float* __restrict__ mat, const int32_t* __restrict__ rng,
             const int32_t* __restrict__ gat, const float* __restrict__ in, float* __restrict__ out,
             float* __restrict__ partial, int32_t* __restrict__ cnt, const SolveState* st) {
    pdl_wait();
    if (st != nullptr && st->done) return;
    pdl_trigger();
    static_assert(LD == 8 || LD == 16 || LD == 32, "k_coarse_mma serves 8, 16 or 32 right-hand sides");
    constexpr int NT = LD * 8;                               // threads
    constexpr int NW = NT / 32;                              // warps (k-step groups)
    constexpr int NFR = LD / 8;                              // 8-column fragments per warp
    constexpr int KC = 64;                                   // columns per stage
    constexpr int NS = kCoarseStages;
    constexpr int SA = KC + 4;
    constexpr int SB = LD >= 16 ? LD + 8 : 24;
    constexpr int STAGE = 32 * SA + KC * SB;                 // floats per ring slot
    constexpr int OUT = 32 * LD;
    constexpr int MV = 32 * KC / 4 / NT;                     // 16-byte tile pieces per thread and stage
    constexpr int XV = KC * LD / 4 / NT;                     // 16-byte input pieces per thread and stage
    extern __shared__ __align__(16) float s_ring[];
    __shared__ int s_last;
    const CoarseItem it = items[blockIdx.x];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int g = lane >> 2, tq = lane & 3;
    const float* M0 = mat + it.moff + (int64_t)it.row_in_node * it.ldm;
    const bool contiguous = it.gat_off < 0;
    const int g0 = contiguous ? rng[2 * it.rng_off] : 0;
    const int32_t* G = gat + (contiguous ? 0 : it.gat_off);
    const int nst = (it.k1 - it.k0 + KC - 1) / KC;
    int gi[XV];                                              // input rows of the next stage to issue (-1: none)
    auto load_idx = [&](int s) {
        const int kb = it.k0 + s * KC;
#pragma unroll
        for (int u = 0; u < XV; ++u) {
            const int k = kb + (t + NT * u) / (LD / 4);
            gi[u] = (s < nst && k < it.k1) ? (contiguous ? g0 + k : __ldg(G + k)) : -1;
            if (gi[u] >= 0 && !AMS_COARSE_OK(gi[u], 3)) gi[u] = -1;
        }
    };
    auto issue = [&](int s) {
        float* sA = s_ring + (s % NS) * STAGE;
        float* sB = sA + 32 * SA;
        const int kb = it.k0 + s * KC, kn = min(KC, it.k1 - kb);
#pragma unroll
        for (int u = 0; u < MV; ++u) {
            const int i = t + NT * u;
            const int r = i / (KC / 4), c4 = i % (KC / 4);
            const bool ok = r < it.nrows && 4 * c4 < kn;   // rows are zero-padded to ldm, a multiple of 4
            cp_async16_zfill(sA + r * SA + 4 * c4, ok ? M0 + (int64_t)r * it.ldm + kb + 4 * c4 : M0, ok);
        }
#pragma unroll
        for (int u = 0; u < XV; ++u) {
            const int i = t + NT * u;
            const int kk = i / (LD / 4), c4 = i % (LD / 4);
            const bool ok = gi[u] >= 0;
            cp_async16_zfill(sB + kk * SB + 4 * c4, ok ? in + (int64_t)gi[u] * LD + 4 * c4 : in, ok);
        }
    };
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) {
        if (s < nst) {
            load_idx(s);
            issue(s);
        }
        cp_async_commit();
    }
    load_idx(NS - 1);
    float acc[2][NFR][4];                                    // [row fragment][column fragment]
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < NFR; ++b)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[a][b][i] = 0.f;
    for (int s = 0; s < nst; ++s) {
        cp_async_wait_n(NS - 2);             // stage s has landed for this thread ...
        __syncthreads();                     // ... and for all; slot (s - 1) % NS is free
        if (s + NS - 1 < nst) issue(s + NS - 1);
        cp_async_commit();
        load_idx(s + NS);
        const float* sA = s_ring + (s % NS) * STAGE;
        const float* sB = sA + 32 * SA;
#pragma unroll
        for (int ks = w; ks < KC / 8; ks += NW) {
            const int k0 = 8 * ks + tq;
            uint32_t ah[2][4], al[2][4];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int r0 = 16 * a + g;
                split_tf32(sA[r0 * SA + k0], ah[a][0], al[a][0]);
                split_tf32(sA[(r0 + 8) * SA + k0], ah[a][1], al[a][1]);
                split_tf32(sA[r0 * SA + k0 + 4], ah[a][2], al[a][2]);
                split_tf32(sA[(r0 + 8) * SA + k0 + 4], ah[a][3], al[a][3]);
            }
#pragma unroll
            for (int b = 0; b < NFR; ++b) {
                uint32_t b0h, b0l, b1h, b1l;
                split_tf32(sB[k0 * SB + 8 * b + g], b0h, b0l);
                split_tf32(sB[(k0 + 4) * SB + 8 * b + g], b1h, b1l);
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    mma_tf32(acc[a][b], al[a], b0h, b1h);
                    mma_tf32(acc[a][b], ah[a], b0l, b1l);
                    mma_tf32(acc[a][b], ah[a], b0h, b1h);
                }
            }
        }
    }
    cp_async_wait_all();
    // sum the warps' partial tiles in warp order (the ring is free now);
    // rows padded to LD + 8 floats: the 8-byte stores of a warp fill the
    // 32 banks twice, the minimum for 256 bytes
    constexpr int SR = LD + 8;
    __syncthreads();
    float* red = s_ring;                                     // NW x 32 x SR
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < NFR; ++b)
#pragma unroll
            for (int h = 0; h < 2; ++h)
                *reinterpret_cast<float2*>(red + (w * 32 + 16 * a + g + 8 * h) * SR + 8 * b + 2 * tq) =
                    make_float2(acc[a][b][2 * h], acc[a][b][2 * h + 1]);
    __syncthreads();
    float res[OUT / NT];                                     // outputs o = t + NT u
#pragma unroll
    for (int u = 0; u < OUT / NT; ++u) {
        const int o = t + NT * u, ro = (o / LD) * SR + o % LD;
        float v = red[ro];
#pragma unroll
        for (int ww = 1; ww < NW; ++ww) v += red[ww * 32 * SR + ro];
        res[u] = v;
    }
    if (it.nchunks == 1) {
#pragma unroll
        for (int u = 0; u < OUT / NT; ++u) {
            const int o = t + NT * u, rr = o / LD;
            if (rr < it.nrows) out[(int64_t)(it.out0 + rr) * LD + o % LD] = res[u];
        }
        return;
    }
    float* P = partial + (int64_t)(it.slot0 + it.chunk) * OUT;
#pragma unroll
    for (int u = 0; u < OUT / NT; ++u) P[t + NT * u] = res[u];
    __syncthreads();
    if (t == 0) {
        __threadfence();
        s_last = (atomicAdd(cnt + it.tile_id, 1) == it.nchunks - 1);
        if (s_last) __threadfence();
    }
    __syncthreads();
    if (!s_last) return;
    for (int o = t; o < OUT; o += NT) {
        float sum = 0.f;
        for (int ch = 0; ch < it.nchunks; ++ch) sum += __ldcg(partial + (int64_t)(it.slot0 + ch) * OUT + o);
        const int rr = o / LD, hh = o % LD;
        if (rr < it.nrows) out[(int64_t)(it.out0 + rr) * LD + hh] = sum;
    }
    if (t == 0) cnt[it.tile_id] = 0;
}

// Few right-hand sides (LD <= 4): each warp streams whole rows of the node
// matrix with coalesced 16-byte loads (lane j covers columns 4j..4j+3 of
// every 128-column group) against the gathered input chunk held in shared
// memory; no per-stage barriers.  Node-matrix rows are padded with zeros to
// a multiple of 4 columns, so every row starts 16-byte aligned.
template <typename TF, int LD>
__global__ void __launch_bounds__(256)
k_coarse_rows(const CoarseItem* __restrict__ items, const TF* __restrict__ mat,
              const int32_t* __restrict__ rng, const TF* __restrict__ in, TF* __restrict__ out,
              TF* __restrict__ partial, int32_t* __restrict__ cnt, const SolveState* st) {
    using A = typename Acc<TF>::type;
    using V4 = typename std::conditional<sizeof(TF) == 4, float4, double4>::type;
    constexpr int OUT = 32 * LD;
    constexpr int MAXR = 64;                  // gather ranges staged in shared memory
    __shared__ __align__(16) TF sx[(kCoarseChunk + 4) * LD];
    __shared__ A sres[OUT];
    __shared__ int srng[2 * MAXR];
    __shared__ int s_last;
    const CoarseItem it = items[blockIdx.x];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int kn = it.k1 - it.k0;
    const int kn4 = (kn + 3) & ~3;
    const int nr = min(it.nrng, MAXR);
    const TF* M0 = mat + it.moff + (int64_t)it.row_in_node * it.ldm + it.k0;
    const bool rv[4] = {warp < it.nrows, warp + 8 < it.nrows, warp + 16 < it.nrows, warp + 24 < it.nrows};
    // warp w owns rows w, w+8, w+16, w+24 of the tile; lane takes 4 columns
    // per step.  The first two steps of the (setup-data) tile are loaded
    // before the input gather so both memory trips overlap.
    auto load_cols = [&](int c4, V4 (&mv)[4]) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (rv[i] && 4 * c4 < kn4) mv[i] = *reinterpret_cast<const V4*>(M0 + (int64_t)(warp + 8 * i) * it.ldm + 4 * c4);
    };
    V4 pre0[4], pre1[4];
    load_cols(lane, pre0);
    load_cols(lane + 32, pre1);
    for (int i = t; i < 2 * nr; i += 256) srng[i] = rng[2 * it.rng_off + i];
    pdl_wait();
    if (st != nullptr && st->done) return;
    pdl_trigger();
    __syncthreads();
    for (int kk = t; kk < kn4; kk += 256) {
        TF v[LD];
#pragma unroll
        for (int h = 0; h < LD; ++h) v[h] = TF(0);
        if (kk < kn) {
            int k = it.k0 + kk, g = 0;
            for (int j = 0; j < it.nrng; ++j) {
                const int s0 = j < MAXR ? srng[2 * j] : rng[2 * (it.rng_off + j)];
                const int len = j < MAXR ? srng[2 * j + 1] : rng[2 * (it.rng_off + j) + 1];
                if (k < len) { g = s0 + k; break; }
                k -= len;
            }
            if (AMS_COARSE_OK(g, 3))
#pragma unroll
                for (int h = 0; h < LD; ++h) v[h] = in[(int64_t)g * LD + h];
        }
#pragma unroll
        for (int h = 0; h < LD; ++h) sx[kk * LD + h] = v[h];
    }
    __syncthreads();
    A acc[4][LD];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int h = 0; h < LD; ++h) acc[i][h] = A(0);
    auto step = [&](int c4, const V4 (&mv)[4]) {
        if (4 * c4 >= kn4) return;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            A xv[LD];
#pragma unroll
            for (int h = 0; h < LD; ++h) xv[h] = (A)sx[(4 * c4 + e) * LD + h];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (rv[i]) {
                    const A m = (A)(e == 0 ? mv[i].x : e == 1 ? mv[i].y : e == 2 ? mv[i].z : mv[i].w);
#pragma unroll
                    for (int h = 0; h < LD; ++h) acc[i][h] += m * xv[h];
                }
            }
        }
    };
    step(lane, pre0);
    step(lane + 32, pre1);
#pragma unroll 2
    for (int c4 = lane + 64; 4 * c4 < kn4; c4 += 32) {
        V4 mv[4];
        load_cols(c4, mv);
        step(c4, mv);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int h = 0; h < LD; ++h) {
            A v = acc[i][h];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) sres[(warp + 8 * i) * LD + h] = v;
        }
    __syncthreads();
    if (it.nchunks == 1) {
        for (int o = t; o < OUT; o += 256) {
            const int r = o / LD;
            if (r < it.nrows) out[(int64_t)(it.out0 + r) * LD + (o % LD)] = (TF)sres[o];
        }
        return;
    }
    TF* P = partial + (int64_t)(it.slot0 + it.chunk) * OUT;
    for (int o = t; o < OUT; o += 256) P[o] = (TF)sres[o];
    __syncthreads();
    if (t == 0) {
        __threadfence();
        s_last = (atomicAdd(cnt + it.tile_id, 1) == it.nchunks - 1);
        if (s_last) __threadfence();
    }
    __syncthreads();
    if (!s_last) return;
    for (int o = t; o < OUT; o += 256) {
        A v = A(0);
        for (int ch = 0; ch < it.nchunks; ++ch) v += (A)__ldcg(partial + (int64_t)(it.slot0 + ch) * OUT + o);
        const int r = o / LD;
        if (r < it.nrows) out[(int64_t)(it.out0 + r) * LD + (o % LD)] = (TF)v;
    }
    if (t == 0) cnt[it.tile_id] = 0;
}

AMS_DEBUG_TU_HOOKS(coarse)

// ---------------------------------------------------------------------------
// launcher
// ---------------------------------------------------------------------------
template <typename TF, int LD>
static void coarse_ld(const CoarseLaunch& c, const void* in, void* out) {
    if (c.nitems == 0) return;
    if (LD <= 4)
        launch_kernel(c.pdl, k_coarse_rows<TF, (LD <= 4 ? LD : 4)>, dim3(c.nitems), dim3(256), 0, c.stream, c.items,
                      (const TF*)c.mat, c.rng, (const TF*)in, (TF*)out, (TF*)c.partial, c.cnt, c.st);
    else
        if constexpr (sizeof(TF) == 4)   // reduced-precision apply: tile products on the tensor cores
        {
            constexpr int L8 = LD >= 8 ? LD : 8;
            constexpr size_t smem = coarse_mma_smem<L8>();
            static bool smem_set = false;   // per template instance
            if (!smem_set) {
                if (cudaFuncSetAttribute(k_coarse_mma<L8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem) != cudaSuccess)
                    return;   // the error stays the last runtime error, which the caller checks
                smem_set = true;
            }
            launch_kernel(c.pdl, k_coarse_mma<L8>, dim3(c.nitems), dim3(L8 * 8), smem, c.stream, c.items,
                          (const float*)c.mat, c.rng, c.gat, (const float*)in, (float*)out, (float*)c.partial, c.cnt,
                          c.st);
        }
        else
            launch_kernel(c.pdl, k_coarse_gemm<TF, (LD >= 8 ? LD : 8)>, dim3(c.nitems), dim3(256), 0, c.stream,
                          c.items, (const TF*)c.mat, c.rng, c.gat, (const TF*)in, (TF*)out, (TF*)c.partial, c.cnt,
                          c.st);
}
template <typename TF>
static void coarse_tf(const CoarseLaunch& c, int ld, const void* in, void* out) {
    switch (ld) {
        case 1: coarse_ld<TF, 1>(c, in, out); break;
        case 2: coarse_ld<TF, 2>(c, in, out); break;
        case 4: coarse_ld<TF, 4>(c, in, out); break;
        case 8: coarse_ld<TF, 8>(c, in, out); break;
        case 16: coarse_ld<TF, 16>(c, in, out); break;
        default: coarse_ld<TF, 32>(c, in, out); break;
    }
}
void launch_coarse_gemm(const CoarseLaunch& c, int prec, int ld, const void* in, void* out) {
    if (prec == AMS_PREC_FP64) coarse_tf<double>(c, ld, in, out);
    else coarse_tf<float>(c, ld, in, out);
}

}  // namespace ams
