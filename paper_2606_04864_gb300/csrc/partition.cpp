// Built-in graph partitioner for matrix-only input.  The method takes a
// non-overlapping partition of the dofs into subdomains as given
// (Section 3.1; the paper's experiments obtain it from METIS, Section 5).
// This file supplies one from the matrix pattern alone: multilevel
// recursive bisection.  Each bisection coarsens the graph by heavy-edge
// matching, splits the coarsest graph by region growing from several seeds,
// and refines the split on every level on the way back with
// Fiduccia-Mattheyses passes under a balance constraint.  Host code only,
// large splits on threads of their own; the result depends on the seed
// alone (integer arithmetic, total orders, per-split generators).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "ams_internal.h"

namespace ams {
namespace {

struct Graph {
    int32_t n = 0;
    std::vector<int64_t> xadj;   // n + 1
    std::vector<int32_t> adj;    // neighbours, no self loops, no duplicates
    std::vector<int64_t> ew;     // edge weights (symmetric)
    std::vector<int64_t> vw;     // vertex weights
    int64_t total = 0;           // sum of vertex weights
};

// splitmix64 (Steele, Lea, Flood 2014)
struct Rng {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    // in [0, m): the high 32 bits scaled by m (multiply-shift, no division)
    uint32_t below(uint32_t m) { return (uint32_t)(((next() >> 32) * (uint64_t)m) >> 32); }
};

std::vector<int32_t> random_order(int32_t n, Rng& rng) {
    std::vector<int32_t> p(n);
    for (int32_t i = 0; i < n; ++i) p[i] = i;
    for (int32_t i = n - 1; i > 0; --i) std::swap(p[i], p[rng.below((uint32_t)i + 1)]);
    return p;
}

// Random order inside consecutive blocks of 2048 vertices, blocks in
// natural order: random enough for matching, and a vertex's neighbours
// (close in index for the meshes this partitions) stay in cache.
std::vector<int32_t> blocked_random_order(int32_t n, Rng& rng) {
    constexpr int32_t kBlock = 2048;
    std::vector<int32_t> p(n);
    for (int32_t i = 0; i < n; ++i) p[i] = i;
    for (int32_t b = 0; b < n; b += kBlock) {
        const int32_t len = std::min(kBlock, n - b);
        for (int32_t i = len - 1; i > 0; --i) std::swap(p[b + i], p[b + rng.below((uint32_t)i + 1)]);
    }
    return p;
}

// Heavy-edge matching: vertices in random order, each unmatched vertex is
// paired with the unmatched neighbour across its heaviest edge, as long as
// the pair weighs at most maxvw; cmap receives the coarse vertex of each
// fine vertex.
Graph coarsen(const Graph& g, std::vector<int32_t>& cmap, int64_t maxvw, Rng& rng) {
    const int32_t n = g.n;
    const std::vector<int32_t> order = blocked_random_order(n, rng);
    std::vector<int32_t> mate(n, -1);
    cmap.assign(n, -1);
    int32_t nc = 0;
    for (int32_t t = 0; t < n; ++t) {
        const int32_t v = order[t];
        if (mate[v] >= 0) continue;
        int32_t best = -1;
        int64_t bw = 0;
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
            const int32_t u = g.adj[e];
            if (mate[u] >= 0 || g.vw[v] + g.vw[u] > maxvw) continue;
            if (best < 0 || g.ew[e] > bw) {
                best = u;
                bw = g.ew[e];
            }
        }
        if (best < 0) {
            mate[v] = v;
            cmap[v] = nc++;
        } else {
            mate[v] = best;
            mate[best] = v;
            cmap[v] = cmap[best] = nc++;
        }
    }
    Graph c;
    c.n = nc;
    c.total = g.total;
    c.vw.assign(nc, 0);
    c.xadj.assign((size_t)nc + 1, 0);
    std::vector<int32_t> first(nc, -1), second(nc, -1);
    for (int32_t v = 0; v < n; ++v) {
        const int32_t cv = cmap[v];
        (first[cv] < 0 ? first[cv] : second[cv]) = v;
        c.vw[cv] += g.vw[v];
    }
    c.adj.reserve(g.adj.size());
    c.ew.reserve(g.adj.size());
    std::vector<int32_t> mark(nc, -1);
    std::vector<int64_t> slot(nc, 0);
    for (int32_t cv = 0; cv < nc; ++cv) {
        for (int32_t v : {first[cv], second[cv]}) {
            if (v < 0) continue;
            for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
                const int32_t cu = cmap[g.adj[e]];
                if (cu == cv) continue;
                if (mark[cu] != cv) {
                    mark[cu] = cv;
                    slot[cu] = (int64_t)c.adj.size();
                    c.adj.push_back(cu);
                    c.ew.push_back(g.ew[e]);
                } else {
                    c.ew[slot[cu]] += g.ew[e];
                }
            }
        }
        c.xadj[cv + 1] = (int64_t)c.adj.size();
    }
    return c;
}

// Weights of the two sides of a split and the bounds they must keep.
struct Balance {
    double target[2];   // ideal weight of each side
    double maxw[2];     // largest admissible weight of each side
};

int64_t cut_of(const Graph& g, const std::vector<uint8_t>& side) {
    int64_t cut = 0;
    for (int32_t v = 0; v < g.n; ++v)
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e)
            if (side[g.adj[e]] != side[v]) cut += g.ew[e];
    return cut / 2;
}

// How far a split is outside its bounds (0 when admissible).
double excess(const int64_t w[2], const Balance& b) {
    return std::max(0.0, (double)w[0] - b.maxw[0]) + std::max(0.0, (double)w[1] - b.maxw[1]);
}

struct HeapEntry {
    int64_t gain;
    uint32_t stamp;
    int32_t v;
};
// Larger gain first; among equal gains the smaller vertex id (a total order,
// so the pop order does not depend on the heap implementation).
struct HeapLess {
    bool operator()(const HeapEntry& a, const HeapEntry& b) const {
        if (a.gain != b.gain) return a.gain < b.gain;
        return a.v > b.v;
    }
};

// Fiduccia-Mattheyses passes.  A move takes the vertex of largest gain
// (cut decrease) from the side that must shed weight, or, when both sides
// are admissible, from whichever side offers the larger gain.  Moved
// vertices are locked for the rest of the pass; the pass keeps the best
// prefix of its moves (admissible before smaller cut) and stops after
// `patience` moves without a better one.
void fm_refine(const Graph& g, std::vector<uint8_t>& side, const Balance& bal, int passes, int patience) {
    const int32_t n = g.n;
    std::vector<int64_t> gain(n), wdeg(n);
    std::vector<uint32_t> stamp(n, 0);
    const int64_t maxvw = n > 0 ? *std::max_element(g.vw.begin(), g.vw.end()) : 1;
    for (int32_t v = 0; v < n; ++v) {
        int64_t d = 0;
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) d += g.ew[e];
        wdeg[v] = d;
    }
    std::vector<uint8_t> locked(n);
    std::vector<int32_t> moves;
    std::vector<HeapEntry> heap[2];
    for (int pass = 0; pass < passes; ++pass) {
        int64_t w[2] = {0, 0};
        int64_t cut = 0;
        for (int32_t v = 0; v < n; ++v) {
            w[side[v]] += g.vw[v];
            int64_t ext = 0, in = 0;
            for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e)
                (side[g.adj[e]] != side[v] ? ext : in) += g.ew[e];
            gain[v] = ext - in;
            cut += ext;
        }
        cut /= 2;
        // boundary vertices enter the queues at once; interior ones only when
        // a side must shed weight and has no boundary vertex left
        heap[0].clear();
        heap[1].clear();
        bool all_in[2] = {false, false};
        for (int32_t v = 0; v < n; ++v)
            if (gain[v] + wdeg[v] > 0 || wdeg[v] == 0) heap[side[v]].push_back({gain[v], stamp[v], v});
        std::make_heap(heap[0].begin(), heap[0].end(), HeapLess());
        std::make_heap(heap[1].begin(), heap[1].end(), HeapLess());
        std::fill(locked.begin(), locked.end(), 0);
        moves.clear();
        auto top = [&](int s) -> int32_t {   // best live entry of side s, or -1
            auto& h = heap[s];
            for (;;) {
                while (!h.empty()) {
                    const HeapEntry& t = h.front();
                    if (!locked[t.v] && side[t.v] == s && stamp[t.v] == t.stamp) return t.v;
                    std::pop_heap(h.begin(), h.end(), HeapLess());
                    h.pop_back();
                }
                if (all_in[s]) return -1;
                all_in[s] = true;
                for (int32_t v = 0; v < n; ++v)
                    if (side[v] == s && !locked[v]) h.push_back({gain[v], stamp[v], v});
                std::make_heap(h.begin(), h.end(), HeapLess());
            }
        };
        const int64_t cut0 = cut;
        double best_exc = excess(w, bal);
        int64_t best_cut = cut;
        size_t best_len = 0;
        int since = 0;
        while (since < patience) {
            int from = -1;
            if ((double)w[0] > bal.maxw[0]) {
                from = 0;
            } else if ((double)w[1] > bal.maxw[1]) {
                from = 1;
            } else {
                // from an admissible state a move may overshoot the other
                // side's bound by one vertex: the next move then comes back
                // from that side, so vertices can trade places
                int64_t bg = 0;
                for (int s = 0; s < 2; ++s) {
                    const int32_t v = top(s);
                    if (v < 0 || (double)(w[1 - s] + g.vw[v]) > bal.maxw[1 - s] + (double)maxvw) continue;
                    if (from < 0 || gain[v] > bg) {
                        from = s;
                        bg = gain[v];
                    }
                }
            }
            if (from < 0) break;
            const int32_t v = top(from);
            if (v < 0) break;
            std::pop_heap(heap[from].begin(), heap[from].end(), HeapLess());
            heap[from].pop_back();
            const int to = 1 - from;
            side[v] = (uint8_t)to;
            locked[v] = 1;
            w[from] -= g.vw[v];
            w[to] += g.vw[v];
            cut -= gain[v];
            moves.push_back(v);
            for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
                const int32_t u = g.adj[e];
                gain[u] += side[u] == to ? -2 * g.ew[e] : 2 * g.ew[e];
                if (locked[u]) continue;
                ++stamp[u];
                heap[side[u]].push_back({gain[u], stamp[u], u});
                std::push_heap(heap[side[u]].begin(), heap[side[u]].end(), HeapLess());
            }
            gain[v] = -gain[v];
            const double exc = excess(w, bal);
            if (exc < best_exc || (exc == best_exc && cut < best_cut)) {
                best_exc = exc;
                best_cut = cut;
                best_len = moves.size();
                since = 0;
            } else {
                ++since;
            }
        }
        for (size_t i = moves.size(); i > best_len; --i) side[moves[i - 1]] ^= 1u;
        if (best_len == 0 || (best_cut >= cut0 && best_exc == 0.0 && pass > 0)) break;
    }
}

// Split of the coarsest graph: grow side 0 breadth-first from a random seed
// (a new seed whenever the region's component is used up) until it reaches
// its target weight, refine, and keep the best of several trials.
std::vector<uint8_t> initial_split(const Graph& g, const Balance& bal, Rng& rng) {
    const int32_t n = g.n;
    std::vector<uint8_t> best;
    double best_exc = 0.0;
    int64_t best_cut = 0;
    const int trials = n <= 1 ? 1 : 8;
    std::vector<int32_t> queue;
    for (int t = 0; t < trials; ++t) {
        std::vector<uint8_t> side(n, 1);
        std::vector<uint8_t> seen(n, 0);
        const std::vector<int32_t> order = random_order(n, rng);
        int64_t w0 = 0;
        size_t next_seed = 0;
        queue.clear();
        size_t head = 0;
        while ((double)w0 < bal.target[0]) {
            if (head == queue.size()) {
                while (next_seed < order.size() && seen[order[next_seed]]) ++next_seed;
                if (next_seed == order.size()) break;
                seen[order[next_seed]] = 1;
                queue.push_back(order[next_seed]);
            }
            const int32_t v = queue[head++];
            if ((double)(w0 + g.vw[v]) > bal.maxw[0] && w0 > 0) continue;
            side[v] = 0;
            w0 += g.vw[v];
            for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
                const int32_t u = g.adj[e];
                if (!seen[u]) {
                    seen[u] = 1;
                    queue.push_back(u);
                }
            }
        }
        fm_refine(g, side, bal, 4, std::max(20, n / 4));
        int64_t w[2] = {0, 0};
        for (int32_t v = 0; v < n; ++v) w[side[v]] += g.vw[v];
        const double exc = excess(w, bal);
        const int64_t cut = cut_of(g, side);
        if (best.empty() || exc < best_exc || (exc == best_exc && cut < best_cut)) {
            best = side;
            best_exc = exc;
            best_cut = cut;
        }
    }
    return best;
}

// Target and largest admissible weight of each side of a split of h into
// fractions frac0 : 1-frac0, each side at most ub times its share.
Balance split_bounds(const Graph& h, double frac0, double ub) {
    Balance b;
    const int64_t maxv = *std::max_element(h.vw.begin(), h.vw.end());
    b.target[0] = frac0 * (double)h.total;
    b.target[1] = (double)h.total - b.target[0];
    for (int s = 0; s < 2; ++s) {
        b.maxw[s] = std::max(ub * b.target[s], std::ceil(b.target[s]));
        // coarse vertices are heavy: allow one of them above the bound
        if (maxv > 1) b.maxw[s] = std::max(b.maxw[s], b.target[s] + (double)maxv);
    }
    return b;
}

// Multilevel bisection of g into sides of weight fractions frac0 : 1-frac0,
// each side at most ub times its share (and never below the next integer).
std::vector<uint8_t> bisect(const Graph& g, double frac0, double ub, Rng& rng) {
    constexpr int32_t kCoarsest = 120;
    std::vector<std::unique_ptr<Graph>> levels;
    std::vector<std::vector<int32_t>> cmaps;
    const Graph* cur = &g;
    while (cur->n > kCoarsest) {
        std::vector<int32_t> cmap;
        const int64_t maxvw = std::max<int64_t>(1, (int64_t)(1.5 * (double)cur->total / kCoarsest));
        auto c = std::make_unique<Graph>(coarsen(*cur, cmap, maxvw, rng));
        if (c->n > cur->n - cur->n / 20) break;   // matching stalled
        cmaps.push_back(std::move(cmap));
        levels.push_back(std::move(c));
        cur = levels.back().get();
    }
    auto bounds = [&](const Graph& h) { return split_bounds(h, frac0, ub); };
    std::vector<uint8_t> side = initial_split(*cur, bounds(*cur), rng);
    for (int l = (int)levels.size() - 1; l >= 0; --l) {
        const Graph& fine = l == 0 ? g : *levels[l - 1];
        std::vector<uint8_t> fs(fine.n);
        for (int32_t v = 0; v < fine.n; ++v) fs[v] = side[cmaps[l][v]];
        side.swap(fs);
        fm_refine(fine, side, bounds(fine), 4, std::max(50, std::min(fine.n / 50, 400)));
    }
    return side;
}

// Subgraph induced by the vertices of one side (ids: local -> parent local).
Graph induced(const Graph& g, const std::vector<uint8_t>& side, int s, std::vector<int32_t>& ids) {
    std::vector<int32_t> loc(g.n, -1);
    ids.clear();
    for (int32_t v = 0; v < g.n; ++v)
        if (side[v] == s) {
            loc[v] = (int32_t)ids.size();
            ids.push_back(v);
        }
    Graph h;
    h.n = (int32_t)ids.size();
    h.xadj.assign((size_t)h.n + 1, 0);
    h.vw.resize(h.n);
    for (int32_t i = 0; i < h.n; ++i) {
        const int32_t v = ids[i];
        h.vw[i] = g.vw[v];
        h.total += g.vw[v];
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
            const int32_t u = loc[g.adj[e]];
            if (u < 0) continue;
            h.adj.push_back(u);
            h.ew.push_back(g.ew[e]);
        }
        h.xadj[i + 1] = (int64_t)h.adj.size();
    }
    return h;
}

// Every side must keep at least as many vertices as the parts it will be
// split into; move the best-gain vertices across where a side fell short.
void ensure_counts(const Graph& g, std::vector<uint8_t>& side, int32_t k0, int32_t k1) {
    int32_t cnt[2] = {0, 0};
    for (int32_t v = 0; v < g.n; ++v) ++cnt[side[v]];
    const int32_t need[2] = {k0, k1};
    for (int s = 0; s < 2; ++s) {
        if (cnt[s] >= need[s]) continue;
        std::vector<std::pair<int64_t, int32_t>> cand;   // (-gain, v) of the other side
        for (int32_t v = 0; v < g.n; ++v) {
            if (side[v] == s) continue;
            int64_t gsum = 0;
            for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) gsum += side[g.adj[e]] == s ? g.ew[e] : -g.ew[e];
            cand.push_back({-gsum, v});
        }
        std::sort(cand.begin(), cand.end());
        for (size_t i = 0; i < cand.size() && cnt[s] < need[s]; ++i) {
            side[cand[i].second] = (uint8_t)s;
            ++cnt[s];
            --cnt[1 - s];
        }
    }
}

// Splits run on their own threads down to subgraphs of kParallelMin
// vertices, at most `threads` at a time.  Each split seeds its generator
// from (seed, first part, parts), so the partition does not depend on the
// thread schedule.
struct RecurseCtx {
    uint64_t seed;
    double ub;
    int32_t* part;
    std::atomic<int> spare;     // threads that may still be started
    std::atomic<bool> failed;   // a split on another thread threw
};
constexpr int32_t kParallelMin = 20000;
constexpr int kBisectTries = 3;      // bisections tried per split ...
constexpr int32_t kTryMin = 64;      // ... of graphs with at least this many vertices

void recurse(const Graph& g, const std::vector<int32_t>& ids, int32_t k, int32_t part0, RecurseCtx& C) {
    if (k == 1) {
        for (int32_t i = 0; i < g.n; ++i) C.part[ids[i]] = part0;
        return;
    }
    const int32_t k0 = k / 2, k1 = k - k0;
    Rng rng{C.seed ^ (0x9E3779B97F4A7C15ull * (uint64_t)(part0 + 1)) ^ ((uint64_t)k << 40)};
    // several multilevel bisections from the same generator, the best kept
    // (balance first, then cut)
    std::vector<uint8_t> side;
    {
        const double frac0 = (double)k0 / k;
        const Balance bal = split_bounds(g, frac0, C.ub);
        double best_exc = 0.0;
        int64_t best_cut = 0;
        const int tries = g.n >= kTryMin ? kBisectTries : 1;
        for (int t = 0; t < tries; ++t) {
            std::vector<uint8_t> s = bisect(g, frac0, C.ub, rng);
            int64_t w[2] = {0, 0};
            for (int32_t v = 0; v < g.n; ++v) w[s[v]] += g.vw[v];
            const double exc = excess(w, bal);
            const int64_t cut = cut_of(g, s);
            if (t == 0 || exc < best_exc || (exc == best_exc && cut < best_cut)) {
                side.swap(s);
                best_exc = exc;
                best_cut = cut;
            }
        }
    }
    ensure_counts(g, side, k0, k1);
    std::vector<int32_t> ids0, ids1;
    Graph h0 = induced(g, side, 0, ids0);
    Graph h1 = induced(g, side, 1, ids1);
    for (auto& v : ids0) v = ids[v];
    for (auto& v : ids1) v = ids[v];
    side.clear();
    side.shrink_to_fit();
    std::thread t;
    if (h0.n >= kParallelMin && k0 > 1 && C.spare.fetch_sub(1) > 0) {
        t = std::thread([&]() {
            try {
                recurse(h0, ids0, k0, part0, C);
            } catch (...) {
                C.failed = true;
            }
        });
    } else {
        if (h0.n >= kParallelMin && k0 > 1) C.spare.fetch_add(1);
        recurse(h0, ids0, k0, part0, C);
    }
    recurse(h1, ids1, k1, part0 + k0, C);
    if (t.joinable()) {
        t.join();
        C.spare.fetch_add(1);
    }
}

// Greedy k-way refinement of the final partition: each boundary vertex
// moves to the neighbouring part it has the most edges into when that beats
// the edges into its own part (or ties them and evens the sizes), as long as
// the receiving part stays within maxsize and the giving part keeps a
// vertex.  Passes repeat until one moves nothing.
void kway_refine(const Graph& g, int32_t* part, int32_t k, int64_t maxsize, int passes) {
    std::vector<int64_t> size(k, 0);
    for (int32_t v = 0; v < g.n; ++v) ++size[part[v]];
    std::vector<int32_t> nb_part;
    std::vector<int64_t> nb_w;
    for (int pass = 0; pass < passes; ++pass) {
        int64_t moved = 0;
        for (int32_t v = 0; v < g.n; ++v) {
            const int32_t own = part[v];
            nb_part.clear();
            nb_w.clear();
            int64_t in = 0;
            for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
                const int32_t q = part[g.adj[e]];
                if (q == own) {
                    in += g.ew[e];
                    continue;
                }
                size_t j = 0;
                while (j < nb_part.size() && nb_part[j] != q) ++j;
                if (j == nb_part.size()) {
                    nb_part.push_back(q);
                    nb_w.push_back(0);
                }
                nb_w[j] += g.ew[e];
            }
            if (nb_part.empty() || size[own] <= 1) continue;
            int32_t best = -1;
            int64_t bw = 0;
            for (size_t j = 0; j < nb_part.size(); ++j) {
                const int32_t q = nb_part[j];
                if (size[q] + 1 > maxsize) continue;
                const bool better = nb_w[j] > in || (nb_w[j] == in && size[q] + 1 < size[own]);
                if (!better) continue;
                if (best < 0 || nb_w[j] > bw || (nb_w[j] == bw && (size[q] < size[best] ||
                                                                   (size[q] == size[best] && q < best)))) {
                    best = q;
                    bw = nb_w[j];
                }
            }
            if (best < 0) continue;
            part[v] = best;
            --size[own];
            ++size[best];
            ++moved;
        }
        if (moved == 0) break;
    }
}

}  // namespace

ams_status partition_graph(int64_t n, const int64_t* rowptr, const int32_t* colind, int32_t nparts,
                           double imbalance, uint64_t seed, int32_t* part, int64_t* edge_cut) {
    if (n <= 0 || n >= (int64_t(1) << 31) || !rowptr || !colind || !part) {
        set_error("partition: n must be in [1, 2^31) and the arrays non-NULL");
        return AMS_ERR_INVALID_ARG;
    }
    if (nparts < 1 || nparts > n) {
        set_error("partition: nparts must be in [1, n]");
        return AMS_ERR_INVALID_ARG;
    }
    if (!(imbalance >= 0.0) || !std::isfinite(imbalance)) {
        set_error("partition: imbalance must be finite and >= 0");
        return AMS_ERR_INVALID_ARG;
    }
    if (imbalance == 0.0) imbalance = 0.03;
    if (rowptr[0] != 0) {
        set_error("partition: rowptr[0] must be 0");
        return AMS_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i]) {
            set_error("partition: rowptr decreases");
            return AMS_ERR_INVALID_ARG;
        }
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
            if (colind[e] < 0 || colind[e] >= n) {
                set_error("partition: column index out of range");
                return AMS_ERR_INVALID_ARG;
            }
    }
    // undirected graph of the pattern: both directions of every off-diagonal
    // entry, duplicates merged
    Graph g;
    g.n = (int32_t)n;
    std::vector<int64_t> deg((size_t)n + 1, 0);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
            if (colind[e] != i) {
                ++deg[i + 1];
                ++deg[(size_t)colind[e] + 1];
            }
    for (int64_t i = 0; i < n; ++i) deg[i + 1] += deg[i];
    std::vector<int32_t> both(deg[n]);
    {
        std::vector<int64_t> fill(deg.begin(), deg.end() - 1);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                const int32_t j = colind[e];
                if (j == i) continue;
                both[fill[i]++] = j;
                both[fill[j]++] = (int32_t)i;
            }
    }
    g.xadj.assign((size_t)n + 1, 0);
    g.adj.reserve(both.size());
    for (int64_t i = 0; i < n; ++i) {
        std::sort(both.begin() + deg[i], both.begin() + deg[i + 1]);
        int32_t* last = std::unique(both.data() + deg[i], both.data() + deg[i + 1]);
        g.adj.insert(g.adj.end(), both.data() + deg[i], last);
        g.xadj[i + 1] = (int64_t)g.adj.size();
    }
    g.ew.assign(g.adj.size(), 1);
    g.vw.assign(n, 1);
    g.total = n;

    // each part's weight may exceed n / nparts by the factor 1 + imbalance:
    // the bisections on the way down share that factor
    const int levels = (int)std::ceil(std::log2((double)nparts));
    const double ub = levels > 0 ? std::pow(1.0 + imbalance, 1.0 / levels) : 1.0 + imbalance;
    std::vector<int32_t> ids(n);
    for (int32_t i = 0; i < (int32_t)n; ++i) ids[i] = i;
    RecurseCtx ctx{seed, ub, part, {}, {}};
    ctx.spare = (int)std::min(std::thread::hardware_concurrency(), 64u) - 1;
    ctx.failed = false;
    try {
        recurse(g, ids, nparts, 0, ctx);
    } catch (const std::exception& e) {   // thread start or allocation failure
        set_error(std::string("partition: ") + e.what());
        return AMS_ERR_OOM;
    }
    if (ctx.failed) {
        set_error("partition: a split failed (allocation or thread start)");
        return AMS_ERR_OOM;
    }
    if (nparts > 1) {
        int64_t largest = 0;
        {
            std::vector<int64_t> size(nparts, 0);
            for (int32_t v = 0; v < (int32_t)n; ++v) largest = std::max(largest, ++size[part[v]]);
        }
        const int64_t maxsize = std::max<int64_t>(largest, (int64_t)std::floor((1.0 + imbalance) * (double)n / nparts));
        kway_refine(g, part, nparts, maxsize, 8);
    }
    if (edge_cut) {
        int64_t cut = 0;
        for (int32_t v = 0; v < (int32_t)n; ++v)
            for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e)
                if (g.adj[e] > v && part[g.adj[e]] != part[v]) ++cut;
        *edge_cut = cut;
    }
    return AMS_OK;
}

}  // namespace ams

extern "C" ams_status ams_partition(int64_t n, const int64_t* rowptr, const int32_t* colind, int32_t nparts,
                                    double imbalance, uint64_t seed, int32_t* part, int64_t* edge_cut) {
    ams::set_error("");
    return ams::partition_graph(n, rowptr, colind, nparts, imbalance, seed, part, edge_cut);
}
