// Host-side graph work of the setup: input validation, the subdomain-major
// index maps (Section 3.1) and a nested-dissection ordering of the coarse
// (subdomain) graph used to lay out the coarse Cholesky factor's inverse.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "ams_internal.h"

namespace ams {

ams_status validate_system(const HostCSR& A, const int32_t* part, int32_t nparts) {
    const int64_t n = A.n;
    char buf[256];
    if (n <= 0 || n >= (int64_t(1) << 31)) {
        set_error("n must be in [1, 2^31)");
        return AMS_ERR_INVALID_ARG;
    }
    if (nparts <= 0 || nparts > n) {
        set_error("nparts must be in [1, n]");
        return AMS_ERR_INVALID_ARG;
    }
    if (A.rowptr[0] != 0) {
        set_error("rowptr[0] must be 0");
        return AMS_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < n; ++i) {
        const int64_t b = A.rowptr[i], e = A.rowptr[i + 1];
        if (e < b) {
            std::snprintf(buf, sizeof buf, "rowptr decreases at row %lld", (long long)i);
            set_error(buf);
            return AMS_ERR_INVALID_ARG;
        }
        bool diag = false;
        for (int64_t t = b; t < e; ++t) {
            const int32_t c = A.colind[t];
            if (c < 0 || c >= n) {
                std::snprintf(buf, sizeof buf, "column index out of range in row %lld", (long long)i);
                set_error(buf);
                return AMS_ERR_INVALID_ARG;
            }
            if (t > b && A.colind[t - 1] >= c) {
                std::snprintf(buf, sizeof buf, "columns not strictly ascending in row %lld", (long long)i);
                set_error(buf);
                return AMS_ERR_INVALID_ARG;
            }
            if (c == i) {
                diag = true;
                if (!(A.vals[t] > 0.0)) {
                    std::snprintf(buf, sizeof buf, "non-positive diagonal in row %lld", (long long)i);
                    set_error(buf);
                    return AMS_ERR_NOT_SPD;
                }
            }
            if (!std::isfinite(A.vals[t])) {
                set_error("non-finite matrix value");
                return AMS_ERR_INVALID_ARG;
            }
            // symmetric partner (c, i) with the identical value
            const int32_t* cb = A.colind.data() + A.rowptr[c];
            const int32_t* ce = A.colind.data() + A.rowptr[c + 1];
            const int32_t* f = std::lower_bound(cb, ce, (int32_t)i);
            if (f == ce || *f != i || A.vals[A.rowptr[c] + (f - cb)] != A.vals[t]) {
                std::snprintf(buf, sizeof buf, "matrix not symmetric at (%lld, %d)", (long long)i, c);
                set_error(buf);
                return AMS_ERR_INVALID_ARG;
            }
        }
        if (!diag) {
            std::snprintf(buf, sizeof buf, "missing diagonal in row %lld", (long long)i);
            set_error(buf);
            return AMS_ERR_INVALID_ARG;
        }
    }
    std::vector<int64_t> cnt(nparts, 0);
    for (int64_t i = 0; i < n; ++i) {
        if (part[i] < 0 || part[i] >= nparts) {
            std::snprintf(buf, sizeof buf, "part[%lld] out of range", (long long)i);
            set_error(buf);
            return AMS_ERR_INVALID_ARG;
        }
        cnt[part[i]]++;
    }
    for (int32_t s = 0; s < nparts; ++s)
        if (cnt[s] == 0) {
            std::snprintf(buf, sizeof buf, "subdomain %d is empty", s);
            set_error(buf);
            return AMS_ERR_INVALID_ARG;
        }
    return AMS_OK;
}

// Stable counting sort by subdomain id: dofs of Omega_i in ascending order.
void build_index_maps(int64_t n, const int32_t* part, int32_t nparts,
                      std::vector<int64_t>& perm, std::vector<int64_t>& iperm,
                      std::vector<int64_t>& sub_ptr) {
    sub_ptr.assign(nparts + 1, 0);
    for (int64_t i = 0; i < n; ++i) sub_ptr[part[i] + 1]++;
    for (int32_t s = 0; s < nparts; ++s) sub_ptr[s + 1] += sub_ptr[s];
    std::vector<int64_t> fill(sub_ptr.begin(), sub_ptr.end() - 1);
    perm.assign(n, 0);
    iperm.assign(n, 0);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t k = fill[part[i]]++;
        perm[k] = i;
        iperm[i] = k;
    }
}

// ---------------------------------------------------------------------------
// Nested dissection of the coarse graph.  Each call splits a connected
// vertex set at the middle level of a breadth-first level structure rooted
// at a pseudo-peripheral vertex: the vertices of that level form a
// separator, since an edge never joins two levels more than one apart.
// Nodes are emitted in post-order, so every subtree owns a contiguous range
// of coarse rows ending with its own rows.
// ---------------------------------------------------------------------------
namespace {

struct NDContext {
    const std::vector<int64_t>* adj_ptr;
    const std::vector<int32_t>* adj;
    const std::vector<int32_t>* weight;
    int32_t leaf_weight;
    std::vector<int32_t> mark;     // subset id of each vertex
    std::vector<int32_t> level;
    int32_t next_mark = 1;
    std::vector<NDNode>* nodes;
    int64_t row = 0;
};

void bfs_levels(NDContext& C, int32_t root, int32_t mk, const std::vector<int32_t>& members,
                std::vector<int32_t>& order, int32_t& nlev) {
    for (int32_t v : members) C.level[v] = -1;
    order.clear();
    order.push_back(root);
    C.level[root] = 0;
    size_t head = 0;
    nlev = 1;
    while (head < order.size()) {
        const int32_t u = order[head++];
        for (int64_t t = (*C.adj_ptr)[u]; t < (*C.adj_ptr)[u + 1]; ++t) {
            const int32_t v = (*C.adj)[t];
            if (C.mark[v] == mk && C.level[v] < 0) {
                C.level[v] = C.level[u] + 1;
                nlev = std::max(nlev, C.level[v] + 1);
                order.push_back(v);
            }
        }
    }
}

// Returns the node ids of the roots emitted for `members`.
std::vector<int32_t> nd_rec(NDContext& C, std::vector<int32_t> members);

int32_t emit_leaf(NDContext& C, std::vector<int32_t> subs, int64_t cstart) {
    std::sort(subs.begin(), subs.end());
    NDNode nd;
    nd.subs = subs;
    nd.cstart = cstart;
    nd.a = C.row;
    for (int32_t s : subs) nd.k += (*C.weight)[s];
    C.row += nd.k;
    C.nodes->push_back(nd);
    return (int32_t)C.nodes->size() - 1;
}

std::vector<int32_t> nd_component(NDContext& C, std::vector<int32_t> members) {
    const int64_t cstart = C.row;
    int64_t wsum = 0;
    for (int32_t v : members) wsum += (*C.weight)[v];
    if (wsum <= C.leaf_weight || members.size() <= 2)
        return {emit_leaf(C, members, cstart)};
    const int32_t mk = C.next_mark++;
    for (int32_t v : members) C.mark[v] = mk;
    std::vector<int32_t> order;
    int32_t nlev = 0;
    // pseudo-peripheral root: repeat BFS from the last vertex reached
    int32_t root = *std::min_element(members.begin(), members.end());
    for (int rep = 0; rep < 3; ++rep) {
        bfs_levels(C, root, mk, members, order, nlev);
        const int32_t far = order.back();
        if (far == root) break;
        int32_t prev = nlev;
        bfs_levels(C, far, mk, members, order, nlev);
        root = far;
        if (nlev <= prev) break;
    }
    bfs_levels(C, root, mk, members, order, nlev);
    if (nlev < 3) return {emit_leaf(C, members, cstart)};
    // level whose cumulative weight first reaches half of the total
    std::vector<int64_t> lw(nlev, 0);
    for (int32_t v : members) lw[C.level[v]] += (*C.weight)[v];
    int64_t acc = 0;
    int32_t L = 1;
    for (int32_t l = 0; l < nlev; ++l) {
        acc += lw[l];
        if (2 * acc >= wsum) { L = l; break; }
    }
    L = std::max(1, std::min(L, nlev - 2));
    std::vector<int32_t> lo, hi, sep;
    for (int32_t v : members) {
        const int32_t l = C.level[v];
        (l < L ? lo : (l > L ? hi : sep)).push_back(v);
    }
    std::vector<int32_t> kids = nd_rec(C, lo);
    std::vector<int32_t> k2 = nd_rec(C, hi);
    kids.insert(kids.end(), k2.begin(), k2.end());
    const int32_t id = emit_leaf(C, sep, cstart);
    for (int32_t c : kids) (*C.nodes)[c].parent = id;
    return {id};
}

std::vector<int32_t> nd_rec(NDContext& C, std::vector<int32_t> members) {
    std::vector<int32_t> roots;
    if (members.empty()) return roots;
    // split into connected components
    const int32_t mk = C.next_mark++;
    for (int32_t v : members) C.mark[v] = mk;
    std::sort(members.begin(), members.end());
    std::vector<int32_t> comp;
    for (int32_t s : members) {
        if (C.mark[s] != mk) continue;
        comp.clear();
        comp.push_back(s);
        C.mark[s] = -mk;
        for (size_t h = 0; h < comp.size(); ++h) {
            const int32_t u = comp[h];
            for (int64_t t = (*C.adj_ptr)[u]; t < (*C.adj_ptr)[u + 1]; ++t) {
                const int32_t v = (*C.adj)[t];
                if (C.mark[v] == mk) {
                    C.mark[v] = -mk;
                    comp.push_back(v);
                }
            }
        }
        std::vector<int32_t> r = nd_component(C, comp);
        roots.insert(roots.end(), r.begin(), r.end());
        // restore marks of remaining members for later components
        for (int32_t v : members)
            if (C.mark[v] != -mk && C.mark[v] != mk) C.mark[v] = -mk;  // visited by recursion
    }
    return roots;
}

}  // namespace

void nested_dissection(int32_t N, const std::vector<int64_t>& adj_ptr,
                       const std::vector<int32_t>& adj, const std::vector<int32_t>& weight,
                       int32_t leaf_weight, std::vector<NDNode>& nodes) {
    NDContext C;
    C.adj_ptr = &adj_ptr;
    C.adj = &adj;
    C.weight = &weight;
    C.leaf_weight = leaf_weight;
    C.mark.assign(N, 0);
    C.level.assign(N, -1);
    C.nodes = &nodes;
    nodes.clear();
    std::vector<int32_t> all(N);
    std::iota(all.begin(), all.end(), 0);
    nd_rec(C, all);
}

}  // namespace ams
