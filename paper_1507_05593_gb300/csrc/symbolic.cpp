// Host symbolic analysis: nested-dissection ordering, within-separator ordering
// and block trees, supernodal row structures, descendants and levels.
//
//  * Nested dissection (Sections 2.2, 3.1) by recursive coordinate bisection of the
//    lattice positions of the nodes: a part with at most leaf_size nodes is a leaf;
//    otherwise the axis of largest extent (ties: lowest axis) is cut at the plane
//    lo + ext/2, the plane's nodes form the separator, numbered after the two
//    halves (postorder).  Inside a part nodes follow (z, y, x) lexicographic order.
//  * Every leaf and separator is one supernode; a separator with >= tau_O unknowns
//    and more than tau_D unknowns is reordered by recursive halving along its
//    longest bounding-box axis (Section 4.1) and gets an in-order labelled block tree.
//  * R_j (Section 2.1) is built per supernode from the rows below C_j of A's
//    columns in C_j and the rows of R_k below C_j for every supernode k whose
//    first row of R_k lies in C_j (its supernodal tree children).  This is the
//    smallest row set with the property the paper states for descendants (R_k
//    meets the rows after C_j only inside R_j); it equals the union of the column
//    structures whenever every supernode is an elimination-tree chain (lattice
//    orderings) and adds rows of exact zeros otherwise (the graph ordering).
#include <algorithm>
#include <iterator>
#include <limits>
#include <cmath>
#include <functional>
#include <numeric>

#include "rsc_internal.h"

namespace rsc {

namespace {

struct NodeSet {
    const int64_t* P;   // [nodes*3] integer lattice coordinates
};

void lex_sort(std::vector<int32_t>& ids, const int64_t* P) {
    std::sort(ids.begin(), ids.end(), [P](int32_t a, int32_t b) {
        for (int ax = 2; ax >= 0; --ax) {
            if (P[3 * a + ax] != P[3 * b + ax]) return P[3 * a + ax] < P[3 * b + ax];
        }
        return a < b;
    });
}

void nd_recurse(std::vector<int32_t>& ids, const int64_t* P, int leaf_size,
                std::vector<std::pair<uint8_t, std::vector<int32_t>>>& parts) {
    if (ids.empty()) return;
    if ((int64_t)ids.size() <= leaf_size) {
        lex_sort(ids, P);
        parts.emplace_back(0, std::move(ids));
        return;
    }
    int64_t lo[3], hi[3];
    for (int ax = 0; ax < 3; ++ax) { lo[ax] = INT64_MAX; hi[ax] = INT64_MIN; }
    for (int32_t i : ids)
        for (int ax = 0; ax < 3; ++ax) {
            lo[ax] = std::min(lo[ax], P[3 * i + ax]);
            hi[ax] = std::max(hi[ax], P[3 * i + ax]);
        }
    int ax = 0;
    int64_t best = -1;
    for (int a = 0; a < 3; ++a) {
        int64_t ext = hi[a] - lo[a] + 1;
        if (ext > best) { best = ext; ax = a; }
    }
    int64_t m = lo[ax] + best / 2;
    std::vector<int32_t> left, right, sep;
    for (int32_t i : ids) {
        int64_t v = P[3 * i + ax];
        if (v < m) left.push_back(i);
        else if (v > m) right.push_back(i);
        else sep.push_back(i);
    }
    std::vector<int32_t>().swap(ids);
    nd_recurse(left, P, leaf_size, parts);
    nd_recurse(right, P, leaf_size, parts);
    if (!sep.empty()) {
        lex_sort(sep, P);
        parts.emplace_back(1, std::move(sep));
    }
}

// Section 4.1: recursive halving along the longest bounding-box axis; returns the
// new node order and fills the in-order labelled tree (ranges in unknowns).
template <class C>
void geometric_split(const std::vector<int32_t>& ids_in, const C* P, int dof, int tau_D,
                     std::vector<int32_t>& out, BlockTree& t) {
    struct Rec { int label; int hi; };
    int counter = 0;
    // first pass counts blocks to size the arrays: a tree with L leaves has 2L-1 nodes
    std::function<int(int64_t)> count_leaves = [&](int64_t cnt) -> int {
        if (cnt * dof <= tau_D) return 1;
        return count_leaves(cnt / 2) + count_leaves(cnt - cnt / 2);
    };
    int L = count_leaves((int64_t)ids_in.size());
    int nb = 2 * L - 1;
    t.nblocks = nb;
    t.leaf.assign(nb + 1, 0);
    t.lo.assign(nb + 1, 0); t.mid.assign(nb + 1, 0); t.hi.assign(nb + 1, 0);
    t.left.assign(nb + 1, 0); t.right.assign(nb + 1, 0); t.parent.assign(nb + 1, 0);
    std::function<Rec(std::vector<int32_t>&, int)> rec = [&](std::vector<int32_t>& ids, int lo) -> Rec {
        if ((int64_t)ids.size() * dof <= tau_D) {
            int s = ++counter;
            t.leaf[s] = 1;
            t.lo[s] = lo;
            t.hi[s] = lo + (int)ids.size() * dof;
            t.mid[s] = t.hi[s];
            out.insert(out.end(), ids.begin(), ids.end());
            return {s, t.hi[s]};
        }
        C mn[3], mx[3];
        for (int a = 0; a < 3; ++a) { mn[a] = std::numeric_limits<C>::max(); mx[a] = std::numeric_limits<C>::lowest(); }
        for (int32_t i : ids)
            for (int a = 0; a < 3; ++a) {
                mn[a] = std::min(mn[a], P[3 * (int64_t)i + a]);
                mx[a] = std::max(mx[a], P[3 * (int64_t)i + a]);
            }
        int ax = 0;
        C best = -1;
        for (int a = 0; a < 3; ++a)
            if (mx[a] - mn[a] > best) { best = mx[a] - mn[a]; ax = a; }
        std::stable_sort(ids.begin(), ids.end(), [P, ax](int32_t a, int32_t b) {
            return P[3 * (int64_t)a + ax] < P[3 * (int64_t)b + ax];
        });
        size_t h = ids.size() / 2;
        std::vector<int32_t> l(ids.begin(), ids.begin() + h), r(ids.begin() + h, ids.end());
        Rec rl = rec(l, lo);
        int s = ++counter;
        Rec rr = rec(r, rl.hi);
        t.leaf[s] = 0;
        t.lo[s] = lo;
        t.mid[s] = rl.hi;
        t.hi[s] = rr.hi;
        t.left[s] = rl.label;
        t.right[s] = rr.label;
        t.parent[rl.label] = s;
        t.parent[rr.label] = s;
        return {s, rr.hi};
    };
    std::vector<int32_t> ids = ids_in;
    Rec root = rec(ids, 0);
    t.root = root.label;
    t.parent[root.label] = 0;
}

}  // namespace

// Supernodal row structures R_j, parents, levels and descendants of the partition S.sn_ptr.
static void build_structure(Symbolic& S) {
    const int64_t n = S.n;
    S.rows.clear();
    S.desc_k.clear();
    S.desc_p0.clear();
    S.desc_p1.clear();
    // supernodal row structures by union through the supernodal tree
    S.rows_ptr.assign(S.M + 1, 0);
    S.parent.assign(S.M, -1);
    S.level.assign(S.M, 0);
    std::vector<std::vector<int32_t>> children(S.M);
    std::vector<int32_t> mark(n, -1);
    std::vector<int32_t> acc;
    for (int j = 0; j < S.M; ++j) {
        int64_t c0 = S.sn_ptr[j], c1 = S.sn_ptr[j + 1];
        acc.clear();
        for (int64_t c = c0; c < c1; ++c)
            for (int64_t e = S.lp[c]; e < S.lp[c + 1]; ++e) {
                int32_t r = S.li[e];
                if (r >= c1 && mark[r] != j) { mark[r] = j; acc.push_back(r); }
            }
        int lev = 0;
        for (int32_t k : children[j]) {
            lev = std::max(lev, S.level[k] + 1);
            for (int64_t e = S.rows_ptr[k]; e < S.rows_ptr[k + 1]; ++e) {
                int32_t r = S.rows[e];
                if (r >= c1 && mark[r] != j) { mark[r] = j; acc.push_back(r); }
            }
        }
        S.level[j] = lev;
        std::sort(acc.begin(), acc.end());
        S.rows.insert(S.rows.end(), acc.begin(), acc.end());
        S.rows_ptr[j + 1] = (int64_t)S.rows.size();
        if (!acc.empty()) {
            S.parent[j] = S.snode_of[acc[0]];
            children[S.parent[j]].push_back(j);
        }
    }
    S.nlevels = 0;
    for (int j = 0; j < S.M; ++j) S.nlevels = std::max(S.nlevels, S.level[j] + 1);
    S.level_nodes.assign(S.nlevels, {});
    for (int j = 0; j < S.M; ++j) S.level_nodes[S.level[j]].push_back(j);

    // descendants: runs of R_k per supernode
    std::vector<std::vector<int32_t>> dk(S.M), d0(S.M), d1(S.M);
    for (int k = 0; k < S.M; ++k) {
        const int32_t* Rk = S.R(k);
        int r = S.nrows(k);
        int p = 0;
        while (p < r) {
            int j = S.snode_of[Rk[p]];
            int q = p;
            while (q < r && Rk[q] < S.sn_ptr[j + 1]) ++q;
            dk[j].push_back(k);
            d0[j].push_back(p);
            d1[j].push_back(q);
            p = q;
        }
    }
    S.desc_ptr.assign(S.M + 1, 0);
    for (int j = 0; j < S.M; ++j) {
        S.desc_ptr[j + 1] = S.desc_ptr[j] + (int64_t)dk[j].size();
        S.desc_k.insert(S.desc_k.end(), dk[j].begin(), dk[j].end());
        S.desc_p0.insert(S.desc_p0.end(), d0[j].begin(), d0[j].end());
        S.desc_p1.insert(S.desc_p1.end(), d1[j].begin(), d1[j].end());
    }
}

// Section 3.1 groups small supernodes "as in CHOLMOD": relaxed amalgamation.  Supernodes are
// visited in order (a postorder of the supernodal tree); group G absorbs the group L before it
// while L's parent lies in G (the first row of R_L is a column of G), neither is a compressed
// separator (>= tau_O columns) nor would the merged separator be one, and, with ns = c_L + c_G,
// R_M = R_G united with the rows of R_L after G, s(c, r) = c (c + 1) / 2 + c r stored entries
// and z = 1 - (s(L) + s(G)) / s(M): ns <= 4, or ns <= 16 and z <= 0.8, or ns <= 48 and z <= 0.1,
// or z <= 0.05 (CHOLMOD's default relaxation).  The merged group keeps G's kind; the structure
// is then rebuilt for the merged partition.  Columns keep their order.
static bool merge_ok(int64_t cL, int64_t rL, int64_t cG, int64_t rG, int64_t rM) {
    auto st = [](int64_t c, int64_t r) { return (double)(c * (c + 1) / 2 + c * r); };
    const int64_t ns = cL + cG;
    const double z = 1.0 - (st(cL, rL) + st(cG, rG)) / st(ns, rM);
    return ns <= 4 || (ns <= 16 && z <= 0.8) || (ns <= 48 && z <= 0.1) || z <= 0.05;
}

static void amalgamate_supernodes(Symbolic& S, int tau_O) {
    struct Grp { int64_t c0, c1; std::vector<int32_t> R; uint8_t kind; int first; int count; };
    std::vector<Grp> st;
    auto compressed = [&](uint8_t kind, int64_t c) { return kind == 1 && c >= tau_O; };
    for (int s = 0; s < S.M; ++s) {
        Grp G{S.sn_ptr[s], S.sn_ptr[s + 1], std::vector<int32_t>(S.R(s), S.R(s) + S.nrows(s)), S.kind[s], s, 1};
        while (!st.empty()) {
            const Grp& L = st.back();
            const int64_t cL = L.c1 - L.c0, cG = G.c1 - G.c0;
            if (L.R.empty() || L.R[0] < G.c0 || L.R[0] >= G.c1) break;
            if (compressed(L.kind, cL) || compressed(G.kind, cG) || compressed(G.kind, cL + cG)) break;
            std::vector<int32_t> RM;
            {
                std::vector<int32_t> tail;
                for (int32_t r : L.R)
                    if (r >= G.c1) tail.push_back(r);
                std::set_union(G.R.begin(), G.R.end(), tail.begin(), tail.end(), std::back_inserter(RM));
            }
            if (!merge_ok(cL, (int64_t)L.R.size(), cG, (int64_t)G.R.size(), (int64_t)RM.size())) break;
            G.c0 = L.c0;
            G.first = L.first;
            G.count += L.count;
            G.R.swap(RM);
            st.pop_back();
        }
        st.push_back(std::move(G));
    }
    if ((int)st.size() == S.M) return;
    std::vector<int64_t> ptr(1, 0);
    std::vector<uint8_t> kind;
    std::vector<BlockTree> tree;
    for (const Grp& g : st) {
        ptr.push_back(g.c1);
        kind.push_back(g.kind);
        tree.push_back(g.count == 1 ? S.tree[g.first] : BlockTree());
    }
    S.M = (int)st.size();
    S.sn_ptr.swap(ptr);
    S.kind.swap(kind);
    S.tree.swap(tree);
    for (int j = 0; j < S.M; ++j)
        for (int64_t c = S.sn_ptr[j]; c < S.sn_ptr[j + 1]; ++c) S.snode_of[c] = j;
    build_structure(S);
}

std::string analyze_symbolic(int64_t n, const int64_t* rp, const int32_t* ci, const double* val,
                             const double* coords, const rsc_options& o, Symbolic& S) {
    if (n <= 0) return "n must be positive";
    if (!rp || !ci || !val) return "row_ptr, col_idx and val are required";
    if (o.ordering != 0 && o.ordering != 1) return "ordering must be 0 (lattice) or 1 (graph)";
    // no positions: spectral positions (Section 4.3) and the graph ordering
    const bool graph = o.ordering == 1 || !coords;
    if (o.dof_per_node < 1 || n % o.dof_per_node) return "n must be a multiple of dof_per_node";
    if (o.leaf_size < 1 || o.tau_D < 1 || o.tau_O < 1) return "leaf_size, tau_O and tau_D must be positive";
    if (o.sample_block != 16) return "sample_block must be 16";
    if (n >= INT32_MAX) return "n must be below 2^31";
    if (rp[0] != 0) return "row_ptr[0] must be 0";
    for (int64_t i = 0; i < n; ++i) {
        if (rp[i + 1] < rp[i]) return "row_ptr must be nondecreasing";
        bool diag = false;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            if (ci[e] < 0 || ci[e] >= n) return "column index out of range";
            if (e > rp[i] && ci[e] <= ci[e - 1]) return "column indices must be sorted and unique";
            if (!std::isfinite(val[e])) return "non-finite matrix value";
            if (ci[e] == i) diag = true;
        }
        if (!diag) return "every row needs its diagonal entry";
    }
    // symmetric pattern: count (i,j) with j>i against (j,i) with i<j via a transpose walk
    {
        std::vector<int64_t> pos(rp, rp + n);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
                int32_t j = ci[e];
                // entry (i, j) must match the next unvisited entry of row j
                if (pos[j] >= rp[j + 1] || ci[pos[j]] != i) return "matrix pattern is not symmetric";
                ++pos[j];
            }
    }
    if (coords)
        for (int64_t i = 0; i < 3 * n; ++i) {
            if (!std::isfinite(coords[i])) return "non-finite coordinate";
            if (!graph && std::fabs(coords[i]) >= 2147483648.0)
                return "coordinates must be lattice positions below 2^31 in magnitude";
        }

    const int dof = o.dof_per_node;
    const int64_t nodes = n / dof;
    std::vector<int64_t> P;
    std::vector<double> X;   // real node positions (graph ordering)
    if (!graph) {
        P.resize(3 * nodes);
        for (int64_t v = 0; v < nodes; ++v)
            for (int a = 0; a < 3; ++a) P[3 * v + a] = (int64_t)std::llround(coords[3 * (v * dof) + a]);
    }

    // connected components of the node graph: each is dissected on its own, in order of
    // its smallest node (independent systems stacked block-diagonally become a forest)
    std::vector<int32_t> comp(nodes, -1);
    std::vector<std::vector<int32_t>> comps;
    {
        std::vector<int32_t> stack;
        for (int64_t v0 = 0; v0 < nodes; ++v0) {
            if (comp[v0] >= 0) continue;
            const int32_t cid = (int32_t)comps.size();
            comps.emplace_back();
            comp[v0] = cid;
            stack.assign(1, (int32_t)v0);
            while (!stack.empty()) {
                const int32_t v = stack.back();
                stack.pop_back();
                comps[cid].push_back(v);
                for (int d = 0; d < dof; ++d) {
                    const int64_t row = (int64_t)v * dof + d;
                    for (int64_t e = rp[row]; e < rp[row + 1]; ++e) {
                        const int32_t w = ci[e] / dof;
                        if (comp[w] < 0) { comp[w] = cid; stack.push_back(w); }
                    }
                }
            }
            std::sort(comps[cid].begin(), comps[cid].end());
        }
    }
    std::vector<std::pair<uint8_t, std::vector<int32_t>>> parts;
    if (graph) {
        std::vector<int64_t> gptr;
        std::vector<int32_t> gidx;
        node_graph(n, rp, ci, dof, gptr, gidx);
        if (coords) {
            X.resize(3 * nodes);
            for (int64_t v = 0; v < nodes; ++v)
                for (int a = 0; a < 3; ++a) X[3 * v + a] = coords[3 * (v * dof) + a];
        } else {
            spectral_positions(gptr, gidx, comps, X);
        }
        for (auto& cnodes : comps) {
            std::vector<int32_t> ids = cnodes;
            graph_nested_dissection(gptr, gidx, X.data(), o.leaf_size, ids, parts);
        }
    } else {
        for (auto& cnodes : comps) nd_recurse(cnodes, P.data(), o.leaf_size, parts);
    }
    const int ncomp_saved = (int)comps.size();
    std::vector<int32_t> comp_saved = std::move(comp);
    S = Symbolic();
    S.ncomp = ncomp_saved;
    S.comp_of = std::move(comp_saved);
    S.graph_ordering = graph;
    if (graph) S.node_pos = X;
    else S.node_pos.assign(P.begin(), P.end());
    S.n = n;
    S.dof = dof;
    S.M = (int)parts.size();
    S.kind.resize(S.M);
    S.tree.resize(S.M);
    S.sn_ptr.assign(S.M + 1, 0);
    S.perm.reserve(n);
    for (int j = 0; j < S.M; ++j) {
        auto& part = parts[j];
        S.kind[j] = part.first;
        int64_t nc = (int64_t)part.second.size() * dof;
        std::vector<int32_t> ids;
        if (part.first == 1 && nc >= o.tau_O && nc > o.tau_D) {
            if (graph) geometric_split(part.second, X.data(), dof, o.tau_D, ids, S.tree[j]);
            else geometric_split(part.second, P.data(), dof, o.tau_D, ids, S.tree[j]);
        } else {
            ids = std::move(part.second);
        }
        for (int32_t v : ids)
            for (int d = 0; d < dof; ++d) S.perm.push_back((int32_t)(v * dof + d));
        S.sn_ptr[j + 1] = S.sn_ptr[j] + nc;
    }
    S.iperm.assign(n, 0);
    for (int64_t i = 0; i < n; ++i) S.iperm[S.perm[i]] = (int32_t)i;
    S.snode_of.assign(n, 0);
    for (int j = 0; j < S.M; ++j)
        for (int64_t c = S.sn_ptr[j]; c < S.sn_ptr[j + 1]; ++c) S.snode_of[c] = j;

    // permuted lower triangle by column (A symmetric: row perm[c] lists column perm[c])
    S.lp.assign(n + 1, 0);
    for (int64_t c = 0; c < n; ++c) {
        int64_t o_ = S.perm[c], cnt = 0;
        for (int64_t e = rp[o_]; e < rp[o_ + 1]; ++e)
            if (S.iperm[ci[e]] >= c) ++cnt;
        S.lp[c + 1] = S.lp[c] + cnt;
    }
    S.li.resize(S.lp[n]);
    S.lsrc.resize(S.lp[n]);
    {
        std::vector<std::pair<int32_t, int64_t>> tmp;
        for (int64_t c = 0; c < n; ++c) {
            tmp.clear();
            int64_t o_ = S.perm[c];
            for (int64_t e = rp[o_]; e < rp[o_ + 1]; ++e) {
                int32_t r = S.iperm[ci[e]];
                if (r >= c) tmp.emplace_back(r, e);
            }
            std::sort(tmp.begin(), tmp.end());
            for (size_t t = 0; t < tmp.size(); ++t) {
                S.li[S.lp[c] + t] = tmp[t].first;
                S.lsrc[S.lp[c] + t] = tmp[t].second;
            }
        }
    }

    build_structure(S);
    if (o.amalgamate) amalgamate_supernodes(S, o.tau_O);
    return "";
}

}  // namespace rsc
