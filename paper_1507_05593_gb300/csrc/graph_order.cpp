// Host ordering for general sparsity: graph nested dissection guided by node
// positions, and spectral positions where none are given (Section 4.3).
//
//  * Graph nested dissection (the paper's partitioner is unnamed; its non-grid
//    examples need one that does not assume a lattice): a node set with at most
//    leaf_size nodes is a leaf; otherwise the nodes are sorted by (X[axis], id) along
//    the axis of largest bounding-box extent (ties: lowest axis) and cut at the
//    median, L = the first floor(size/2) nodes, R = the rest.  The vertex separator
//    is the smaller boundary of the cut, S_L = nodes of L with a neighbour in R or
//    S_R = nodes of R with a neighbour in L (S_L on ties); removing it leaves no edge
//    between the halves.  Recursion on L - S and R - S, then the separator
//    (postorder); nodes inside a leaf or separator in ascending id order.
//  * Spectral positions (Section 4.3): node i sits at (v1_i, v2_i, v3_i) for the
//    three lowest eigenvectors of the node graph's Laplacian (off-diagonal -1 per
//    edge, diagonal = degree), per connected component, the component's constant
//    null vector skipped.  The paper asks only for low accuracy: a Lanczos run with
//    full reorthogonalisation (every new vector projected twice against the earlier
//    ones and the constant vector, so the null vector never enters the Krylov space),
//    then the Ritz vectors of the three smallest Ritz values of the tridiagonal
//    matrix, whose eigenproblem is solved by cyclic Jacobi rotations.  The run takes
//    min(m - 1, LANCZOS_MAX) steps for a component of m nodes: exact (up to rounding)
//    for small components, an approximation for large ones.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "rsc_internal.h"

namespace rsc {

namespace {

constexpr int LANCZOS_MAX = 160;      // largest Krylov dimension
constexpr int64_t LANCZOS_BIG = 200000;   // components above this many nodes use 64 steps

// eigenvalues (ascending) and eigenvectors (columns of Z, k x k row-major) of the
// symmetric k x k matrix A (row-major, overwritten) by cyclic Jacobi rotations
void jacobi_eigen(std::vector<double>& A, int k, std::vector<double>& w, std::vector<double>& Z) {
    Z.assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) Z[(size_t)i * k + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < k; ++p) {
            diag += A[(size_t)p * k + p] * A[(size_t)p * k + p];
            for (int q = p + 1; q < k; ++q) off += A[(size_t)p * k + q] * A[(size_t)p * k + q];
        }
        if (off <= 1e-30 * diag || off == 0.0) break;
        for (int p = 0; p < k - 1; ++p)
            for (int q = p + 1; q < k; ++q) {
                const double apq = A[(size_t)p * k + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * k + p], aqq = A[(size_t)q * k + q];
                // rotation angle that zeroes A[p][q]: tan(2 theta) = 2 apq / (aqq - app)
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < k; ++r) {   // columns p, q
                    const double arp = A[(size_t)r * k + p], arq = A[(size_t)r * k + q];
                    A[(size_t)r * k + p] = c * arp - s * arq;
                    A[(size_t)r * k + q] = s * arp + c * arq;
                }
                for (int r = 0; r < k; ++r) {   // rows p, q
                    const double apr = A[(size_t)p * k + r], aqr = A[(size_t)q * k + r];
                    A[(size_t)p * k + r] = c * apr - s * aqr;
                    A[(size_t)q * k + r] = s * apr + c * aqr;
                }
                for (int r = 0; r < k; ++r) {
                    const double zrp = Z[(size_t)r * k + p], zrq = Z[(size_t)r * k + q];
                    Z[(size_t)r * k + p] = c * zrp - s * zrq;
                    Z[(size_t)r * k + q] = s * zrp + c * zrq;
                }
            }
    }
    // sort ascending
    std::vector<int> ord(k);
    for (int i = 0; i < k; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return A[(size_t)a * k + a] < A[(size_t)b * k + b]; });
    w.resize(k);
    std::vector<double> Zs((size_t)k * k);
    for (int j = 0; j < k; ++j) {
        w[j] = A[(size_t)ord[j] * k + ord[j]];
        for (int r = 0; r < k; ++r) Zs[(size_t)r * k + j] = Z[(size_t)r * k + ord[j]];
    }
    Z.swap(Zs);
}

// positions of one component (nodes ids, m of them) into X (nodes x 3)
void component_positions(const std::vector<int64_t>& ptr, const std::vector<int32_t>& idx,
                         const std::vector<int32_t>& ids, std::vector<int32_t>& loc, double* X) {
    const int64_t m = (int64_t)ids.size();
    if (m < 2) return;
    for (int64_t a = 0; a < m; ++a) loc[ids[a]] = (int32_t)a;
    const int kmax = m > LANCZOS_BIG ? 64 : LANCZOS_MAX;
    const int k = (int)std::min<int64_t>(m - 1, kmax);
    std::vector<double> Q((size_t)(k + 1) * m), alpha(k, 0.0), beta(k + 1, 0.0), w(m);
    auto lap = [&](const double* x, double* y) {
        for (int64_t a = 0; a < m; ++a) {
            const int32_t v = ids[a];
            double s = (double)(ptr[v + 1] - ptr[v]) * x[a];
            for (int64_t e = ptr[v]; e < ptr[v + 1]; ++e) s -= x[loc[idx[e]]];
            y[a] = s;
        }
    };
    // project out the constant vector and the accepted Lanczos vectors, twice
    auto orth = [&](double* x, int upto) {
        for (int pass = 0; pass < 2; ++pass) {
            double mean = 0.0;
            for (int64_t a = 0; a < m; ++a) mean += x[a];
            mean /= (double)m;
            for (int64_t a = 0; a < m; ++a) x[a] -= mean;
            for (int j = 0; j < upto; ++j) {
                const double* q = Q.data() + (size_t)j * m;
                double d = 0.0;
                for (int64_t a = 0; a < m; ++a) d += q[a] * x[a];
                for (int64_t a = 0; a < m; ++a) x[a] -= d * q[a];
            }
        }
    };
    auto norm = [&](const double* x) {
        double s = 0.0;
        for (int64_t a = 0; a < m; ++a) s += x[a] * x[a];
        return std::sqrt(s);
    };
    // deterministic start: a multiplicative hash of the local index
    double* q0 = Q.data();
    for (int64_t a = 0; a < m; ++a) q0[a] = (double)((uint32_t)((uint64_t)(a + 1) * 2654435761ull)) / 4294967296.0 - 0.5;
    orth(q0, 0);
    double nq = norm(q0);
    for (int64_t a = 0; a < m; ++a) q0[a] /= nq;
    int steps = k;
    for (int j = 0; j < k; ++j) {
        const double* q = Q.data() + (size_t)j * m;
        lap(q, w.data());
        double aj = 0.0;
        for (int64_t a = 0; a < m; ++a) aj += q[a] * w[a];
        alpha[j] = aj;
        orth(w.data(), j + 1);
        const double b = norm(w.data());
        if (j + 1 == k || b <= 1e-12 * std::fabs(aj) + 1e-300) { steps = j + 1; break; }
        beta[j + 1] = b;
        double* qn = Q.data() + (size_t)(j + 1) * m;
        for (int64_t a = 0; a < m; ++a) qn[a] = w[a] / b;
    }
    // Rayleigh-Ritz on the tridiagonal T (steps x steps)
    std::vector<double> T((size_t)steps * steps, 0.0), ev, Z;
    for (int j = 0; j < steps; ++j) {
        T[(size_t)j * steps + j] = alpha[j];
        if (j + 1 < steps) T[(size_t)j * steps + j + 1] = T[(size_t)(j + 1) * steps + j] = beta[j + 1];
    }
    jacobi_eigen(T, steps, ev, Z);
    const int nc = std::min(3, steps);
    for (int c = 0; c < nc; ++c)
        for (int64_t a = 0; a < m; ++a) {
            double s = 0.0;
            for (int j = 0; j < steps; ++j) s += Q[(size_t)j * m + a] * Z[(size_t)j * steps + c];
            X[3 * (int64_t)ids[a] + c] = s;
        }
}

void graph_nd_recurse(const std::vector<int64_t>& ptr, const std::vector<int32_t>& idx, const double* X,
                      int leaf_size, std::vector<int32_t>& ids, std::vector<uint8_t>& side,
                      std::vector<std::pair<uint8_t, std::vector<int32_t>>>& parts) {
    if (ids.empty()) return;
    if ((int64_t)ids.size() <= leaf_size) {
        std::sort(ids.begin(), ids.end());
        parts.emplace_back(0, std::move(ids));
        return;
    }
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = INFINITY; hi[a] = -INFINITY; }
    for (int32_t v : ids)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], X[3 * (int64_t)v + a]);
            hi[a] = std::max(hi[a], X[3 * (int64_t)v + a]);
        }
    int ax = 0;
    for (int a = 1; a < 3; ++a)
        if (hi[a] - lo[a] > hi[ax] - lo[ax]) ax = a;
    std::sort(ids.begin(), ids.end(), [X, ax](int32_t a, int32_t b) {
        const double xa = X[3 * (int64_t)a + ax], xb = X[3 * (int64_t)b + ax];
        return xa < xb || (xa == xb && a < b);
    });
    const size_t h = ids.size() / 2;
    for (size_t i = 0; i < ids.size(); ++i) side[ids[i]] = i < h ? 1 : 2;
    std::vector<int32_t> SL, SR;
    for (size_t i = 0; i < ids.size(); ++i) {
        const int32_t v = ids[i];
        const uint8_t mine = side[v], other = mine == 1 ? 2 : 1;
        for (int64_t e = ptr[v]; e < ptr[v + 1]; ++e)
            if (side[idx[e]] == other) { (mine == 1 ? SL : SR).push_back(v); break; }
    }
    const bool take_left = SL.size() <= SR.size();
    std::vector<int32_t>& S = take_left ? SL : SR;
    for (int32_t v : S) side[v] = 3;   // in the separator
    std::vector<int32_t> L, R;
    for (int32_t v : ids) {
        if (side[v] == 1) L.push_back(v);
        else if (side[v] == 2) R.push_back(v);
        side[v] = 0;
    }
    std::vector<int32_t>().swap(ids);
    std::sort(L.begin(), L.end());
    std::sort(R.begin(), R.end());
    graph_nd_recurse(ptr, idx, X, leaf_size, L, side, parts);
    graph_nd_recurse(ptr, idx, X, leaf_size, R, side, parts);
    if (!S.empty()) {
        std::sort(S.begin(), S.end());
        parts.emplace_back(1, std::move(S));
    }
}

}  // namespace

void node_graph(int64_t n, const int64_t* rp, const int32_t* ci, int dof, std::vector<int64_t>& ptr,
                std::vector<int32_t>& idx) {
    const int64_t nodes = n / dof;
    ptr.assign(nodes + 1, 0);
    idx.clear();
    std::vector<int32_t> nb;
    for (int64_t v = 0; v < nodes; ++v) {
        nb.clear();
        for (int d = 0; d < dof; ++d) {
            const int64_t row = v * dof + d;
            for (int64_t e = rp[row]; e < rp[row + 1]; ++e) {
                const int32_t u = ci[e] / dof;
                if (u != v) nb.push_back(u);
            }
        }
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        idx.insert(idx.end(), nb.begin(), nb.end());
        ptr[v + 1] = (int64_t)idx.size();
    }
}

void spectral_positions(const std::vector<int64_t>& ptr, const std::vector<int32_t>& idx,
                        const std::vector<std::vector<int32_t>>& comps, std::vector<double>& X) {
    const int64_t nodes = (int64_t)ptr.size() - 1;
    X.assign(3 * nodes, 0.0);
    std::vector<int32_t> loc(nodes, 0);
    for (const auto& ids : comps) component_positions(ptr, idx, ids, loc, X.data());
}

void graph_nested_dissection(const std::vector<int64_t>& ptr, const std::vector<int32_t>& idx, const double* X,
                             int leaf_size, std::vector<int32_t>& ids,
                             std::vector<std::pair<uint8_t, std::vector<int32_t>>>& parts) {
    std::vector<uint8_t> side(ptr.size() - 1, 0);
    graph_nd_recurse(ptr, idx, X, leaf_size, ids, side, parts);
}

}  // namespace rsc
