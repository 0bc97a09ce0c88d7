"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: the worked
example of Section 2.1, published known-answer vectors, brute-force symbolic
elimination, a library dense Cholesky of the permuted matrix, explicitly formed
dense blocks, dense SVDs and PCG residuals.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import dense
from oracle import factor as F
from oracle.ordering import geometric_split, nested_dissection
from oracle.philox import gaussian_block, philox4x32_10
from oracle.scatter import gather_rows, scatter_rows

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mat(txt):
    return np.array([[float(x) for x in r.split()] for r in txt.split(";")])


# --------------------------------------------------------------------------- scatter / gather

def test_scatter_rows_worked_example():
    rec = {}
    for line in open(os.path.join(GOLDEN, "scatter_rows_example.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split(":", 1)
        rec[k.strip()] = v.strip()
    B = _mat(rec["B"])
    R1 = [int(x) for x in rec["R1"].split()]
    R2 = [int(x) for x in rec["R2"].split()]
    out = scatter_rows(B, R1, R2)
    np.testing.assert_array_equal(out, _mat(rec["OUT"]))
    np.testing.assert_array_equal(gather_rows(out, R2, R1), B)


def test_gather_inverts_scatter_random():
    rng = np.random.default_rng(1)
    R2 = np.sort(rng.choice(1000, 60, replace=False))
    R1 = np.sort(rng.choice(R2, 25, replace=False))
    B = rng.standard_normal((25, 3))
    np.testing.assert_array_equal(gather_rows(scatter_rows(B, R1, R2), R2, R1), B)
    with pytest.raises(ValueError):
        scatter_rows(B[:1], [1001], R2)


# --------------------------------------------------------------------------- Philox

def test_philox_known_answers():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        out = philox4x32_10(np.array(w[:4], np.uint32), np.array(w[4:6], np.uint32))
        assert [int(x) for x in out] == w[6:10]


def test_gaussian_moments_and_counter_independence():
    g = gaussian_block(20000, 16, seed=7, block_id=3, pass_=0, attempt=0)
    assert abs(g.mean()) < 0.01
    assert abs(g.var() - 1.0) < 0.02
    assert abs(np.mean(g ** 4) - 3.0) < 0.1          # Gaussian kurtosis
    c = np.corrcoef(g[:, 0], g[:, 1])[0, 1]
    assert abs(c) < 0.03
    g2 = gaussian_block(20000, 16, seed=7, block_id=3, pass_=1, attempt=0)
    assert abs(np.corrcoef(g.ravel(), g2.ravel())[0, 1]) < 0.01
    # same counters -> same numbers; a prefix of rows is a prefix of the matrix
    np.testing.assert_array_equal(g[:100], gaussian_block(100, 16, 7, 3, 0, 0))


# --------------------------------------------------------------------------- dense kernels

def test_dense_kernels_vs_library():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((40, 40))
    S = X @ X.T + 40 * np.eye(40)
    L = dense.cholesky(S)
    np.testing.assert_allclose(L, np.linalg.cholesky(S), rtol=1e-13, atol=1e-13)
    B = rng.standard_normal((40, 5))
    np.testing.assert_allclose(dense.solve_lower(L, B), sla.solve_triangular(L, B, lower=True), rtol=1e-12)
    np.testing.assert_allclose(dense.solve_lower_T(L, B), sla.solve_triangular(L.T, B, lower=False),
                               rtol=1e-12)
    with pytest.raises(dense.NotPositiveDefinite):
        dense.cholesky(S - 1000 * np.eye(40))
    Y = rng.standard_normal((50, 16))
    Q = dense.householder_q(Y)
    np.testing.assert_allclose(Q.T @ Q, np.eye(16), atol=1e-14)
    np.testing.assert_allclose(Q @ (Q.T @ Y), Y, atol=1e-12)


# --------------------------------------------------------------------------- ordering

def test_nested_dissection_grid_closed_form():
    p = W.poisson7(32)
    order, parts = nested_dissection(p.coords, 64)
    assert sorted(order.tolist()) == list(range(p.n))
    # last part = top separator: the plane x = 16 (32*32 nodes)
    kind, top = parts[-1]
    assert kind == "sep" and top.size == 1024
    assert np.all(p.coords[top, 0] == 16)
    # its in-plane order is lexicographic (z, y, x)
    zyx = p.coords[top][:, ::-1]
    assert all(tuple(zyx[i]) < tuple(zyx[i + 1]) for i in range(len(top) - 1))
    assert all(ids.size <= 64 for k, ids in parts if k == "leaf")
    # every separator is a plane (one coordinate constant)
    for k, ids in parts:
        if k == "sep":
            assert any(np.ptp(p.coords[ids, a]) == 0 for a in range(3))


def test_nested_dissection_separates():
    """Nodes of two sibling subtrees are never adjacent in A (vertex separators)."""
    p = W.poisson7(12)
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, F.Options(leaf_size=16))
    L = _brute_structure(an.Ap.toarray() != 0)
    # A separator property implies: columns of two different leaves never share a
    # nonzero of L below the leaves (fill stays inside ancestor separators).
    leaves = [j for j in range(an.nsuper) if an.ordering.kinds[j] == "leaf"]
    for a in leaves[:6]:
        a0, a1 = an.cols(a)
        for b in leaves:
            if b == a:
                continue
            b0, b1 = an.cols(b)
            assert not L[b0:b1, a0:a1].any()


def test_block_tree_inorder_labels():
    """Section 4.1, Eq. (ldjLabel): a 4-leaf tree has 7 blocks, root 4 with
    children 2 and 6, leaves 1, 3, 5, 7 on the diagonal in order."""
    p = W.poisson7(32)
    _, parts = nested_dissection(p.coords, 64)
    top = parts[-1][1]
    ids, t = geometric_split(top, p.coords, 256)
    assert t.nblocks == 7 and t.root == 4
    assert (t.left[4], t.right[4]) == (2, 6)
    assert (t.left[2], t.right[2], t.left[6], t.right[6]) == (1, 3, 5, 7)
    assert [s for s in range(1, 8) if t.leaf[s]] == [1, 3, 5, 7]
    assert [t.lo[s] for s in (1, 3, 5, 7)] == [0, 256, 512, 768]
    assert t.rows(4) == (512, 1024) and t.cols(4) == (0, 512)
    assert t.rows(2) == (256, 512) and t.cols(2) == (0, 256)
    # halves are split along the longest bounding-box axis: y first (plane x = 16)
    assert np.all(p.coords[ids[:512], 1] < 16) and np.all(p.coords[ids[512:], 1] >= 16)
    # labels of a complete in-order tree: node at height h has children s -/+ 2^(h-1)
    _, t16 = geometric_split(top, p.coords, 64)
    assert t16.nblocks == 31 and t16.root == 16
    for s in range(1, 32):
        h = (s & -s).bit_length() - 1
        if h:
            assert (t16.left[s], t16.right[s]) == (s - (1 << (h - 1)), s + (1 << (h - 1)))


# --------------------------------------------------------------------------- symbolic

def _brute_structure(nz):
    """Boolean Gaussian elimination: structure of the Cholesky factor (lower)."""
    nz = nz.copy()
    n = nz.shape[0]
    for k in range(n):
        rows = np.nonzero(nz[k + 1:, k])[0] + k + 1
        nz[np.ix_(rows, rows)] = True
    return np.tril(nz)


@pytest.mark.parametrize("maker", [lambda: W.poisson7(6), lambda: W.poisson7(5, 7, 4),
                                   lambda: W.elasticity_q1(3, incl=(1, 2))])
def test_symbolic_vs_brute_force(maker):
    p = maker()
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords,
                   F.Options(leaf_size=8, dof_per_node=p.dof_per_node))
    L = _brute_structure(an.Ap.toarray() != 0)
    sym = an.sym
    for j in range(an.nsuper):
        c0, c1 = an.cols(j)
        brute = np.nonzero(L[c1:, c0:c1].any(axis=1))[0] + c1
        np.testing.assert_array_equal(sym.rows[j], brute)
    for j in range(an.nsuper):
        c0, c1 = an.cols(j)
        brute_D = [k for k in range(j) if np.any((sym.rows[k] >= c0) & (sym.rows[k] < c1))]
        assert [k for k, _, _ in sym.desc[j]] == brute_D
        for k, pD, pO in sym.desc[j]:
            Rk = sym.rows[k]
            assert pD.tolist() == [q for q in range(Rk.size) if c0 <= Rk[q] < c1]
            assert pO.tolist() == [q for q in range(Rk.size) if Rk[q] in set(sym.rows[j].tolist())]
            # R_k meets C^O_j only inside R_j (Section 2.1)
            assert set(Rk[Rk >= c1].tolist()) <= set(sym.rows[j].tolist())


# --------------------------------------------------------------------------- exact factor

def _assemble_L(f):
    """Dense approximate factor from the oracle's blocks (hierarchical blocks expanded)."""
    an = f.an
    n = an.n
    L = np.zeros((n, n))
    for j in range(an.nsuper):
        c0, c1 = an.cols(j)
        L[c0:c1, c0:c1] = _assemble_LD(f, j)
        s = f.sn[j]
        Rj = an.sym.rows[j]
        if Rj.size:
            L[Rj, c0:c1] = s.V @ s.U.T if s.compressed else s.LO
    return L


def _assemble_LD(f, j):
    D = f.sn[j].D
    if not D.hierarchical:
        return D.L
    t = D.tree
    c = t.hi[t.root]
    H = np.zeros((c, c))
    for s in range(1, t.nblocks + 1):
        r0, r1 = t.rows(s)
        q0, q1 = t.cols(s)
        H[r0:r1, q0:q1] = D.leafL[s] if t.leaf[s] else D.V[s] @ D.U[s].T
    return H


@pytest.mark.parametrize("maker", [lambda: W.poisson7(4), lambda: W.poisson7(8), lambda: W.poisson7(6, 9, 5),
                                   lambda: W.diffusion_grf(8, 2.0, 3.0, 0),
                                   lambda: W.elasticity_q1(4, incl=(1, 3))])
def test_exact_factor_matches_dense_cholesky(maker):
    p = maker()
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords,
                   F.Options(leaf_size=8, tau_O=16, tau_D=8, dof_per_node=p.dof_per_node))
    f = F.factor(an, 0.0)
    L = _assemble_L(f)
    Ap = an.Ap.toarray()
    assert np.linalg.norm(L @ L.T - Ap) / np.linalg.norm(Ap) <= 1e-13
    Lref = np.linalg.cholesky(Ap)
    assert np.abs(L - Lref).max() <= 1e-12 * np.abs(Lref).max()
    x, it, rr, ok = F.solve(an, f, p.b, 1e-8)
    assert ok and it <= 2 and rr <= 1e-8


# --------------------------------------------------------------------------- compressed factor

@pytest.fixture(scope="module")
def compressed8():
    p = W.poisson7(10)
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords,
                   F.Options(leaf_size=8, tau_O=24, tau_D=16))
    f = F.factor(an, 0.05)
    return p, an, f


def _prefix_schur(f, j):
    """Dense Schur complement block column of supernode j from the dense factor of
    all earlier supernodes: A(:, C_j) - L(:, <C_j) L(C_j, <C_j)^T."""
    an = f.an
    c0, c1 = an.cols(j)
    L = _assemble_L(f)
    Ap = an.Ap.toarray()
    return Ap[:, c0:c1] - L[:, :c0] @ L[c0:c1, :c0].T


def test_offdiag_multiply_vs_explicit(compressed8):
    p, an, f = compressed8
    js = [j for j in range(an.nsuper) if f.sn[j].compressed and an.sym.rows[j].size]
    assert js
    rng = np.random.default_rng(2)
    for j in js:
        c0, c1 = an.cols(j)
        Rj = an.sym.rows[j]
        S = _prefix_schur(f, j)
        LD = _assemble_LD(f, j)
        LO = sla.solve_triangular(LD, S[Rj].T, lower=True).T        # U^O_j (L^D_j)^{-T}
        G = rng.standard_normal((c1 - c0, 5))
        np.testing.assert_allclose(f.offdiag_multiply(j, G), LO @ G, rtol=1e-10, atol=1e-11)
        H = rng.standard_normal((Rj.size, 5))
        np.testing.assert_allclose(f.offdiag_multiply_T(j, H), LO.T @ H, rtol=1e-10, atol=1e-11)
        # the stored compression meets its tolerance against the explicit block
        s = f.sn[j]
        err = np.linalg.norm(LO - s.V @ s.U.T) / np.linalg.norm(LO)
        assert err <= 2 * f.tol
        np.testing.assert_allclose(s.U.T @ s.U, np.eye(s.U.shape[1]), atol=1e-13)
        # rank is at most one 16-column pass beyond the passes that reach the SVD
        # rank needed for tol/2 in Frobenius norm
        sv = np.linalg.svd(LO, compute_uv=False)
        tail = np.sqrt(np.cumsum((sv ** 2)[::-1]))[::-1] / np.linalg.norm(sv)
        need = int(np.sum(tail > f.tol / 2))
        assert s.U.shape[1] <= 16 * ((need + 15) // 16) + 16


def test_diagonal_blocks_vs_explicit(compressed8):
    p, an, f = compressed8
    rng = np.random.default_rng(3)
    js = [j for j in range(an.nsuper) if f.sn[j].compressed and f.sn[j].D.hierarchical]
    assert js
    for j in js:
        D = f.sn[j].D
        t = D.tree
        c0, c1 = an.cols(j)
        S = _prefix_schur(f, j)[c0:c1]                  # U^D_j as a dense matrix
        H = _assemble_LD(f, j)
        # Alg. 4: hierarchical solves equal dense triangular solves with the assembled block
        G = rng.standard_normal((c1 - c0, 3))
        np.testing.assert_allclose(f.diagonal_solve(j, G, False), sla.solve_triangular(H, G, lower=True),
                                   rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(f.diagonal_solve(j, G, True),
                                   sla.solve_triangular(H.T, G, lower=False), rtol=1e-10, atol=1e-10)
        for s in range(1, t.nblocks + 1):
            r0, r1 = t.rows(s)
            q0, q1 = t.cols(s)
            # block Cholesky relation: L_s = (S(rows,cols) - H(rows,:lo) H(cols,:lo)^T) H(cols,cols)^{-T}
            rhs = S[r0:r1, q0:q1] - H[r0:r1, :q0] @ H[q0:q1, :q0].T
            if t.leaf[s]:
                np.testing.assert_allclose(D.leafL[s], np.linalg.cholesky(rhs), rtol=1e-10, atol=1e-12)
                continue
            Ls = sla.solve_triangular(H[q0:q1, q0:q1], rhs.T, lower=True).T
            Gs = rng.standard_normal((q1 - q0, 4))
            np.testing.assert_allclose(f.diagonal_multiply(j, s, Gs), Ls @ Gs, rtol=1e-9, atol=1e-11)
            Gr = rng.standard_normal((r1 - r0, 4))
            np.testing.assert_allclose(f.diagonal_multiply_T(j, s, Gr), Ls.T @ Gr, rtol=1e-9, atol=1e-11)
            assert np.linalg.norm(Ls - D.V[s] @ D.U[s].T) <= 2 * f.tol_D * np.linalg.norm(Ls) + 1e-14


def test_preconditioner_apply_vs_dense(compressed8):
    p, an, f = compressed8
    L = _assemble_L(f)
    r = np.random.default_rng(4).standard_normal(p.n)
    z = F.apply_preconditioner(f, r)
    P = an.ordering.perm
    y = np.linalg.solve(L @ L.T, r[P])
    zz = np.empty_like(y)
    zz[P] = y
    np.testing.assert_allclose(z, zz, rtol=1e-9, atol=1e-12)


def test_offdiag_compression_keeps_schur_pd():
    """Section 3.2 (Eq. scPlusPos): with diagonal blocks exact, the Schur complement
    after a compressed supernode exceeds the exact one by L^O (I - U U^T) L^O^T >= 0,
    and the factorization never needs a restart."""
    for maker in (lambda: W.poisson7(10), lambda: W.diffusion_grf(10, 2.0, 3.0, 1)):
        p = maker()
        an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords,
                       F.Options(leaf_size=8, tau_O=24, tau_D=16, diag_compress=False))
        f = F.factor(an, 0.5)
        assert f.restarts == 0
        for j in range(an.nsuper):
            s = f.sn[j]
            if not (s.compressed and an.sym.rows[j].size):
                continue
            S = _prefix_schur(f, j)
            c0, c1 = an.cols(j)
            LO = sla.solve_triangular(s.D.L, S[an.sym.rows[j]].T, lower=True).T
            diff = LO @ LO.T - s.V @ s.V.T
            assert np.linalg.eigvalsh(diff).min() >= -1e-12 * np.abs(LO @ LO.T).max()


def test_restart_path(monkeypatch):
    """Section 5.3: an indefinite diagonal block restarts with a tighter diagonal
    tolerance (tol_D / 1.25); the planted failure is in the oracle, on the CPU."""
    p = W.poisson7(10)
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, F.Options(leaf_size=8, tau_O=24, tau_D=16))
    calls = {"n": 0}
    orig = F.Factor.factor_diagonal

    def failing(self, j, s):
        if self.restarts == 0 and calls["n"] == 0:
            calls["n"] += 1
            raise dense.NotPositiveDefinite("planted")
        return orig(self, j, s)

    monkeypatch.setattr(F.Factor, "factor_diagonal", failing)
    f = F.factor(an, 0.1)
    assert f.restarts == 1 and abs(f.tol_D - 0.1 / 1.25) < 1e-15 and f.diag_compress


def test_restart_switches_diag_compression_off(monkeypatch):
    p = W.poisson7(10)
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords,
                   F.Options(leaf_size=8, tau_O=24, tau_D=16, max_restarts=2))
    orig = F.Factor.factor_diagonal

    def always_fail(self, j, s):
        raise dense.NotPositiveDefinite("planted")

    monkeypatch.setattr(F.Factor, "factor_diagonal", always_fail)
    f = F.factor(an, 0.1)
    assert f.restarts == 3 and not f.diag_compress
    x, it, rr, ok = F.solve(an, f, p.b)
    assert ok


# --------------------------------------------------------------------------- PCG

@pytest.mark.parametrize("tol", [0.3, 0.1, 0.01])
def test_pcg_reaches_tolerance(tol):
    p = W.diffusion_grf(12, 2.0, 3.0, 0)
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, F.Options(leaf_size=16, tau_O=40, tau_D=32))
    f = F.factor(an, tol)
    assert any(s.compressed for s in f.sn)
    x, it, rr, ok = F.solve(an, f, p.b, 1e-8)
    assert ok and rr <= 1e-8
    A = p.scipy()
    assert np.linalg.norm(p.b - A @ x) / np.linalg.norm(p.b) <= 1e-8


# --------------------------------------------------------------------------- fixed-rank form (Section 5.2)

def test_rank_heuristic_closed_form():
    """Eq. rankFunction with k = min(m, n): hand-computed values, the cap at k, and the
    degenerate sizes."""
    assert F.rank_heuristic(256, 300, 0.5, 8) == 72          # 0.5 * 16 * 8 + 8
    assert F.rank_heuristic(5000, 1024, 1.0, 5) == 325       # 1 * 32 * 10 + 5
    assert F.rank_heuristic(100, 100, 0.5, 0) == 34          # ceil(0.5 * 10 * 6.64386) = ceil(33.22)
    assert F.rank_heuristic(20, 64, 2.0, 8) == 20            # 38.66 -> 39 + 8 = 47, capped at 20
    assert F.rank_heuristic(1, 9, 3.0, 4) == 1               # log2(1) = 0: p, capped at 1
    assert F.rank_heuristic(0, 9, 3.0, 4) == 0
    assert F.rank_heuristic(64, 64, 0.0, 6) == 6


def _spectrum_matrix(m, c, sv, seed):
    rng = np.random.default_rng(seed)
    Qa, _ = np.linalg.qr(rng.standard_normal((m, len(sv))))
    Qb, _ = np.linalg.qr(rng.standard_normal((c, len(sv))))
    return (Qa * sv) @ Qb.T


@pytest.mark.parametrize("q", [0, 1, 2])
@pytest.mark.parametrize("r", [16, 40, 57])
def test_fixed_rank_range_finder_is_one_shot_alg3(q, r):
    """The blocked 16-column passes with the stopping test off span exactly what Alg. 3's
    one-shot form spans: orth((B^T B)^q B^T G) for G the first r sampled columns, formed
    here directly with numpy from the same Philox stream; V = B U, U orthonormal.  A
    missing or extra power iteration, or a wrong sample column, moves the subspace by O(1)."""
    p = W.poisson7(4)
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, F.Options(power_iters=q, seed=7))
    f = F.Factor(an)
    m, c = 150, 120
    sv = 1.0 / (1.0 + np.arange(min(m, c)))
    B = _spectrum_matrix(m, c, sv, 11)
    bid = (5 << 12) | 3
    V, U = f._range_finder(m, c, 0.0, bid, lambda X: B @ X, lambda G: B.T @ G, cap=r)
    assert U.shape == (c, r) and V.shape == (m, r)
    np.testing.assert_allclose(U.T @ U, np.eye(r), atol=1e-13)
    np.testing.assert_allclose(V, B @ U, atol=1e-13)
    G = np.hstack([gaussian_block(m, 16, 7, bid, t, 0) for t in range((r + 15) // 16)])[:, :r]
    Y = B.T @ G
    for _ in range(q):
        Y = B.T @ (B @ Y)
    Qref, _ = np.linalg.qr(Y)
    # two backward-stable orthonormalisations of Y span subspaces within O(u cond(Y))
    assert np.linalg.norm(U @ U.T - Qref @ Qref.T, 2) <= 20 * 1.1e-16 * np.linalg.cond(Y)


@pytest.mark.parametrize("q", [0, 1])
def test_fixed_rank_error_within_randomized_bound(q):
    """Halko, Martinsson and Tropp (2011), Thm. 10.5: with k = r - p and p >= 2 oversampling
    columns, E||B - B U U^T||_F <= sqrt(1 + k/(p - 1)) (sum_{i>k} s_i^2)^{1/2}.  One seeded
    draw is checked against 3x that expectation; power iterations may only help."""
    p_ = W.poisson7(4)
    an = F.analyze(p_.n, p_.row_ptr, p_.col_idx, p_.val, p_.coords, F.Options(power_iters=q, seed=3))
    f = F.Factor(an)
    m, c, r, ov = 200, 160, 48, 8
    sv = np.exp(-np.arange(160) / 15.0)
    B = _spectrum_matrix(m, c, sv, 4)
    _, U = f._range_finder(m, c, 0.0, 9, lambda X: B @ X, lambda G: B.T @ G, cap=r)
    err = np.linalg.norm(B - B @ U @ U.T)
    k = r - ov
    bound = np.sqrt(1 + k / (ov - 1)) * np.sqrt(np.sum(sv[k:] ** 2))
    assert err <= 3 * bound
    assert err >= np.sqrt(np.sum(sv[r:] ** 2)) * (1 - 1e-12)   # never better than the SVD


@pytest.mark.parametrize("maker", [lambda: W.poisson7(8), lambda: W.diffusion_grf(8, 2.0, 3.0, 0),
                                   lambda: W.elasticity_q1(4, incl=(1, 3))])
def test_fixed_rank_full_rank_is_exact(maker):
    """Ranks of Eq. rankFunction at or above min(m, n) for every block: nothing is dropped
    and the compressed factor is the exact Cholesky factor (Alg. 1) to rounding."""
    p = maker()
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords,
                   F.Options(leaf_size=8, tau_O=16, tau_D=8, dof_per_node=p.dof_per_node))
    f = F.factor_fixed_rank(an, 100.0, 100.0, 0)
    assert any(s.compressed for s in f.sn) and any(s.compressed and s.D.hierarchical for s in f.sn)
    L = _assemble_L(f)
    Ap = an.Ap.toarray()
    assert np.linalg.norm(L @ L.T - Ap) / np.linalg.norm(Ap) <= 1e-12
    x, it, rr, ok = F.solve(an, f, p.b, 1e-8)
    assert ok and it <= 2


def test_fixed_rank_block_ranks_and_errors():
    """Every compressed block gets exactly the rank of Eq. rankFunction (alpha^O for L^O_j,
    alpha^D for internal diagonal blocks, k = min(m, n)), with an orthonormal U, and its
    error is within the randomized bound of the explicit block's SVD tail; PCG converges."""
    p = W.poisson7(10)
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, F.Options(leaf_size=8, tau_O=24, tau_D=16))
    aO, aD, ov = 0.4, 0.7, 4
    f = F.factor_fixed_rank(an, aO, aD, ov)
    assert f.restarts == 0
    n_off = n_diag = 0
    for j in range(an.nsuper):
        s = f.sn[j]
        if not s.compressed:
            continue
        c0, c1 = an.cols(j)
        m = an.sym.rows[j].size
        if m:
            n_off += 1
            r = s.U.shape[1]
            assert r == F.rank_heuristic(m, c1 - c0, aO, ov) < min(m, c1 - c0), j
            np.testing.assert_allclose(s.U.T @ s.U, np.eye(r), atol=1e-13)
            S = _prefix_schur(f, j)
            LO = sla.solve_triangular(_assemble_LD(f, j), S[an.sym.rows[j]].T, lower=True).T
            sv = np.linalg.svd(LO, compute_uv=False)
            k = r - ov
            bound = np.sqrt(1 + k / (ov - 1)) * np.sqrt(np.sum(sv[k:] ** 2))
            assert np.linalg.norm(LO - s.V @ s.U.T) <= 3 * bound, j
        if s.D.hierarchical:
            t = s.D.tree
            for b in range(1, t.nblocks + 1):
                if not t.leaf[b]:
                    n_diag += 1
                    r0, r1 = t.rows(b)
                    q0, q1 = t.cols(b)
                    assert s.D.U[b].shape[1] == F.rank_heuristic(r1 - r0, q1 - q0, aD, ov), (j, b)
    assert n_off and n_diag
    x, it, rr, ok = F.solve(an, f, p.b, 1e-8)
    assert ok and rr <= 1e-8
    A = p.scipy()
    assert np.linalg.norm(p.b - A @ x) / np.linalg.norm(p.b) <= 1e-8


def test_fixed_rank_restart_grows_alpha_D(monkeypatch):
    """Section 5.3: an indefinite diagonal block restarts with alpha^D <- 1.25 alpha^D
    (planted failure in the oracle, on the CPU)."""
    p = W.poisson7(10)
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, F.Options(leaf_size=8, tau_O=24, tau_D=16))
    calls = {"n": 0}
    orig = F.Factor.factor_diagonal

    def failing(self, j, s):
        if self.restarts < 2 and calls["n"] < 2:
            calls["n"] += 1
            raise dense.NotPositiveDefinite("planted")
        return orig(self, j, s)

    monkeypatch.setattr(F.Factor, "factor_diagonal", failing)
    f = F.factor_fixed_rank(an, 0.5, 0.5, 4)
    assert f.restarts == 2 and abs(f.alpha_D - 0.5 * 1.25 ** 2) < 1e-15 and f.diag_compress
    with pytest.raises(ValueError):
        F.factor_fixed_rank(an, -1.0)


# --------------------------------------------------------------------------- graph ordering, spectral coordinates

from oracle.ordering import graph_nested_dissection, node_graph, spectral_coordinates  # noqa: E402


def _path_graph(n):
    ptr = [0]
    idx = []
    for v in range(n):
        nb = [u for u in (v - 1, v + 1) if 0 <= u < n]
        idx += nb
        ptr.append(len(idx))
    return np.array(ptr), np.array(idx)


def test_graph_nd_path_worked_example():
    """Hand-computed from the definition (path 0-1-...-9, X = index, leaf_size 2):
    [0..9] -> L [0..4], R [5..9], S_L {4} (ties go to L);  [0..3] -> S {1}, leaves [0], [2,3];
    [5..9] -> S {6}, leaf [5], [7..9] -> S {7}, leaf [8,9].  Postorder: 0 | 2 3 | 1 | 5 |
    8 9 | 7 | 6 | 4."""
    ptr, idx = _path_graph(10)
    X = np.stack([np.arange(10.0), np.zeros(10), np.zeros(10)], axis=1)
    order, parts = graph_nested_dissection(ptr, idx, X, leaf_size=2)
    assert order.tolist() == [0, 2, 3, 1, 5, 8, 9, 7, 6, 4]
    assert [k for k, _ in parts] == ["leaf", "leaf", "sep", "leaf", "leaf", "sep", "sep", "sep"]


def test_graph_nd_grid_top_separator_is_a_grid_line():
    """8 x 8 grid (5-point graph), X = lattice positions: the median cut along x puts
    columns 0-3 in L; both boundaries are one column of 8 nodes, the tie goes to L, so the
    last part is the column x = 3; every node appears once."""
    p = W.poisson7(8, 8, 1)
    ptr, idx = node_graph(p.n, p.row_ptr, p.col_idx)
    order, parts = graph_nested_dissection(ptr, idx, p.coords, leaf_size=4)
    assert sorted(order.tolist()) == list(range(64))
    kind, top = parts[-1]
    assert kind == "sep" and sorted(top.tolist()) == [3 + 8 * y for y in range(8)]


@pytest.mark.parametrize("maker", [lambda: W.poisson7(6, 5, 4), lambda: W.diffusion_grf(7, 2.0, 3.0, 1),
                                   lambda: W.elasticity_q1(3, incl=(1, 2))])
def test_graph_nd_separators_separate(maker):
    """Every separator the recursion emits cuts its node set in two: re-running the
    definition's steps independently (component labelling of the set minus S by BFS), no
    edge joins the two remaining halves; and the exact factor with this ordering is the
    Cholesky factor of the permuted matrix."""
    p = maker()
    dof = p.dof_per_node
    ptr, idx = node_graph(p.n, p.row_ptr, p.col_idx, dof)
    X = p.coords[::dof]
    order, parts = graph_nested_dissection(ptr, idx, X, leaf_size=6)
    assert sorted(order.tolist()) == list(range(p.n // dof))
    # reconstruct each call's node set: in postorder, a separator's set is itself plus the
    # parts emitted since the call began; recompute the median halves and check the cut
    pos = {}
    for i, (_, ids) in enumerate(parts):
        for v in ids.tolist():
            pos[v] = i
    seen = 0
    for i, (kind, S) in enumerate(parts):
        if kind != "sep":
            continue
        # the call that emitted S dissected S plus a contiguous run of earlier parts; find the
        # largest run whose union with S is connected through edges touching S or each other
        run = []
        for j in range(i - 1, -1, -1):
            run.append(parts[j][1])
            allv = np.concatenate(run + [S])
            pts = X[allv]
            ext = pts.max(axis=0) - pts.min(axis=0)
            ax = int(np.argmax(ext))
            srt = allv[np.lexsort((allv, pts[:, ax]))]
            h = allv.size // 2
            L, R = set(srt[:h].tolist()), set(srt[h:].tolist())
            sset = set(S.tolist())
            SL = {v for v in L if any(u in R for u in idx[ptr[v]:ptr[v + 1]])}
            SR = {v for v in R if any(u in L for u in idx[ptr[v]:ptr[v + 1]])}
            if (SL if len(SL) <= len(SR) else SR) == sset:
                Lr, Rr = L - sset, R - sset
                for v in Lr:
                    assert not any(u in Rr for u in idx[ptr[v]:ptr[v + 1]].tolist())
                seen += 1
                break
    assert seen == sum(k == "sep" for k, _ in parts)
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords,
                   F.Options(leaf_size=6, tau_O=10 ** 9, dof_per_node=dof, ordering=1))
    f = F.factor(an, 0.0)
    L = _assemble_L(f)
    Ap = an.Ap.toarray()
    assert np.linalg.norm(L @ L.T - Ap) / np.linalg.norm(Ap) <= 1e-13


def test_spectral_coordinates_path_closed_form():
    """Path graph of n nodes: Laplacian eigenvectors cos(pi k (i + 1/2) / n), eigenvalues
    2 - 2 cos(pi k / n); the coordinates are the modes k = 1, 2, 3 up to sign."""
    n = 40
    ptr, idx = _path_graph(n)
    X = spectral_coordinates(ptr, idx)
    i = np.arange(n)
    for k in (1, 2, 3):
        v = np.cos(np.pi * k * (i + 0.5) / n)
        v /= np.linalg.norm(v)
        assert abs(abs(X[:, k - 1] @ v) - 1.0) <= 1e-10


def test_spectral_coordinates_box_grid_modes():
    """9 x 7 x 5 grid graph: the Laplacian of a Cartesian product has the products of the
    path modes c_m,k(t) = cos(pi k (t + 1/2) / m) as eigenvectors, eigenvalue the sum of
    2 - 2 cos(pi k / m).  Lowest non-constant: c_9,1(x) (0.121), c_7,1(y) (0.198), then
    c_9,1(x) c_7,1(y) (0.319) below c_5,1(z) (0.382): the three coordinates, up to sign."""
    p = W.poisson7(9, 7, 5)
    ptr, idx = node_graph(p.n, p.row_ptr, p.col_idx)
    X = spectral_coordinates(ptr, idx)
    x, y = p.coords[:, 0], p.coords[:, 1]
    cx = np.cos(np.pi * (x + 0.5) / 9)
    cy = np.cos(np.pi * (y + 0.5) / 7)
    for c, v in enumerate((cx, cy, cx * cy)):
        v = v / np.linalg.norm(v)
        assert abs(abs(X[:, c] @ v) - 1.0) <= 1e-10


def test_spectral_coordinates_components_and_end_to_end():
    """Two disjoint grids: each component gets its own modes (no constant vector, zero mean
    per component); analysis without coordinates uses them and PCG reaches 1e-8 with the
    compressed factor."""
    import scipy.sparse as sp
    a, b = W.poisson7(6), W.poisson7(5, 4, 3)
    A = sp.block_diag([a.scipy(), b.scipy()]).tocsr()
    A.sort_indices()
    ptr, idx = node_graph(A.shape[0], A.indptr, A.indices)
    comp = np.r_[np.zeros(a.n, int), np.ones(b.n, int)]
    X = spectral_coordinates(ptr, idx, comp)
    for c in (0, 1):
        assert np.abs(X[comp == c].mean(axis=0)).max() <= 1e-12
        assert np.abs(np.linalg.norm(X[comp == c], axis=0) - 1.0).max() <= 1e-12
    p = W.diffusion_grf(12, 2.0, 3.0, 0)
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, None, F.Options(leaf_size=16, tau_O=40, tau_D=32))
    f = F.factor(an, 0.05)
    assert any(s.compressed for s in f.sn)
    x, it, rr, ok = F.solve(an, f, p.b, 1e-8)
    assert ok and rr <= 1e-8


@pytest.mark.parametrize("maker", [lambda: W.random_geometric(400, 0.16, seed=1), lambda: W.poisson7(7, 6, 5)])
def test_symbolic_closed_rows_graph_ordering(maker):
    """Graph ordering, whose separators and leaves need not be elimination-tree chains:
    R_j contains the brute-force union of the column structures, keeps the Section 2.1
    property (R_k after C_j inside R_j for every k in D_j), and is the smallest such set:
    every extra row comes from a descendant's R_k.  The exact factor with this structure is
    the Cholesky factor (the extra rows are zeros)."""
    p = maker()
    X = p.coords + (0.0 if p.shape == () else 0.3 * np.random.default_rng(4).uniform(-1, 1, p.coords.shape))
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, X, F.Options(leaf_size=6, tau_O=10 ** 9, ordering=1))
    L = _brute_structure(an.Ap.toarray() != 0)
    sym = an.sym
    Ap = an.Ap.tocsc()
    strict = 0
    for j in range(an.nsuper):
        c0, c1 = an.cols(j)
        brute = set((np.nonzero(L[c1:, c0:c1].any(axis=1))[0] + c1).tolist())
        Rj = set(sym.rows[j].tolist())
        assert brute <= Rj
        strict += len(Rj - brute)
        a_part = set(r for p_ in range(c0, c1) for r in Ap.indices[Ap.indptr[p_]:Ap.indptr[p_ + 1]].tolist()
                     if r >= c1)
        from_desc = set()
        for k, pD, pO in sym.desc[j]:
            Rk = sym.rows[k]
            tail = set(Rk[Rk >= c1].tolist())
            assert tail <= Rj
            from_desc |= tail
        assert Rj == a_part | from_desc
    f = F.factor(an, 0.0)
    Lf = _assemble_L(f)
    Apd = an.Ap.toarray()
    assert np.linalg.norm(Lf @ Lf.T - Apd) / np.linalg.norm(Apd) <= 1e-13
    if p.shape == ():
        assert strict > 0        # this graph has non-chain supernodes: the closure adds rows


# --------------------------------------------------------------------------- interior blocks (Section 5.1)

@pytest.mark.parametrize("maker,kw", [
    (lambda: W.poisson7(10), dict(leaf_size=8, tau_O=24, tau_D=16)),
    (lambda: W.diffusion_grf(12, 2.0, 3.0, 0), dict(leaf_size=16, tau_O=40, tau_D=32)),
    (lambda: W.elasticity_q1(4, incl=(1, 3)), dict(leaf_size=8, tau_O=48, tau_D=24, dof_per_node=3)),
])
def test_interior_blocks_closed_form_and_apply(maker, kw):
    """Eq. interiorBlockClosedForm: an interior block's columns of the factor are untouched
    by compression, so A(X, C_B) L_B^{-T} equals the library Cholesky factor of the permuted
    matrix in those columns; the preconditioner with interior blocks equals the one that
    stores every block (ranks equal, apply within 1e-12, same PCG iterations), and it stores
    exactly the off-block entries c_j |R_j after C_B| fewer."""
    p = maker()
    an_s = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, F.Options(**kw))
    an_i = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, F.Options(interior_blocks=True, **kw))
    fs, fi = F.factor(an_s, 0.05), F.factor(an_i, 0.05)
    assert len(fi.iblocks) >= 2 and any(B["RB"].size for B in fi.iblocks)
    Lx = np.linalg.cholesky(an_i.Ap.toarray())
    saved = 0
    for b, B in enumerate(fi.iblocks):
        c0, c1 = B["c0"], B["c1"]
        rows = np.arange(c0, p.n)
        np.testing.assert_allclose(fi._ib_L(b, rows), Lx[c0:, c0:c1], atol=1e-12 * np.abs(Lx).max())
        for j in range(B["first"], B["last"] + 1):
            jc0, jc1 = an_i.cols(j)
            saved += (jc1 - jc0) * int(np.sum(an_i.sym.rows[j] >= c1))
    for j in range(an_s.nsuper):
        if fs.sn[j].compressed:
            assert fi.sn[j].compressed and fi.sn[j].U.shape[1] == fs.sn[j].U.shape[1], j
    r = np.random.default_rng(3).standard_normal(p.n)
    zs, zi = F.apply_preconditioner(fs, r), F.apply_preconditioner(fi, r)
    assert np.abs(zs - zi).max() <= 1e-12 * np.abs(zs).max()
    _, its, _, ok_s = F.solve(an_s, fs, p.b, 1e-8)
    _, iti, rr, ok_i = F.solve(an_i, fi, p.b, 1e-8)
    assert ok_s and ok_i and its == iti and rr <= 1e-8
    assert F.factor_bytes(fs) - F.factor_bytes(fi) == 8 * saved > 0


def test_interior_blocks_cover_the_uncompressed_subtrees():
    """Blocks are the maximal subtrees without a compressed supernode: contiguous, disjoint,
    every supernode outside them is compressed or has a compressed descendant."""
    p = W.poisson7(12)
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords,
                   F.Options(leaf_size=16, tau_O=40, tau_D=32, interior_blocks=True))
    f = F.factor(an, 0.1)
    parent = an.sym.parent
    ib = f.iblock_of
    for b, B in enumerate(f.iblocks):
        assert np.all(ib[B["first"]:B["last"] + 1] == b)
        assert parent[B["last"]] < 0 or ib[parent[B["last"]]] < 0
    comp_desc = np.array([f.is_compressed(j) for j in range(an.nsuper)])
    for j in range(an.nsuper):
        if parent[j] >= 0:
            comp_desc[parent[j]] |= comp_desc[j]
    assert np.array_equal(ib < 0, comp_desc)


# ----------------------------------------------------------------------------- relaxed amalgamation (Section 3.1)

from oracle.amalgamate import merge_ok  # noqa: E402

AMALG_CASES = [
    ("poisson10", lambda: W.poisson7(10), dict(leaf_size=8, tau_O=40, tau_D=32)),
    ("poisson_7x5x6", lambda: W.poisson7(7, 5, 6), dict(leaf_size=4, tau_O=12, tau_D=8)),
    ("rgg600", lambda: W.random_geometric(600, 0.16, seed=2), dict(leaf_size=12, tau_O=30, tau_D=16, ordering=1)),
]


def test_merge_rule_closed_form():
    """The relaxation thresholds (CHOLMOD's defaults): blocks of at most 4 columns always merge;
    up to 16 columns at most 80% new entries, up to 48 at most 10%, any size at most 5%."""
    assert merge_ok(2, 3, 2, 9, 9)                     # 4 columns, whatever the fill
    # 8 + 8 columns, rows 8 -> 8: s(L) = 36 + 64, s(G) = 36 + 64, s(M) = 136 + 128, z = 0.24
    assert merge_ok(8, 8, 8, 8, 8)
    # 24 + 24 columns into 30 rows: s(M) = 1176 + 1440 = 2616, s(L) + s(G) = 2 (300 + 720), z = 0.22
    assert not merge_ok(24, 30, 24, 30, 30)
    # 40 + 8 columns: s(L) = 820 + 40 * 48 = 2740, s(G) = 36 + 8 * 40 = 356, s(M) = 1176 + 48 * 40 = 3096
    assert merge_ok(40, 48, 8, 40, 40)                 # z = 0.0 <= 0.1 at 48 columns
    assert not merge_ok(40, 8, 9, 40, 40)              # 49 columns, z = 0.51


@pytest.mark.parametrize("name,maker,kw", AMALG_CASES, ids=[c[0] for c in AMALG_CASES])
def test_amalgamation_against_brute_force(name, maker, kw):
    """Merged supernodes: contiguous groups of the unmerged ones in which every member but the
    last has its supernodal parent inside the group; no compressed separator merged; fewer
    supernodes; every nonzero of the exact factor (dense Cholesky of P A P^T, brute force)
    inside the merged partition's stored blocks; the exact factor computed blockwise with the
    merged partition equals the dense factor (the Cholesky factor is unique)."""
    p = maker()
    a0 = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, F.Options(**kw))
    a1 = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, F.Options(amalgamate=True, **kw))
    assert np.array_equal(a0.ordering.perm, a1.ordering.perm)
    p0, p1 = a0.sym.snode_ptr, a1.sym.snode_ptr
    assert a1.nsuper < a0.nsuper and set(p1.tolist()) <= set(p0.tolist())
    for g in range(a1.nsuper):
        c0, c1 = int(p1[g]), int(p1[g + 1])
        members = [j for j in range(a0.nsuper) if c0 <= p0[j] < c1]
        for j in members[:-1]:
            assert a0.sym.parent[j] in members, (g, j)
        if len(members) > 1:
            assert not (a1.ordering.kinds[g] == "sep" and c1 - c0 >= kw["tau_O"])
            assert all(not (a0.ordering.kinds[j] == "sep" and p0[j + 1] - p0[j] >= kw["tau_O"]) for j in members)
    Ad = a1.Ap.toarray()
    Ld = np.linalg.cholesky(Ad)
    nz = np.abs(Ld) > 1e-14 * np.abs(Ld).max()
    for g in range(a1.nsuper):
        c0, c1 = int(p1[g]), int(p1[g + 1])
        allowed = np.zeros(p.n, bool)
        allowed[c0:c1] = True
        allowed[a1.sym.rows[g]] = True
        for c in range(c0, c1):
            rows = np.nonzero(nz[c:, c])[0] + c
            assert allowed[rows].all(), (g, c)
    f = F.factor(a1, 0.0)
    L = np.zeros_like(Ad)
    for g in range(a1.nsuper):
        c0, c1 = a1.cols(g)
        L[c0:c1, c0:c1] = f.sn[g].D.L
        if a1.sym.rows[g].size:
            L[np.ix_(a1.sym.rows[g], np.arange(c0, c1))] = f.sn[g].LO
    assert np.abs(L - Ld).max() <= 1e-12 * np.abs(Ld).max()
