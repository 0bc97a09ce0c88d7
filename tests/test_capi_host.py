"""Host-side tests of the C-ABI library (no GPU): exported symbols, input
validation and bit-exact symbolic parity with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1507_05593_gb300 as R
import workloads as W
from oracle import factor as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "rsc.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(rsc_\w+)\s*\(", txt, re.M)))


def test_library_exports_every_declared_symbol():
    names = _declared_symbols()
    assert "rsc_analyze" in names and "rsc_factor" in names and "rsc_solve" in names
    lib = ctypes.CDLL(R.LIB_PATH)
    for nm in names:
        assert hasattr(lib, nm), nm


def test_options_default_values():
    o = R.rsc_options_default()
    assert (o.tau_O, o.tau_D, o.leaf_size, o.sample_block, o.power_iters, o.dof_per_node) == (256, 256, 64, 16, 0, 1)
    assert (o.max_restarts, o.precision, o.diag_compress, o.seed) == (8, 0, 1, 0)
    assert (o.amalgamate, o.interior_blocks) == (0, 0)


def _bad(p, **changes):
    rp, ci, v, xyz = p.row_ptr.copy(), p.col_idx.copy(), p.val.copy(), p.coords.copy()
    loc = dict(rp=rp, ci=ci, v=v, xyz=xyz)
    for k, f in changes.items():
        loc[k] = f(loc[k])
    return loc


@pytest.mark.parametrize("what", ["asym", "unsorted", "nodiag", "nan", "badordering", "dof", "range", "hugecoord",
                                  "badinterior"])
def test_analyze_rejects_bad_input(what):
    p = W.poisson7(4)
    rp, ci, v, xyz = p.row_ptr.copy(), p.col_idx.copy(), p.val.copy(), p.coords.copy()
    opts = R.rsc_options_default()
    n = p.n
    if what == "asym":      # drop one off-diagonal entry of row 0
        keep = np.ones(ci.size, bool)
        keep[1] = False
        ci, v = ci[keep], v[keep]
        rp = rp.copy()
        rp[1:] -= 1
    elif what == "unsorted":
        ci[[0, 1]] = ci[[1, 0]]
    elif what == "nodiag":
        ci, v = ci.copy(), v.copy()
        d = np.nonzero(ci[rp[0]:rp[1]] == 0)[0][0]
        ci[d] = 63
    elif what == "nan":
        v[5] = np.nan
    elif what == "badordering":
        opts.ordering = 2
    elif what == "dof":
        opts.dof_per_node = 5
    elif what == "range":
        ci[3] = 10_000
    elif what == "hugecoord":
        xyz[5, 0] = 1e12
    elif what == "badinterior":
        opts.interior_blocks = 2
    with pytest.raises(R.RscError) as e:
        R.rsc_analyze(n, rp, ci, v, xyz, opts)
    assert e.value.status == 1
    assert R.rsc_last_error()


def _oracle_opts(o):
    return F.Options(tau_O=o.tau_O, tau_D=o.tau_D, leaf_size=o.leaf_size, dof_per_node=o.dof_per_node,
                     ordering=o.ordering, amalgamate=bool(o.amalgamate))


@pytest.mark.parametrize("maker,kw", [
    (lambda: W.poisson7(6), dict(leaf_size=8)),
    (lambda: W.poisson7(5, 7, 4), dict(leaf_size=8)),
    (lambda: W.poisson7(12), dict(leaf_size=16, tau_O=40, tau_D=32)),
    (lambda: W.poisson7(32), dict()),
    (lambda: W.elasticity_q1(3, incl=(1, 2)), dict(leaf_size=8, dof_per_node=3)),
    (lambda: W.elasticity_q1(8), dict(dof_per_node=3)),
    (lambda: W.diffusion_grf(20, 2.0, 4.0, 1), dict(leaf_size=32, tau_O=64, tau_D=64)),
    # relaxed amalgamation (Section 3.1) on lattice and graph orderings, scalar and 3-DOF nodes
    (lambda: W.poisson7(12), dict(leaf_size=8, tau_O=40, tau_D=32, amalgamate=1)),
    (lambda: W.poisson7(7, 5, 6), dict(leaf_size=4, tau_O=12, tau_D=8, amalgamate=1)),
    (lambda: W.poisson7(32), dict(amalgamate=1)),
    (lambda: W.elasticity_q1(4, incl=(1, 3)), dict(leaf_size=4, tau_O=48, tau_D=24, dof_per_node=3, amalgamate=1)),
    (lambda: W.random_geometric(1500, 0.12, seed=0), dict(leaf_size=16, tau_O=40, tau_D=32, ordering=1,
                                                          amalgamate=1)),
])
def test_symbolic_bit_exact_vs_oracle(maker, kw):
    p = maker()
    o = R.rsc_options_default(**kw)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, o)
    perm, sp = R.rsc_get_ordering(h)
    rows_ptr, rows, parent, level, kind = R.rsc_get_structure(h)
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, _oracle_opts(o))
    np.testing.assert_array_equal(perm, an.ordering.perm)
    np.testing.assert_array_equal(sp, an.ordering.snode_ptr)
    for j in range(an.nsuper):
        np.testing.assert_array_equal(rows[rows_ptr[j]:rows_ptr[j + 1]], an.sym.rows[j])
    np.testing.assert_array_equal(parent, an.sym.parent)
    assert [int(k) for k in kind] == [1 if x == "sep" else 0 for x in an.ordering.kinds]
    if kw.get("amalgamate"):   # never more supernodes than without (fewer where small ones exist)
        assert an.nsuper <= F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords,
                                     _oracle_opts(R.rsc_options_default(**dict(kw, amalgamate=0)))).nsuper
    # levels: children strictly below parents, leaves at 0
    for j in range(an.nsuper):
        if parent[j] >= 0:
            assert level[parent[j]] > level[j]


def test_symbolic_properties_full_size():
    """96^3 (884,736 unknowns): properties that hold at any size."""
    p = W.poisson7(96)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, R.rsc_options_default())
    perm, sp = R.rsc_get_ordering(h)
    rows_ptr, rows, parent, level, kind = R.rsc_get_structure(h)
    assert np.array_equal(np.sort(perm), np.arange(p.n))
    M = sp.size - 1
    c = np.diff(sp)
    assert c.max() == 96 * 96 and kind[-1] == 1 and parent[-1] == -1
    assert ((kind == 1) & (c >= 256)).sum() == 165
    snode_of = np.repeat(np.arange(M), c)
    iperm = np.empty_like(perm)
    iperm[perm] = np.arange(p.n)
    # every entry of A below the diagonal block lies in R_j of its column's supernode
    A = p.scipy().tocoo()
    r, cc = iperm[A.row], iperm[A.col]
    low = r > cc
    r, cc = r[low], cc[low]
    j = snode_of[cc]
    outside = r >= sp[j + 1]
    for jj, rr in zip(j[outside][::997], r[outside][::997]):
        R_j = rows[rows_ptr[jj]:rows_ptr[jj + 1]]
        assert R_j[np.searchsorted(R_j, rr)] == rr
    # R_k meets C^O_j only inside R_j for j = parent(k) (Section 2.1)
    for k in range(0, M, 97):
        pk = parent[k]
        if pk < 0:
            continue
        Rk = rows[rows_ptr[k]:rows_ptr[k + 1]]
        tail = Rk[Rk >= sp[pk + 1]]
        Rp = rows[rows_ptr[pk]:rows_ptr[pk + 1]]
        assert np.all(np.isin(tail, Rp))


@pytest.mark.parametrize("args", [(-1.0, 0.5, 8), (1.0, float("nan"), 8), (1.0, 0.5, -1), (float("inf"), 0.5, 4)])
def test_factor_fixed_rank_rejects_bad_parameters(args):
    """rsc_factor_fixed_rank checks alpha_O, alpha_D and p on the host, before any GPU work."""
    p = W.poisson7(4)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, R.rsc_options_default())
    with pytest.raises(R.RscError) as e:
        R.rsc_factor_fixed_rank(h, *args)
    assert e.value.status == 1 and "alpha" in R.rsc_last_error(h)


# ----------------------------------------------------------------------------- graph ordering

def _jittered(p, seed=3):
    X = p.coords + 0.3 * np.random.default_rng(seed).uniform(-1, 1, p.coords.shape)
    return X if p.dof_per_node == 1 else np.repeat(X[::p.dof_per_node], p.dof_per_node, axis=0)


@pytest.mark.parametrize("maker,kw,pos", [
    (lambda: W.poisson7(8), dict(leaf_size=8, tau_O=24, tau_D=16), "lattice"),
    (lambda: W.poisson7(12), dict(leaf_size=16, tau_O=40, tau_D=32), "jitter"),
    (lambda: W.elasticity_q1(4, incl=(1, 3)), dict(leaf_size=8, tau_O=48, tau_D=24, dof_per_node=3), "jitter"),
    (lambda: W.random_geometric(1500, 0.12, seed=2), dict(leaf_size=24, tau_O=60, tau_D=40), "points"),
    (lambda: W.diffusion_grf(20, 2.0, 4.0, 1), dict(leaf_size=32, tau_O=64, tau_D=64), "jitter"),
])
def test_graph_ordering_bit_exact_vs_oracle(maker, kw, pos):
    """Graph nested dissection (ordering 1) with the same real positions on both sides:
    permutation, supernodes, row structures, tree and kinds equal the oracle's bit for bit,
    block trees included."""
    p = maker()
    X = _jittered(p) if pos == "jitter" else p.coords
    o = R.rsc_options_default(ordering=1, **kw)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, X, o)
    perm, sp = R.rsc_get_ordering(h)
    rows_ptr, rows, parent, level, kind = R.rsc_get_structure(h)
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, X, _oracle_opts(o))
    np.testing.assert_array_equal(perm, an.ordering.perm)
    np.testing.assert_array_equal(sp, an.ordering.snode_ptr)
    for j in range(an.nsuper):
        np.testing.assert_array_equal(rows[rows_ptr[j]:rows_ptr[j + 1]], an.sym.rows[j])
    np.testing.assert_array_equal(parent, an.sym.parent)
    assert [int(k) for k in kind] == [1 if x == "sep" else 0 for x in an.ordering.kinds]
    if kw.get("amalgamate"):   # never more supernodes than without (fewer where small ones exist)
        assert an.nsuper <= F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords,
                                     _oracle_opts(R.rsc_options_default(**dict(kw, amalgamate=0)))).nsuper
    np.testing.assert_array_equal(R.rsc_get_coordinates(h), X[::p.dof_per_node])
    assert any(t is not None for t in an.ordering.trees)


def _proj(V):
    Q, _ = np.linalg.qr(V)
    return Q @ Q.T


def test_spectral_positions_small_graph_equal_oracle():
    """No coordinates, 6 x 5 x 4 grid (120 nodes, so the Lanczos run spans the whole space
    orthogonal to the constant vector): the three positions span the oracle's eigenvectors of
    the Laplacian (eigenvalues 0.268, 0.382, 0.586 against 0.650 next, non-degenerate) to
    rounding, each column orthogonal to the constant vector."""
    from oracle.ordering import node_graph, spectral_coordinates
    p = W.poisson7(6, 5, 4)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, None, R.rsc_options_default(leaf_size=8))
    X = R.rsc_get_coordinates(h)
    ptr, idx = node_graph(p.n, p.row_ptr, p.col_idx)
    Xo = spectral_coordinates(ptr, idx)
    for c in range(3):
        assert abs(abs(X[:, c] @ Xo[:, c]) / np.linalg.norm(X[:, c]) - 1.0) <= 1e-9
    assert np.abs(X.sum(axis=0)).max() <= 1e-10
    perm, _ = R.rsc_get_ordering(h)
    assert np.array_equal(np.sort(perm), np.arange(p.n))


@pytest.mark.parametrize("maker", [lambda: W.poisson7(14, 12, 10), lambda: W.random_geometric(2500, 0.1, seed=5)])
def test_spectral_positions_larger_graph_are_low_modes(maker):
    """Larger graphs (the Lanczos run stops at 160 steps): the positions are orthonormal,
    orthogonal to the constant vector, and their Rayleigh quotients lie within 5% of the
    three lowest non-zero Laplacian eigenvalues (dense reference); the ordering they guide
    is a valid permutation whose separators the analysis accepts."""
    from oracle.ordering import node_graph
    p = maker()
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, None, R.rsc_options_default(leaf_size=16))
    X = R.rsc_get_coordinates(h)
    ptr, idx = node_graph(p.n, p.row_ptr, p.col_idx)
    n = p.n
    import scipy.sparse as sp_
    Adj = sp_.csr_matrix((np.ones(idx.size), idx, ptr), shape=(n, n))
    Lap = sp_.diags(np.asarray(Adj.sum(axis=1)).ravel()) - Adj
    comps = sp_.csgraph.connected_components(Adj, directed=False)[0]
    w = np.linalg.eigvalsh(Lap.toarray())
    lam = w[comps:comps + 3]
    np.testing.assert_allclose(X.T @ X, np.eye(3), atol=1e-8)
    if comps == 1:
        assert np.abs(X.sum(axis=0)).max() <= 1e-8
        rq = np.sort(np.einsum("ic,ic->c", X, Lap @ X))
        assert np.all(np.abs(rq - lam) <= 0.05 * lam), (rq, lam)
    perm, _ = R.rsc_get_ordering(h)
    assert np.array_equal(np.sort(perm), np.arange(n))


def test_graph_ordering_disconnected_and_tiny_components():
    """A stack of two grids, an isolated node and 2- and 3-node paths: with shared positions
    the graph ordering is bit-exact vs the oracle; without positions every component gets
    its own spectral positions (a single node at 0, a 2-node path +-1/sqrt 2 on one axis),
    equal to the oracle's up to sign per column."""
    import scipy.sparse as sp_
    from oracle.ordering import node_graph, spectral_coordinates
    a, b = W.poisson7(5), W.poisson7(4, 3, 2)
    blocks = [a.scipy(), sp_.csr_matrix(np.array([[2.0]])), b.scipy(),
              sp_.csr_matrix(np.array([[2.0, -1.0], [-1.0, 2.0]])),
              sp_.csr_matrix(np.array([[2.0, -1.0, 0.0], [-1.0, 2.0, -1.0], [0.0, -1.0, 2.0]]))]
    A = sp_.block_diag(blocks).tocsr()
    A.sort_indices()
    n = A.shape[0]
    Xg = np.random.default_rng(0).uniform(size=(n, 3))
    h = R.rsc_analyze(n, A.indptr, A.indices, A.data, Xg, R.rsc_options_default(leaf_size=4, ordering=1))
    an = F.analyze(n, A.indptr, A.indices, A.data, Xg, F.Options(leaf_size=4, ordering=1))
    np.testing.assert_array_equal(R.rsc_get_ordering(h)[0], an.ordering.perm)
    h = R.rsc_analyze(n, A.indptr, A.indices, A.data, None, R.rsc_options_default(leaf_size=4))
    X = R.rsc_get_coordinates(h)
    ptr, idx = node_graph(n, A.indptr, A.indices)
    comp = np.repeat(np.arange(5), [m.shape[0] for m in blocks])
    Xo = spectral_coordinates(ptr, idx, comp)
    for c in range(5):            # the subspace is unique (the 5^3 cube's 3 modes share one eigenvalue)
        sel = comp == c
        k = min(3, int(sel.sum()) - 1)
        if k <= 0:
            continue
        assert np.abs(_proj(X[sel, :k]) - _proj(Xo[sel, :k])).max() <= 1e-9, c
    assert X[a.n, :].tolist() == [0.0, 0.0, 0.0]
    perm, _ = R.rsc_get_ordering(h)
    assert np.array_equal(np.sort(perm), np.arange(n))


def test_no_gpu_fails_loudly():
    """Without a usable GPU the numeric calls return RSC_ERR_CUDA with a message and leave
    the handle unfactored (a later solve is RSC_ERR_STATE): there is no CPU fallback."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = W.poisson7(4)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, R.rsc_options_default())
    for call in (lambda: R.rsc_factor(h, 0.1), lambda: R.rsc_factor_fixed_rank(h, 0.5)):
        with pytest.raises(R.RscError) as e:
            call()
        assert e.value.status == 5 and "CUDA" in str(e.value)
    with pytest.raises(R.RscError) as e:
        R.rsc_solve(h, p.b)
    assert e.value.status == 7
