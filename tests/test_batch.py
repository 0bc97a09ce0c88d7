"""Batching form: independent systems stacked block-diagonally are analysed as a forest
(one nested dissection per connected component), factored level by level together,
and solved by per-(system, right-hand side) PCG recurrences."""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_1507_05593_gb300 as R
import workloads as W
from oracle import factor as F


def stack(problems, gap=3):
    A = sp.block_diag([p.scipy() for p in problems]).tocsr()
    A.sort_indices()
    coords, off = [], 0
    for p in problems:
        c = p.coords.copy()
        c[:, 0] += off
        off += int(c[:, 0].max() - c[:, 0].min()) + 1 + gap
        coords.append(c)
    return A, np.vstack(coords)


def test_forest_symbolic_matches_oracle_per_system():
    ps = [W.diffusion_lognormal(s, 1.0, seed=i) for i, s in enumerate([7, 9, 6, 8])]
    A, coords = stack(ps)
    kw = dict(leaf_size=16, tau_O=24, tau_D=16)
    h = R.rsc_analyze(A.shape[0], A.indptr, A.indices, A.data, coords, R.rsc_options_default(**kw))
    ptr = R.rsc_get_systems(h)
    assert ptr.tolist() == np.concatenate([[0], np.cumsum([p.n for p in ps])]).tolist()
    perm, snp = R.rsc_get_ordering(h)
    rows_ptr, rows, parent, level, kind = R.rsc_get_structure(h)
    assert (parent < 0).sum() == len(ps)
    an = F.analyze(A.shape[0], A.indptr, A.indices, A.data, coords, F.Options(**kw))
    np.testing.assert_array_equal(perm, an.ordering.perm)
    np.testing.assert_array_equal(snp, an.ordering.snode_ptr)
    # each system alone orders its unknowns the same way (shifted)
    off, m0 = 0, 0
    for p in ps:
        an1 = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, F.Options(**kw))
        np.testing.assert_array_equal(perm[off:off + p.n], an1.ordering.perm + off)
        off += p.n


def test_noncontiguous_systems_rejected():
    ps = [W.poisson7(4), W.poisson7(3)]
    A, coords = stack(ps)
    q = np.r_[np.arange(0, A.shape[0], 2), np.arange(1, A.shape[0], 2)]   # interleave the systems
    B = A[q][:, q].tocsr()
    B.sort_indices()
    h = R.rsc_analyze(B.shape[0], B.indptr, B.indices, B.data, coords[q], R.rsc_options_default(leaf_size=8))
    with pytest.raises(R.RscError) as e:
        R.rsc_get_systems(h)
    assert e.value.status == 1


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_solve_per_system(prec):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    sides = rng.integers(6, 13, 6)
    ps = [W.diffusion_lognormal(int(s), 1.0, seed=i) for i, s in enumerate(sides)]
    A, coords = stack(ps)
    n = A.shape[0]
    kw = dict(leaf_size=16, tau_O=40, tau_D=32)
    h = R.rsc_analyze(n, A.indptr, A.indices, A.data, coords, R.rsc_options_default(precision=prec, **kw))
    R.rsc_factor(h, 0.1)
    nrhs = 3
    B = np.stack([W.rhs_uniform(n, seed=100 + c) for c in range(nrhs)])
    dB = torch.tensor(B, device="cuda")
    dX = torch.empty_like(dB)
    its, rr = R.rsc_solve_batch_device(h, dB, dX, 1e-8, 500)
    X = dX.cpu().numpy()
    ptr = R.rsc_get_systems(h)
    for c in range(nrhs):
        for s, p in enumerate(ps):
            lo, hi = ptr[s], ptr[s + 1]
            Ai = A[lo:hi][:, lo:hi]
            res = np.linalg.norm(B[c, lo:hi] - Ai @ X[c, lo:hi]) / np.linalg.norm(B[c, lo:hi])
            assert res <= 1e-8 and rr[c, s] <= 1e-8
            if c == 0:   # iteration counts close to the oracle solving this system alone
                an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, F.Options(**kw))
                f = F.factor(an, 0.1)
                _, it_ref, _, ok = F.solve(an, f, B[c, lo:hi], 1e-8, 500)
                assert ok and abs(int(its[c, s]) - it_ref) <= 2, (s, its[c, s], it_ref)
