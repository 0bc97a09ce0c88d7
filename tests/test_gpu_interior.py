"""GPU parity of interior blocks (Section 5.1) against the oracle's interior-block path.

An interior block's factor L_B = chol(A(C_B, C_B)) is exact, and every use of L(R_B, C_B)
goes through A(., C_B) L_B^{-T} on both sides (Eqs. interiorBlockClosedForm,
interiorBlockMult), so the tolerances are those of the stored-block parity tests: ranks
equal, compressed blocks and the in-block panels within 1e-8 (FP64), the preconditioner
within 1e-8 relative, PCG to 1e-8 within +-2 iterations of the oracle.  The stored factor
shrinks by exactly c_j x (rows of R_j after C_B) per interior supernode, the oracle's count.
"""
import numpy as np
import pytest

import paper_1507_05593_gb300 as R
import workloads as W
from oracle import factor as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    ("poisson10", lambda: W.poisson7(10), dict(leaf_size=8, tau_O=24, tau_D=16)),
    ("grf12", lambda: W.diffusion_grf(12, 2.0, 3.0, 0), dict(leaf_size=16, tau_O=40, tau_D=32)),
    ("elast4", lambda: W.elasticity_q1(4, incl=(1, 3)), dict(leaf_size=8, tau_O=48, tau_D=24, dof_per_node=3)),
    ("poisson20", lambda: W.poisson7(20), dict(leaf_size=32, tau_O=100, tau_D=64)),
]


def _oracle(p, kw, tol, interior):
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, F.Options(interior_blocks=interior, **kw))
    return an, F.factor(an, tol)


def _gpu(p, kw, tol, interior, **extra):
    o = R.rsc_options_default(interior_blocks=int(interior), **kw, **extra)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, o)
    R.rsc_factor(h, tol)
    return h


def _apply(h, r):
    d_r = torch.tensor(r, device="cuda")
    d_z = torch.empty_like(d_r)
    R.rsc_apply_preconditioner_device(h, d_r, d_z)
    return d_z.cpu().numpy()


@pytest.mark.parametrize("name,maker,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("tol", [0.1, 0.01])
def test_interior_blocks_parity(name, maker, kw, tol):
    p = maker()
    an, f = _oracle(p, kw, tol, True)
    assert f.iblocks and any(B["RB"].size for B in f.iblocks)
    h = _gpu(p, kw, tol, True)
    st = R.rsc_get_stats(h)
    assert st["restarts"] == f.restarts
    for j in range(an.nsuper):
        info = R.rsc_get_supernode_info(h, j)
        assert info["compressed"] == int(f.sn[j].compressed)
        LD, LO = R.rsc_get_supernode_blocks(h, j)
        b = int(f.iblock_of[j])
        if b >= 0:   # in-block rows of the panel: the exact factor L_B; the rest is not stored
            B = f.iblocks[b]
            c0, c1 = an.cols(j)
            L = B["L"]
            Lb = L[c0 - B["c0"]:, c0 - B["c0"]:c1 - B["c0"]]
            sc = max(1.0, np.abs(L).max())
            assert np.abs(np.tril(LD) - np.tril(Lb[:c1 - c0])).max() <= 1e-8 * sc, j
            Rj = an.sym.rows[j]
            rin = int(np.sum(Rj < B["c1"]))
            if rin:
                ref = Lb[Rj[:rin] - c0]
                assert np.abs(LO[:rin] - ref).max() <= 1e-8 * sc, j
            assert np.isnan(LO[rin:]).all()
            continue
        if f.sn[j].compressed:
            assert info["rank"] == f.sn[j].U.shape[1], j
            s = f.sn[j]
            LDo = s.D.L if not s.D.hierarchical else None
            if LDo is not None:
                assert np.abs(np.tril(LD) - np.tril(LDo)).max() <= 1e-8 * max(1.0, np.abs(LDo).max()), j
            if s.V.size:
                LOo = s.V @ s.U.T
                assert np.abs(LO - LOo).max() <= 1e-8 * max(1.0, np.abs(LOo).max()), j
    r = np.random.default_rng(5).standard_normal(p.n)
    z_ref = F.apply_preconditioner(f, r)
    z = _apply(h, r)
    assert np.abs(z - z_ref).max() <= 1e-8 * np.abs(z_ref).max()
    x, it, rr = R.rsc_solve(h, p.b, 1e-8, 500)
    _, it_ref, rr_ref, ok = F.solve(an, f, p.b, 1e-8, 500)
    assert ok and rr <= 1e-8 and abs(it - it_ref) <= 2
    A = p.scipy()
    assert np.linalg.norm(p.b - A @ x) / np.linalg.norm(p.b) <= 1e-8


@pytest.mark.parametrize("name,maker,kw", CASES[:2], ids=[c[0] for c in CASES[:2]])
def test_interior_blocks_save_the_off_block_rows(name, maker, kw):
    """With and without interior blocks on the GPU: the same ranks and preconditioner (within
    1e-8), and the stored factor smaller by exactly the off-block panel entries."""
    p = maker()
    tol = 0.05
    hs, hi = _gpu(p, kw, tol, False), _gpu(p, kw, tol, True)
    an, f = _oracle(p, kw, tol, True)
    saved = 0
    for B in f.iblocks:
        for j in range(B["first"], B["last"] + 1):
            c0, c1 = an.cols(j)
            saved += (c1 - c0) * int(np.sum(an.sym.rows[j] >= B["c1"]))
    assert saved > 0
    ss, si = R.rsc_get_stats(hs), R.rsc_get_stats(hi)
    assert ss["factor_bytes"] - si["factor_bytes"] == 8 * saved
    for j in range(an.nsuper):
        a, b = R.rsc_get_supernode_info(hs, j), R.rsc_get_supernode_info(hi, j)
        assert a["rank"] == b["rank"], j
    r = np.random.default_rng(7).standard_normal(p.n)
    zs, zi = _apply(hs, r), _apply(hi, r)
    assert np.abs(zs - zi).max() <= 1e-8 * np.abs(zs).max()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_interior_blocks_mixed_forms(prec):
    """The FP32 and BF16 forms with interior blocks: the ranks of the FP64 oracle's
    interior-block path, the preconditioner within the form's tolerance, PCG to 1e-8."""
    name, maker, kw = CASES[1]
    p = maker()
    an, f = _oracle(p, kw, 0.01, True)
    h = _gpu(p, kw, 0.01, True, precision=prec)
    for j in range(an.nsuper):
        if f.sn[j].compressed:
            assert R.rsc_get_supernode_info(h, j)["rank"] == f.sn[j].U.shape[1], j
    r = np.random.default_rng(9).standard_normal(p.n)
    z_ref = F.apply_preconditioner(f, r)
    z = _apply(h, r)
    bound = {"fp32": 1e-4, "bf16": 1e-2}[prec]
    assert np.abs(z - z_ref).max() <= bound * np.abs(z_ref).max()
    x, it, rr = R.rsc_solve(h, p.b, 1e-8, 500)
    assert rr <= 1e-8


def test_interior_blocks_multi_rhs_and_exact_mode():
    """Several right-hand sides at once (the N-column apply) match one at a time; with
    compression off the whole tree is one interior block per root and the factor is the
    exact Cholesky factor."""
    name, maker, kw = CASES[0]
    p = maker()
    h = _gpu(p, kw, 0.1, True)
    rng = np.random.default_rng(11)
    Bm = rng.standard_normal((4, p.n))
    d_B = torch.tensor(Bm, device="cuda")
    d_X = torch.zeros_like(d_B)
    its, rrs = R.rsc_solve_batch_device(h, d_B, d_X, 1e-8, 500)
    X = d_X.cpu().numpy()
    A = p.scipy()
    for c in range(4):
        x1, it1, rr1 = R.rsc_solve(h, Bm[c], 1e-8, 500)
        assert abs(int(its[c, 0]) - it1) <= 1 and rrs[c, 0] <= 1e-8
        assert np.linalg.norm(Bm[c] - A @ X[c]) <= 1e-8 * np.linalg.norm(Bm[c])
    h0 = _gpu(p, kw, 0.0, True)
    x, it, rr = R.rsc_solve(h0, p.b, 1e-10, 5)
    assert it <= 2 and rr <= 1e-10


def test_interior_blocks_refused_by_the_allocation_free_apply():
    name, maker, kw = CASES[0]
    p = maker()
    h = _gpu(p, kw, 0.1, True)
    d_r = torch.tensor(p.b, device="cuda")
    d_z = torch.empty_like(d_r)
    with pytest.raises(R.RscError) as e:
        R.rsc_apply_preconditioner_device_noalloc(h, d_r, d_z)
    assert e.value.status == 1
