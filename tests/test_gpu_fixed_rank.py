"""GPU parity of the fixed-rank form (Section 5.2, Eq. rankFunction) against the oracle.

Both sides draw the same Philox samples in 16-column passes with the stopping test
off, so the ranks and the Section 5.3 restart counts are equal (integers, exact).
The bases U span orth((B^T B)^q B^T G).  A singular direction of B at s = sigma/sigma_1
enters Y = (B^T B)^q B^T G with weight s^(2q+1), so rounding (unit u) fixes it only to
u s^-(2q+1) relative and moves B U U^T along it by at most min(s, u s^-2q) of ||B||;
that is largest, u^(1/(2q+1)), at s = u^(1/(2q+1)).  The FP64 tolerance on blocks is
max(1e-8, 10 u^(1/(2q+1))): 1e-8, 4.8e-5 and 6.6e-3 for q = 0, 1, 2.  One preconditioner
application z = P (L L^T)^-1 P^T r is checked by its componentwise backward error against
the oracle's factor, ||L L^T z' - r'|| / || |L| |L|^T |z'| || (z' = P^T z), within the same
tolerance; the forward error of z also grows with the factor's condition number (3% at
q = 2 on the elasticity problem with its stiff inclusion), so z is compared element by
element only for q <= 1.  PCG reaches 1e-8 with iteration counts within +-2 of the
oracle's.
"""
import numpy as np
import pytest

import paper_1507_05593_gb300 as R
import workloads as W
from oracle import factor as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64 = 1.1102230246251565e-16

CASES = [
    ("poisson8", lambda: W.poisson7(8), dict(leaf_size=8, tau_O=16, tau_D=8)),
    ("grf12", lambda: W.diffusion_grf(12, 2.0, 3.0, 0), dict(leaf_size=16, tau_O=40, tau_D=32)),
    ("elast4", lambda: W.elasticity_q1(4, incl=(1, 3)), dict(leaf_size=8, tau_O=48, tau_D=24, dof_per_node=3)),
    ("poisson20", lambda: W.poisson7(20), dict(leaf_size=32, tau_O=100, tau_D=64)),
]


def _oracle_fixed(p, o, aO, aD, ov):
    oo = F.Options(tau_O=o.tau_O, tau_D=o.tau_D, leaf_size=o.leaf_size, dof_per_node=o.dof_per_node,
                   power_iters=o.power_iters, max_restarts=o.max_restarts, seed=o.seed,
                   diag_compress=bool(o.diag_compress))
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, oo)
    return an, F.factor_fixed_rank(an, aO, aD, ov)


def _blocks(f, j):
    an = f.an
    s = f.sn[j]
    D = s.D
    c0, c1 = an.cols(j)
    if D.hierarchical:
        t = D.tree
        LD = np.zeros((c1 - c0, c1 - c0))
        for b in range(1, t.nblocks + 1):
            r0, r1 = t.rows(b)
            q0, q1 = t.cols(b)
            LD[r0:r1, q0:q1] = D.leafL[b] if t.leaf[b] else D.V[b] @ D.U[b].T
    else:
        LD = D.L
    if an.sym.rows[j].size == 0:
        LO = np.zeros((0, c1 - c0))
    else:
        LO = s.V @ s.U.T if s.compressed else s.LO
    return LD, LO


def _llt(f, x, absval):
    """L L^T x (absval: |L| |L|^T x) over the oracle's blocks, in the permuted order."""
    an = f.an
    y = np.zeros_like(x)
    w = np.zeros_like(x)
    bl = [_blocks(f, j) for j in range(an.nsuper)]
    if absval:
        bl = [(np.abs(a), np.abs(b)) for a, b in bl]
    for j, (LD, LO) in enumerate(bl):
        c0, c1 = an.cols(j)
        Rj = an.sym.rows[j]
        y[c0:c1] = LD.T @ x[c0:c1] + (LO.T @ x[Rj] if Rj.size else 0.0)
    for j, (LD, LO) in enumerate(bl):
        c0, c1 = an.cols(j)
        Rj = an.sym.rows[j]
        w[c0:c1] += LD @ y[c0:c1]
        if Rj.size:
            w[Rj] += LO @ y[c0:c1]
    return w


def _check(p, o, h, an, f, tol, forward=True):
    st = R.rsc_get_stats(h)
    assert st["restarts"] == f.restarts
    worst = 0.0
    for j in range(an.nsuper):
        info = R.rsc_get_supernode_info(h, j)
        assert info["compressed"] == int(f.sn[j].compressed), j
        if f.sn[j].compressed:
            assert info["rank"] == f.sn[j].U.shape[1], j
        LD, LO = R.rsc_get_supernode_blocks(h, j)
        LDo, LOo = _blocks(f, j)
        sc = max(1.0, np.abs(LDo).max())
        worst = max(worst, np.abs(np.tril(LD) - np.tril(LDo)).max() / sc)
        if LOo.size:
            worst = max(worst, np.abs(LO - LOo).max() / max(1.0, np.abs(LOo).max()))
    assert worst <= tol, (worst, tol)
    r = np.random.default_rng(8).standard_normal(p.n)
    z_ref = F.apply_preconditioner(f, r)
    d_r = torch.tensor(r, device="cuda")
    d_z = torch.empty_like(d_r)
    R.rsc_apply_preconditioner_device(h, d_r, d_z)
    z = d_z.cpu().numpy()
    perm = an.ordering.perm
    zp = z[perm]
    eta = np.linalg.norm(_llt(f, zp, False) - r[perm]) / np.linalg.norm(_llt(f, np.abs(zp), True))
    assert eta <= tol, (eta, tol)
    if forward:
        assert np.abs(z - z_ref).max() <= tol * np.abs(z_ref).max()
    x, it, rr = R.rsc_solve(h, p.b, 1e-8, 500)
    _, it_ref, rr_ref, ok = F.solve(an, f, p.b, 1e-8, 500)
    assert ok and rr <= 1e-8 and abs(it - it_ref) <= 2, (it, it_ref)
    A = p.scipy()
    assert np.linalg.norm(p.b - A @ x) / np.linalg.norm(p.b) <= 1e-8
    return worst


@pytest.mark.parametrize("name,maker,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("q", [0, 1, 2])
def test_fixed_rank_parity(name, maker, kw, q):
    """Ranks, restarts and compressed flags equal; blocks and the backward error of one
    preconditioner application within max(1e-8, 10 u^(1/(2q+1))), z itself for q <= 1;
    PCG iterations within +-2."""
    p = maker()
    o = R.rsc_options_default(power_iters=q, **kw)
    aO, aD, ov = 0.5, 0.4, 4
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, o)
    R.rsc_factor_fixed_rank(h, aO, aD, ov)
    an, f = _oracle_fixed(p, o, aO, aD, ov)
    assert any(s.compressed for s in f.sn)
    tol = max(1e-8, 10 * U64 ** (1.0 / (2 * q + 1)))
    _check(p, o, h, an, f, tol, forward=q <= 1)


def test_fixed_rank_full_rank_matches_exact_factor():
    """alpha large enough that every rank reaches min(m, n): the fixed-rank factor is the
    exact factor, within 1e-12 of the uncompressed GPU factor's largest entry."""
    p = W.poisson7(12)
    kw = dict(leaf_size=16, tau_O=40, tau_D=32)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, R.rsc_options_default(**kw))
    R.rsc_factor_fixed_rank(h, 100.0, 100.0, 0)
    he = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, R.rsc_options_default(**kw))
    R.rsc_factor(he, 0.0)
    st = R.rsc_get_stats(h)
    assert st["n_compressed"] >= 1
    M = st["n_supernodes"]
    scale = max(np.abs(R.rsc_get_supernode_blocks(he, j)[0]).max() for j in range(M))
    for j in range(M):
        LD, LO = R.rsc_get_supernode_blocks(h, j)
        LDe, LOe = R.rsc_get_supernode_blocks(he, j)
        assert np.abs(np.tril(LD) - np.tril(LDe)).max() <= 1e-12 * scale, j
        if LOe.size:
            assert np.abs(LO - LOe).max() <= 1e-12 * scale, j
    x, it, rr = R.rsc_solve(h, p.b, 1e-8, 10)
    assert it <= 2 and rr <= 1e-8


def test_fixed_rank_poisson32_defaults():
    """32^3 Poisson with tau_O = tau_D = 256 and the defaults alpha^O = alpha^D = 0.5, p = 8
    (RSC0) and one power iteration (RSC1): ranks equal the oracle's and PCG iteration
    counts are within +-2."""
    p = W.poisson7(32)
    for q in (0, 1):
        o = R.rsc_options_default(power_iters=q)
        h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, o)
        R.rsc_factor_fixed_rank(h, 0.5, 0.5, 8)
        an, f = _oracle_fixed(p, o, 0.5, 0.5, 8)
        for j in range(an.nsuper):
            if f.sn[j].compressed:
                assert R.rsc_get_supernode_info(h, j)["rank"] == f.sn[j].U.shape[1], (q, j)
        x, it, rr = R.rsc_solve(h, p.b, 1e-8, 500)
        _, it_ref, _, _ = F.solve(an, f, p.b, 1e-8, 500)
        assert rr <= 1e-8 and abs(it - it_ref) <= 2, (q, it, it_ref)


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
def test_fixed_rank_mixed_precision(prec):
    """FP32, TF32 and BF16 forms with fixed ranks: ranks equal the FP64 oracle's (the cap
    decides them, not a rounding-sensitive test), blocks within the forms' rounding (1e-4
    FP32 and split TF32, 3e-2 BF16 operands of the Schur updates), PCG to 1e-8."""
    p = W.diffusion_grf(12, 2.0, 3.0, 0)
    kw = dict(leaf_size=16, tau_O=40, tau_D=32)
    o = R.rsc_options_default(precision=prec, **kw)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, o)
    R.rsc_factor_fixed_rank(h, 0.5, 0.5, 8)
    an, f = _oracle_fixed(p, R.rsc_options_default(**kw), 0.5, 0.5, 8)
    tol_blk = {"fp32": 1e-4, "tf32": 1e-4, "bf16": 3e-2}[prec]
    for j in range(an.nsuper):
        if f.sn[j].compressed:
            assert R.rsc_get_supernode_info(h, j)["rank"] == f.sn[j].U.shape[1], j
        LD, _ = R.rsc_get_supernode_blocks(h, j)
        LDo, _ = _blocks(f, j)
        assert np.abs(np.tril(LD) - np.tril(LDo)).max() <= tol_blk * max(1, np.abs(LDo).max()), j
    x, it, rr = R.rsc_solve(h, p.b, 1e-8, 500)
    _, it_ref, _, _ = F.solve(an, f, p.b, 1e-8, 500)
    assert rr <= 1e-8 and it <= it_ref + {"fp32": 3, "tf32": 3, "bf16": 10}[prec]
