"""GPU parity of the indefinite restart of Section 5.3 against the oracle.

A diagonal block whose hierarchical compression (Section 4) is too rough can leave an
indefinite Schur complement for the supernodes above it; the factorization then starts
again with more accurate diagonal blocks (tolerance form: tol_D <- tol_D / 1.25; fixed-rank
form: alpha_D <- 1.25 alpha_D), and after max_restarts restarts switches diagonal
compression off.  Every attempt draws its Gaussian test matrices from the Philox stream
with the attempt number in counter word 3, so both sides must take the same number of
restarts, end with the same diagonal-compression state, find the same ranks from the
attempt-k samples and produce the same blocks.

The problems are nearly incompressible linear elasticity (Q1, nu = 0.49 or 0.499, a stiff
inclusion), whose diagonal blocks at coarse diagonal tolerances are indefinite in the
oracle by a wide margin: the failing pivots lie between -0.3% and -500x of their
diagonal entry, and the smallest pivot of the successful attempt is at least 1% of its
diagonal entry, so rounding cannot change a restart decision.

Tolerances as in the other FP64 parity tests: blocks within 1e-8 relative, one
preconditioner application within 1e-8 in componentwise backward error against the
oracle's factor (and in forward error where the factor is well enough conditioned), PCG
to 1e-8 with iteration counts within +-2 of the oracle's.
"""
import numpy as np
import pytest

import paper_1507_05593_gb300 as R
import workloads as W
from oracle import factor as F

from test_gpu_fixed_rank import _blocks, _llt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _elast(ne, nu, incl):
    return W.elasticity_q1(ne, nu=nu, incl=incl)


def _oracle_an(p, kw):
    return F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, F.Options(**kw))


def _compare(p, h, an, f, forward_tol):
    st = R.rsc_get_stats(h)
    assert st["restarts"] == f.restarts, (st["restarts"], f.restarts)
    worst = 0.0
    for j in range(an.nsuper):
        info = R.rsc_get_supernode_info(h, j)
        assert info["compressed"] == int(f.sn[j].compressed), j
        assert info["hierarchical"] == int(f.sn[j].D.hierarchical), j
        if f.sn[j].compressed:
            assert info["rank"] == f.sn[j].U.shape[1], j
        LD, LO = R.rsc_get_supernode_blocks(h, j)
        LDo, LOo = _blocks(f, j)
        worst = max(worst, np.abs(np.tril(LD) - np.tril(LDo)).max() / max(1.0, np.abs(LDo).max()))
        if LOo.size:
            worst = max(worst, np.abs(LO - LOo).max() / max(1.0, np.abs(LOo).max()))
    assert worst <= 1e-8, worst
    r = np.random.default_rng(9).standard_normal(p.n)
    d_r = torch.tensor(r, device="cuda")
    d_z = torch.empty_like(d_r)
    R.rsc_apply_preconditioner_device(h, d_r, d_z)
    z = d_z.cpu().numpy()
    perm = an.ordering.perm
    zp = z[perm]
    eta = np.linalg.norm(_llt(f, zp, False) - r[perm]) / np.linalg.norm(_llt(f, np.abs(zp), True))
    assert eta <= 1e-8, eta
    z_ref = F.apply_preconditioner(f, r)
    fwd = np.abs(z - z_ref).max() / np.abs(z_ref).max()
    assert fwd <= forward_tol, fwd
    x, it, rr = R.rsc_solve(h, p.b, 1e-8, 1000)
    _, it_ref, _, ok = F.solve(an, f, p.b, 1e-8, 1000)
    assert ok and rr <= 1e-8 and abs(it - it_ref) <= 2, (it, it_ref)
    A = p.scipy()
    assert np.linalg.norm(p.b - A @ x) / np.linalg.norm(p.b) <= 1e-8


TOL_KW = dict(leaf_size=8, tau_O=64, tau_D=48, dof_per_node=3)


def _tol_problem():
    return W.elasticity_q1(10, nu=0.499, incl=(3, 7), e_stiff=1e3)


def test_restart_tolerance_form():
    """Tolerance form at tol 0.1: four restarts (tol_D = 0.1 / 1.25^4), diagonal compression
    still on at the end."""
    p = _tol_problem()
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, R.rsc_options_default(**TOL_KW))
    R.rsc_factor(h, 0.1)
    an = _oracle_an(p, TOL_KW)
    f = F.factor(an, 0.1)
    assert f.restarts == 4 and f.diag_compress
    _compare(p, h, an, f, 1e-6)


def test_restart_tolerance_form_exhausts_budget():
    """max_restarts = 1: the first attempt and the restarted one both fail, so the third
    attempt runs with diagonal compression switched off (no hierarchical block left)."""
    p = _tol_problem()
    kw = dict(TOL_KW, max_restarts=1)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, R.rsc_options_default(**kw))
    R.rsc_factor(h, 0.1)
    an = _oracle_an(p, kw)
    f = F.factor(an, 0.1)
    assert f.restarts == 2 and not f.diag_compress
    assert not any(R.rsc_get_supernode_info(h, j)["hierarchical"] for j in range(an.nsuper))
    _compare(p, h, an, f, 1e-6)


FR_KW = dict(leaf_size=8, tau_O=48, tau_D=24, dof_per_node=3)


def test_restart_fixed_rank_form():
    """Fixed-rank form (alpha_O 0.3, alpha_D 0.1, p 0): four restarts, alpha_D = 0.1 * 1.25^4."""
    p = _elast(8, 0.49, (3, 5))
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, R.rsc_options_default(**FR_KW))
    R.rsc_factor_fixed_rank(h, 0.3, 0.1, 0)
    an = _oracle_an(p, FR_KW)
    f = F.factor_fixed_rank(an, 0.3, 0.1, 0)
    assert f.restarts == 4 and f.diag_compress
    _compare(p, h, an, f, 1e-6)


def test_restart_fixed_rank_form_exhausts_budget():
    """alpha_D = 0.02: every one of the 8 restarts fails, the ninth attempt runs without
    diagonal compression."""
    p = _elast(6, 0.49, (2, 4))
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, R.rsc_options_default(**FR_KW))
    R.rsc_factor_fixed_rank(h, 0.3, 0.02, 0)
    an = _oracle_an(p, FR_KW)
    f = F.factor_fixed_rank(an, 0.3, 0.02, 0)
    assert f.restarts == 9 and not f.diag_compress
    _compare(p, h, an, f, 1e-6)


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_restart_mixed_precision_reaches_residual(prec):
    """The FP32 and split-TF32 forms take the restarts of their own rounding (the count need
    not equal the FP64 oracle's); the outer FP64 PCG still reaches 1e-8."""
    p = _tol_problem()
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, R.rsc_options_default(precision=prec, **TOL_KW))
    R.rsc_factor(h, 0.1)
    x, it, rr = R.rsc_solve(h, p.b, 1e-8, 2000)
    A = p.scipy()
    # the library confirms its own true residual; recomputed here in another summation order on
    # this nearly singular system it may differ by a few per cent
    assert rr <= 1e-8 and np.linalg.norm(p.b - A @ x) / np.linalg.norm(p.b) <= 1.1e-8


def test_restart_bf16_reports_not_spd():
    """BF16 operands (8-bit significand) in the Schur updates of this nearly incompressible
    problem leave the dense top separator indefinite; the restarts only make diagonal
    compression more accurate, so after max_restarts + 1 attempts the factorization reports
    RSC_ERR_NOT_SPD (no CUDA error, no hang), and the handle factors new values afterwards."""
    p = _tol_problem()
    kw = dict(TOL_KW, max_restarts=2)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, R.rsc_options_default(precision="bf16", **kw))
    with pytest.raises(R.RscError) as e:
        R.rsc_factor(h, 0.1)
    assert e.value.status == 2
    q = W.elasticity_q1(10, nu=0.3, incl=(3, 7), e_stiff=1.0)
    assert np.array_equal(q.col_idx, p.col_idx)
    R.rsc_refactor_values(h, q.val)
    R.rsc_factor(h, 0.1)
    x, it, rr = R.rsc_solve(h, q.b, 1e-8, 2000)
    assert rr <= 1e-8
