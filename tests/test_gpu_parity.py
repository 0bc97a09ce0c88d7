"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (FP64 path): the exact factor agrees within 1e-12 of the factor's
largest entry; compressed blocks agree within 1e-8 relative (the same Philox
test matrices drive both sides; only rounding differs); ranks are equal; the
preconditioner applications agree within 1e-8 relative; PCG reaches 1e-8 with
iteration counts within +-2 of the oracle's.  FP32 path: blocks within 1e-4
relative of the FP64 oracle, PCG still to 1e-8.
"""
import numpy as np
import pytest

import paper_1507_05593_gb300 as R
import workloads as W
from oracle import factor as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _opts(**kw):
    return R.rsc_options_default(**kw)


def _oracle(p, o, tol):
    oo = F.Options(tau_O=o.tau_O, tau_D=o.tau_D, leaf_size=o.leaf_size, dof_per_node=o.dof_per_node,
                   power_iters=o.power_iters, max_restarts=o.max_restarts, seed=o.seed,
                   diag_compress=bool(o.diag_compress))
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, oo)
    return an, F.factor(an, tol)


def _oracle_blocks(f, j):
    an = f.an
    s = f.sn[j]
    D = s.D
    c0, c1 = an.cols(j)
    c = c1 - c0
    if D.hierarchical:
        t = D.tree
        LD = np.zeros((c, c))
        for b in range(1, t.nblocks + 1):
            r0, r1 = t.rows(b)
            q0, q1 = t.cols(b)
            LD[r0:r1, q0:q1] = D.leafL[b] if t.leaf[b] else D.V[b] @ D.U[b].T
    else:
        LD = D.L
    r = an.sym.rows[j].size
    if r == 0:
        LO = np.zeros((0, c))
    elif s.compressed:
        LO = s.V @ s.U.T
    else:
        LO = s.LO
    return LD, LO


def _gpu(p, o, tol):
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, o)
    R.rsc_factor(h, tol)
    return h


CASES = [
    ("poisson8", lambda: W.poisson7(8), dict(leaf_size=8, tau_O=16, tau_D=8)),
    ("poisson_5x7x4", lambda: W.poisson7(5, 7, 4), dict(leaf_size=8, tau_O=12, tau_D=8)),
    ("grf12", lambda: W.diffusion_grf(12, 2.0, 3.0, 0), dict(leaf_size=16, tau_O=40, tau_D=32)),
    ("elast4", lambda: W.elasticity_q1(4, incl=(1, 3)), dict(leaf_size=8, tau_O=48, tau_D=24, dof_per_node=3)),
    ("poisson20", lambda: W.poisson7(20), dict(leaf_size=32, tau_O=100, tau_D=64)),
]


@pytest.mark.parametrize("name,maker,kw", CASES, ids=[c[0] for c in CASES])
def test_exact_factor_parity(name, maker, kw):
    p = maker()
    o = _opts(**kw)
    h = _gpu(p, o, 0.0)
    an, f = _oracle(p, o, 0.0)
    scale = max(np.abs(_oracle_blocks(f, j)[0]).max() for j in range(an.nsuper))
    for j in range(an.nsuper):
        LD, LO = R.rsc_get_supernode_blocks(h, j)
        LDo, LOo = _oracle_blocks(f, j)
        assert np.abs(np.tril(LD) - np.tril(LDo)).max() <= 1e-12 * scale, j
        if LOo.size:
            assert np.abs(LO - LOo).max() <= 1e-12 * scale, j
    x, it, rr = R.rsc_solve(h, p.b, 1e-8, 50)
    assert it <= 2 and rr <= 1e-8


@pytest.mark.parametrize("name,maker,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("tol", [0.1, 0.01])
def test_compressed_factor_parity(name, maker, kw, tol):
    p = maker()
    o = _opts(**kw)
    h = _gpu(p, o, tol)
    an, f = _oracle(p, o, tol)
    st = R.rsc_get_stats(h)
    assert st["restarts"] == f.restarts
    ncomp = 0
    for j in range(an.nsuper):
        info = R.rsc_get_supernode_info(h, j)
        assert info["compressed"] == int(f.sn[j].compressed)
        if f.sn[j].compressed:
            ncomp += 1
            assert info["rank"] == f.sn[j].U.shape[1], j
            if info["hierarchical"]:
                D = f.sn[j].D
                assert info["nblocks"] == D.tree.nblocks
        LD, LO = R.rsc_get_supernode_blocks(h, j)
        LDo, LOo = _oracle_blocks(f, j)
        sc = max(1.0, np.abs(LDo).max())
        assert np.abs(np.tril(LD) - np.tril(LDo)).max() <= 1e-8 * sc, j
        if LOo.size:
            assert np.abs(LO - LOo).max() <= 1e-8 * max(1.0, np.abs(LOo).max()), j
    assert ncomp == st["n_compressed"]
    # one preconditioner application, element by element
    r = np.random.default_rng(5).standard_normal(p.n)
    z_ref = F.apply_preconditioner(f, r)
    d_r = torch.tensor(r, device="cuda")
    d_z = torch.empty_like(d_r)
    R.rsc_apply_preconditioner_device(h, d_r, d_z)
    z = d_z.cpu().numpy()
    assert np.abs(z - z_ref).max() <= 1e-8 * np.abs(z_ref).max()
    x, it, rr = R.rsc_solve(h, p.b, 1e-8, 500)
    _, it_ref, rr_ref, ok = F.solve(an, f, p.b, 1e-8, 500)
    assert ok and rr <= 1e-8 and abs(it - it_ref) <= 2
    A = p.scipy()
    assert np.linalg.norm(p.b - A @ x) / np.linalg.norm(p.b) <= 1e-8


def test_poisson32_config_parity():
    """32^3 Poisson, tau_O = 256, tol 1e-1, 16-column samples, PCG to 1e-8 (all FP64)."""
    p = W.poisson7(32)
    o = _opts()
    h = _gpu(p, o, 0.1)
    an, f = _oracle(p, o, 0.1)
    for j in range(an.nsuper):
        if f.sn[j].compressed:
            assert R.rsc_get_supernode_info(h, j)["rank"] == f.sn[j].U.shape[1]
    r = np.random.default_rng(6).standard_normal(p.n)
    z_ref = F.apply_preconditioner(f, r)
    d_r = torch.tensor(r, device="cuda")
    d_z = torch.empty_like(d_r)
    R.rsc_apply_preconditioner_device(h, d_r, d_z)
    assert np.abs(d_z.cpu().numpy() - z_ref).max() <= 1e-8 * np.abs(z_ref).max()
    x, it, rr = R.rsc_solve(h, p.b, 1e-8, 500)
    _, it_ref, _, _ = F.solve(an, f, p.b, 1e-8, 500)
    assert rr <= 1e-8 and abs(it - it_ref) <= 2


def test_poisson40_large_blocks_parity():
    """40^3 Poisson, tol 1e-1: the top separator (1,600 columns) has internal blocks of 800
    columns, compressed by the cooperative pass kernel's full 13-phase mode (more than 8
    row chunks), the small blocks by the dense mode: ranks equal the oracle's, and the
    preconditioner applications agree within 1e-8."""
    p = W.poisson7(40)
    o = _opts()
    h = _gpu(p, o, 0.1)
    an, f = _oracle(p, o, 0.1)
    big = 0
    for j in range(an.nsuper):
        if not f.sn[j].compressed:
            continue
        info = R.rsc_get_supernode_info(h, j)
        assert info["rank"] == f.sn[j].U.shape[1], j
        big += info["c"] > 512
    assert big >= 1
    r = np.random.default_rng(7).standard_normal(p.n)
    z_ref = F.apply_preconditioner(f, r)
    d_r = torch.tensor(r, device="cuda")
    d_z = torch.empty_like(d_r)
    R.rsc_apply_preconditioner_device(h, d_r, d_z)
    assert np.abs(d_z.cpu().numpy() - z_ref).max() <= 1e-8 * np.abs(z_ref).max()


def test_poisson32_exact_sampled_blocks():
    """Exact 32^3 factor (dense 1024-column top separator): sampled supernodes vs oracle."""
    p = W.poisson7(32)
    o = _opts()
    h = _gpu(p, o, 0.0)
    an, f = _oracle(p, o, 0.0)
    for j in list(range(0, an.nsuper, 37)) + [an.nsuper - 1, an.nsuper - 2]:
        LD, LO = R.rsc_get_supernode_blocks(h, j)
        LDo, LOo = _oracle_blocks(f, j)
        assert np.abs(np.tril(LD) - LDo).max() <= 1e-12 * max(1, np.abs(LDo).max())
        if LOo.size:
            assert np.abs(LO - LOo).max() <= 1e-12 * max(1, np.abs(LDo).max())
    x, it, rr = R.rsc_solve(h, p.b, 1e-8, 50)
    assert it <= 2 and rr <= 1e-8


# Block tolerances of the mixed forms against the FP64 oracle (relative to the block's largest
# entry, diagonal blocks and V U^T alike).  FP32: products and storage in FP32 (unit 6e-8);
# TF32: Schur updates from split (high + low) TF32 operands, near FP32 accuracy; BF16: Schur
# updates from BF16 operands (unit 2^-8 = 3.9e-3).  Measured on a GB300 at 12^3 and 40^3:
# at most 4e-6 (FP32), 1.6e-6 (TF32), 1.7e-3 (BF16), ranks equal to the oracle's, PCG
# iterations equal.
MIXED_TOL = {"fp32": 1e-4, "tf32": 1e-4, "bf16": 1e-2}
MIXED_CASES = [
    ("grf12", lambda: W.diffusion_grf(12, 2.0, 3.0, 0), dict(leaf_size=16, tau_O=40, tau_D=32)),
    # 40^3 with the default parameters: a 1,600-column hierarchical top separator (800-column
    # internal blocks through the batched cooperative range finder), 760 x 1,600 off-diagonal
    # blocks, and multi-chunk tensor-core extend-add tiles
    ("grf40", lambda: W.diffusion_grf(40, 2.0, 8.0, 0), dict()),
]


@pytest.mark.parametrize("name,maker,kw", MIXED_CASES, ids=[c[0] for c in MIXED_CASES])
@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
def test_mixed_precision_parity(prec, name, maker, kw):
    """The FP32, split-TF32 and BF16 forms against the FP64 oracle at tol 1e-2: equal ranks,
    every diagonal block and every off-diagonal block (L^O_j, or V_j U_j^T) within the form's
    tolerance, PCG to 1e-8 within +-2 iterations of the oracle's."""
    p = maker()
    o = _opts(precision=prec, **kw)
    h = _gpu(p, o, 0.01)
    an, f = _oracle(p, R.rsc_options_default(**kw), 0.01)
    tol_blk = MIXED_TOL[prec]
    worst_d = worst_o = 0.0
    for j in range(an.nsuper):
        if f.sn[j].compressed:
            assert R.rsc_get_supernode_info(h, j)["rank"] == f.sn[j].U.shape[1], j
        LD, LO = R.rsc_get_supernode_blocks(h, j)
        LDo, LOo = _oracle_blocks(f, j)
        worst_d = max(worst_d, np.abs(np.tril(LD) - np.tril(LDo)).max() / max(1, np.abs(LDo).max()))
        if LOo.size:
            worst_o = max(worst_o, np.abs(LO - LOo).max() / max(1, np.abs(LOo).max()))
    assert worst_d <= tol_blk and worst_o <= tol_blk, (worst_d, worst_o)
    x, it, rr = R.rsc_solve(h, p.b, 1e-8, 500)
    _, it_ref, _, _ = F.solve(an, f, p.b, 1e-8, 500)
    assert rr <= 1e-8 and abs(it - it_ref) <= 2, (it, it_ref)


@pytest.mark.parametrize("prec,bound", [("bf16", 3e-2), ("tf32", 1e-4)])
def test_tensor_core_exact_mode_matches_fp32_path(prec, bound):
    """Compression off, so every Schur update goes through the tensor-core extend-add: the
    BF16 factor is within 8 units of BF16 rounding of the FP32 one; the split-TF32 factor
    (high and low parts, three products) within FP32 rounding (1e-4: one TF32 product
    alone would miss it); neither equals it (the tensor-core path ran); PCG restores 1e-8."""
    p = W.diffusion_grf(16, 1.0, 3.0, 0)
    kw = dict(leaf_size=16, tau_O=40, tau_D=32)
    h32 = _gpu(p, _opts(precision="fp32", **kw), 0.0)
    h16 = _gpu(p, _opts(precision=prec, **kw), 0.0)
    M = R.rsc_get_stats(h32)["n_supernodes"]
    worst = 0.0
    for j in range(M):
        a, ao = R.rsc_get_supernode_blocks(h32, j)
        b, bo = R.rsc_get_supernode_blocks(h16, j)
        worst = max(worst, np.abs(np.tril(a) - np.tril(b)).max() / max(1.0, np.abs(a).max()))
        if ao.size:
            worst = max(worst, np.abs(ao - bo).max() / max(1.0, np.abs(a).max()))
    assert 0 < worst <= bound, worst
    x, it, rr = R.rsc_solve(h16, p.b, 1e-8, 100)
    assert rr <= 1e-8


# ----------------------------------------------------------------------------- edge cases

def test_single_unknown_and_single_leaf():
    for p in (W.poisson7(1), W.poisson7(2), W.poisson7(4, 1, 1)):
        h = _gpu(p, _opts(), 0.1)
        x, it, rr = R.rsc_solve(h, p.b, 1e-8, 10)
        np.testing.assert_allclose(p.scipy() @ x, p.b, rtol=1e-10, atol=1e-12)
        assert it <= 2


def test_zero_rhs_and_state_errors():
    p = W.poisson7(6)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, _opts(leaf_size=8))
    with pytest.raises(R.RscError) as e:
        R.rsc_solve(h, p.b)
    assert e.value.status == 7
    R.rsc_factor(h, 0.1)
    x, it, rr = R.rsc_solve(h, np.zeros(p.n))
    assert it == 0 and np.all(x == 0)


def test_indefinite_matrix_reports_not_spd():
    p = W.poisson7(6)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, -p.val, p.coords, _opts(leaf_size=8))
    with pytest.raises(R.RscError) as e:
        R.rsc_factor(h, 0.0)
    assert e.value.status == 2
    # the handle stays usable: new values, factor again
    R.rsc_refactor_values(h, p.val)
    R.rsc_factor(h, 0.0)
    x, it, rr = R.rsc_solve(h, p.b)
    assert rr <= 1e-8


def test_refactor_values_changes_factor():
    p = W.diffusion_grf(10, 1.0, 3.0, 0)
    q = W.diffusion_grf(10, 1.0, 3.0, 1)
    assert np.array_equal(p.col_idx, q.col_idx)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, _opts(leaf_size=16))
    R.rsc_factor(h, 0.0)
    R.rsc_refactor_values(h, q.val)
    R.rsc_factor(h, 0.0)
    x, it, rr = R.rsc_solve(h, q.b)
    np.testing.assert_allclose(q.scipy() @ x, q.b, rtol=0, atol=1e-8 * np.abs(q.b).max() * 10)


def test_solve_device_matches_host():
    p = W.poisson7(12)
    h = _gpu(p, _opts(leaf_size=16, tau_O=40, tau_D=32), 0.1)
    x, it, rr = R.rsc_solve(h, p.b)
    d_b = torch.tensor(p.b, device="cuda")
    d_x = torch.empty_like(d_b)
    it2, rr2 = R.rsc_solve_device(h, d_b, d_x)
    assert it2 == it
    np.testing.assert_allclose(d_x.cpu().numpy(), x, rtol=1e-12, atol=1e-14)


# ----------------------------------------------------------------------------- full size (96^3)

@pytest.mark.slow
def test_diffusion96_full_size_properties():
    """96^3 FV diffusion with GRF conductivity (sigma 2, correlation length 8), tol 1e-2:
    PCG reaches 1e-8 (true residual checked on the CPU); FP64 and FP32 forms."""
    p = W.diffusion_grf(96, 2.0, 8.0, 0)
    A = p.scipy()
    for prec in ("fp64", "fp32"):
        h = _gpu(p, _opts(precision=prec), 1e-2)
        x, it, rr = R.rsc_solve(h, p.b, 1e-8, 1000)
        assert rr <= 1e-8
        assert np.linalg.norm(p.b - A @ x) / np.linalg.norm(p.b) <= 1e-8
        st = R.rsc_get_stats(h)
        assert st["n_compressed"] == 165 and st["factor_bytes"] > 0


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_autotuned_products_agree(prec):
    """The first factorization of a BF16 / TF32 handle alternates the SIMT and tensor-core thin
    products to time them; the second uses the faster one per key.  Both factorizations give the
    oracle's ranks and blocks within the form's tolerance, and PCG reaches 1e-8."""
    p = W.diffusion_grf(24, 2.0, 4.0, 0)
    kw = dict(leaf_size=32, tau_O=64, tau_D=64)
    h = _gpu(p, _opts(precision=prec, **kw), 0.01)
    tab = R.rsc_get_autotune(h)
    assert any(v["launches"][0] > 0 and v["launches"][1] > 0 for v in tab.values()), tab
    assert all(v["choice"] in (-1, 0, 1) for v in tab.values())
    an, f = _oracle(p, R.rsc_options_default(**kw), 0.01)
    for rep in range(2):
        if rep:
            R.rsc_factor(h, 0.01)
        for j in range(an.nsuper):
            if f.sn[j].compressed:
                assert R.rsc_get_supernode_info(h, j)["rank"] == f.sn[j].U.shape[1], (rep, j)
            LD, LO = R.rsc_get_supernode_blocks(h, j)
            LDo, LOo = _oracle_blocks(f, j)
            assert np.abs(np.tril(LD) - np.tril(LDo)).max() <= MIXED_TOL[prec] * max(1, np.abs(LDo).max()), (rep, j)
            if LOo.size:
                assert np.abs(LO - LOo).max() <= MIXED_TOL[prec] * max(1, np.abs(LOo).max()), (rep, j)
        x, it, rr = R.rsc_solve(h, p.b, 1e-8, 500)
        assert rr <= 1e-8


def test_expired_barrier_wait_reports_timeout_and_handle_recovers():
    """A grid-barrier wait of the cooperative range-finder kernel that runs out (wait limit set
    to one poll, so a block that reaches a barrier before the others gives up) ends the
    factorization with RSC_ERR_TIMEOUT instead of hanging or faulting; with the default limit
    restored and the values set again the handle factors and solves as before."""
    p = W.poisson7(32)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, _opts())
    R.rsc_set_wait_limit(h, 1)
    with pytest.raises(R.RscError) as e:
        R.rsc_factor(h, 0.1)
    assert e.value.status == 6, e.value
    with pytest.raises(R.RscError) as e:
        R.rsc_solve(h, p.b)
    assert e.value.status == 7
    R.rsc_set_wait_limit(h, 0)
    R.rsc_refactor_values(h, p.val)
    R.rsc_factor(h, 0.1)
    x, it, rr = R.rsc_solve(h, p.b, 1e-8, 200)
    an, f = _oracle(p, _opts(), 0.1)
    _, it_ref, _, _ = F.solve(an, f, p.b, 1e-8, 200)
    assert rr <= 1e-8 and abs(it - it_ref) <= 2
    with pytest.raises(R.RscError):
        R.rsc_set_wait_limit(h, -1)


def test_refactor_values_device_matches_host_values():
    """New values given on the device (no host copy) factor and solve like the same values given
    on the host; a non-finite device value is rejected; host values take over again afterwards."""
    p = W.diffusion_grf(12, 1.0, 3.0, 0)
    q = W.diffusion_grf(12, 1.0, 3.0, 1)
    kw = dict(leaf_size=16, tau_O=40, tau_D=32)
    h_host = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, _opts(**kw))
    h_dev = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, _opts(**kw))
    R.rsc_refactor_values(h_host, q.val)
    R.rsc_refactor_values_device(h_dev, torch.tensor(q.val, device="cuda"))
    for h in (h_host, h_dev):
        R.rsc_factor(h, 0.1)
    for j in range(R.rsc_get_stats(h_host)["n_supernodes"]):
        a, ao = R.rsc_get_supernode_blocks(h_host, j)
        b, bo = R.rsc_get_supernode_blocks(h_dev, j)
        assert np.abs(a - b).max() <= 1e-12 * max(1, np.abs(a).max()), j
        if ao.size:
            assert np.abs(ao - bo).max() <= 1e-12 * max(1, np.abs(ao).max()), j
    x, it, rr = R.rsc_solve(h_dev, q.b, 1e-8, 200)     # the SpMV uses the device values too
    assert rr <= 1e-8
    assert np.linalg.norm(q.b - q.scipy() @ x) / np.linalg.norm(q.b) <= 1e-8
    bad = torch.tensor(q.val, device="cuda")
    bad[5] = float("nan")
    with pytest.raises(R.RscError) as e:
        R.rsc_refactor_values_device(h_dev, bad)
    assert e.value.status == 1
    R.rsc_refactor_values(h_dev, p.val)                 # host values again
    R.rsc_factor(h_dev, 0.1)
    x, it, rr = R.rsc_solve(h_dev, p.b, 1e-8, 200)
    assert np.linalg.norm(p.b - p.scipy() @ x) / np.linalg.norm(p.b) <= 1e-8
