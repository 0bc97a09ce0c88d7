"""The allocation-free preconditioner application against the regular one.

rsc_apply_preconditioner_device_noalloc serves callers that cannot call
cudaMalloc (their device memory belongs to another allocator or budget, or they
cannot afford its implicit synchronisation); it keeps its scratch in a static
device array instead.  It must give the same z = M^{-1} r as
rsc_apply_preconditioner_device, call after call, and must not take device
memory.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import paper_1507_05593_gb300 as R
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-8, "fp32": 1e-4}   # the preconditioner tolerances of the parity tests


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_apply_matches_regular_apply(prec):
    p = W.diffusion_grf(24, 2.0, 4.0, 0)
    o = R.rsc_options_default(precision=prec, leaf_size=32, tau_O=64, tau_D=64)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, o)
    R.rsc_factor(h, 0.01)
    assert any(R.rsc_get_supernode_info(h, j)["hierarchical"] for j in range(R.rsc_get_stats(h)["n_supernodes"]))
    rng = np.random.default_rng(11)
    for call in range(3):
        r = torch.tensor(rng.standard_normal(p.n), device="cuda")
        z_ref = torch.empty_like(r)
        z = torch.full_like(r, float("nan"))
        R.rsc_apply_preconditioner_device(h, r, z_ref)
        torch.cuda.synchronize()
        # the reading is taken before every call, the first (loading) one included
        free_before, _ = torch.cuda.mem_get_info()
        R.rsc_apply_preconditioner_device_noalloc(h, r, z)
        torch.cuda.synchronize()
        free_after, _ = torch.cuda.mem_get_info()
        # one cudaMalloc takes at least a 2 MiB granule; the call must take nothing
        assert free_before - free_after == 0, (call, free_before - free_after)
        err = ((z - z_ref).abs().max() / z_ref.abs().max()).item()
        assert err <= TOL[prec], (call, err)


def test_noalloc_apply_blocks_until_done():
    """Every call synchronises the stream it is given: on return the stream is idle and z holds
    the result, without a synchronisation by the caller."""
    p = W.diffusion_grf(16, 1.0, 3.0, 2)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords,
                      R.rsc_options_default(leaf_size=16, tau_O=40, tau_D=32))
    R.rsc_factor(h, 0.1)
    r = torch.tensor(np.random.default_rng(4).standard_normal(p.n), device="cuda")
    z_ref = torch.empty_like(r)
    R.rsc_apply_preconditioner_device(h, r, z_ref)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    for call in range(2):
        z = torch.full_like(r, float("nan"))
        torch.cuda.synchronize()
        R.rsc_apply_preconditioner_device_noalloc(h, r, z, stream=side)
        assert side.query(), call
        assert ((z - z_ref).abs().max() / z_ref.abs().max()).item() <= TOL["fp64"], call


def test_noalloc_apply_follows_refactor():
    """After a new factorization the next call reloads its records (same result as the regular apply)."""
    p = W.diffusion_grf(16, 1.0, 3.0, 1)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords,
                      R.rsc_options_default(leaf_size=16, tau_O=40, tau_D=32))
    r = torch.tensor(np.random.default_rng(3).standard_normal(p.n), device="cuda")
    for tol in (0.1, 0.0):
        R.rsc_factor(h, tol)
        z_ref = torch.empty_like(r)
        z = torch.empty_like(r)
        R.rsc_apply_preconditioner_device(h, r, z_ref)
        R.rsc_apply_preconditioner_device_noalloc(h, r, z)
        assert ((z - z_ref).abs().max() / z_ref.abs().max()).item() <= TOL["fp64"]
