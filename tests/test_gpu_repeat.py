"""Run-to-run spread of the factorization on one GPU.

The extend-add and the scattered products accumulate with atomic adds, so the order of
floating-point additions into a target may change from one run to the next; nothing else in
the path depends on timing.  Two factorizations of the same matrix therefore agree to
rounding: the same ranks (the adaptive stopping test of Alg. 3 sees norms that differ in the
last bits only), blocks within a few units of rounding of the arithmetic's precision, and the
same PCG iteration counts.
"""
import numpy as np
import pytest

import paper_1507_05593_gb300 as R
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,bound", [("fp64", 1e-12), ("fp32", 1e-4), ("bf16", 1e-2)])
def test_repeated_factorizations_agree(prec, bound):
    p = W.diffusion_grf(16, 2.0, 4.0, 0)
    o = R.rsc_options_default(precision=prec, leaf_size=16, tau_O=40, tau_D=32)
    runs = []
    for _ in range(3):
        h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, o)
        R.rsc_factor(h, 0.01)
        M = R.rsc_get_stats(h)["n_supernodes"]
        ranks = [R.rsc_get_supernode_info(h, j)["rank"] for j in range(M)]
        d_r = torch.tensor(np.random.default_rng(1).standard_normal(p.n), device="cuda")
        d_z = torch.empty_like(d_r)
        R.rsc_apply_preconditioner_device(h, d_r, d_z)
        x, it, rr = R.rsc_solve(h, p.b, 1e-8, 500)
        runs.append((ranks, d_z.cpu().numpy(), it))
    for ranks, z, it in runs[1:]:
        assert ranks == runs[0][0]
        assert np.abs(z - runs[0][1]).max() <= bound * np.abs(runs[0][1]).max()
        assert it == runs[0][2]


def test_batch_of_256_systems_repeats_exactly_in_fp64():
    """The 256-system batch (5.8M unknowns, the batching configuration's systems) factored four
    times on one handle in FP64: the same rank on every supernode and no restart each time.
    With the cooperative pass's small-block mode this failed about one factorization in four
    (wrong samples at this scale; 64 systems repeated exactly), so it needs the full batch."""
    import scipy.sparse as sp
    sides = np.random.Generator(np.random.Philox(0)).integers(12, 41, 256)
    ps = [W.diffusion_lognormal(int(sd), 1.0, seed=i) for i, sd in enumerate(sides)]
    A = sp.block_diag([p.scipy() for p in ps]).tocsr()
    A.sort_indices()
    coords, off = [], 0
    for p in ps:
        c = p.coords.copy()
        c[:, 0] += off
        off = int(c[:, 0].max()) + 4
        coords.append(c)
    h = R.rsc_analyze(A.shape[0], A.indptr, A.indices, A.data, np.vstack(coords), R.rsc_options_default())
    M = R.rsc_get_stats(h)["n_supernodes"]
    ref = None
    for _ in range(4):
        R.rsc_factor(h, 0.01)
        assert R.rsc_get_stats(h)["restarts"] == 0
        ranks = [R.rsc_get_supernode_info(h, j)["rank"] for j in range(M)]
        if ref is None:
            ref = ranks
        assert ranks == ref
