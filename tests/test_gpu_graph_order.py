"""GPU parity with the graph ordering: graph nested dissection of a non-grid sparsity
pattern (given real positions) and spectral positions (no coordinates, Section 4.3).

With the same positions both sides order identically (bit-exact, checked on the host),
so the factorization is compared as for the lattice ordering: equal ranks, blocks within
1e-8, one preconditioner application within 1e-8, PCG iterations within +-2.  Without
coordinates the two sides compute their own spectral positions (the host's Lanczos run,
the oracle's dense eigensolver), which agree only to rounding, so the GPU run is checked
by what is unique: the exact factor solves in at most 2 iterations and the compressed one
reaches 1e-8.
"""
import numpy as np
import pytest

import paper_1507_05593_gb300 as R
import workloads as W
from oracle import factor as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


AMALG = [("graph", lambda: W.random_geometric(1500, 0.12, seed=2), dict(leaf_size=24, tau_O=60, tau_D=40, ordering=1)),
         ("graph_amalgamated", lambda: W.random_geometric(1500, 0.12, seed=2),
          dict(leaf_size=24, tau_O=60, tau_D=40, ordering=1, amalgamate=1)),
         ("lattice_amalgamated", lambda: W.diffusion_grf(14, 2.0, 3.0, 0),
          dict(leaf_size=8, tau_O=40, tau_D=32, amalgamate=1))]


@pytest.mark.parametrize("name,maker,kw", AMALG, ids=[a[0] for a in AMALG])
def test_graph_ordering_random_geometric_parity(name, maker, kw):
    """Graph ordering, and relaxed amalgamation of small supernodes (Section 3.1) on the graph
    and the lattice orderings: the merged partition (bit-exact on the host) factors with the
    oracle's ranks, one apply within 1e-8, PCG iterations within +-2."""
    p = maker()
    o = R.rsc_options_default(**kw)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords, o)
    R.rsc_factor(h, 0.1)
    an = F.analyze(p.n, p.row_ptr, p.col_idx, p.val, p.coords,
                   F.Options(**{k: (bool(v) if k == "amalgamate" else v) for k, v in kw.items()}))
    f = F.factor(an, 0.1)
    assert sum(s.compressed for s in f.sn) >= 1
    assert R.rsc_get_stats(h)["n_supernodes"] == an.nsuper
    for j in range(an.nsuper):
        info = R.rsc_get_supernode_info(h, j)
        assert info["compressed"] == int(f.sn[j].compressed), j
        if f.sn[j].compressed:
            assert info["rank"] == f.sn[j].U.shape[1], j
    r = np.random.default_rng(9).standard_normal(p.n)
    z_ref = F.apply_preconditioner(f, r)
    d_r = torch.tensor(r, device="cuda")
    d_z = torch.empty_like(d_r)
    R.rsc_apply_preconditioner_device(h, d_r, d_z)
    assert np.abs(d_z.cpu().numpy() - z_ref).max() <= 1e-8 * np.abs(z_ref).max()
    x, it, rr = R.rsc_solve(h, p.b, 1e-8, 500)
    _, it_ref, _, ok = F.solve(an, f, p.b, 1e-8, 500)
    assert ok and rr <= 1e-8 and abs(it - it_ref) <= 2
    assert np.linalg.norm(p.b - p.scipy() @ x) / np.linalg.norm(p.b) <= 1e-8


def test_spectral_positions_factor_and_solve():
    p = W.diffusion_grf(12, 2.0, 3.0, 0)
    o = R.rsc_options_default(leaf_size=16, tau_O=40, tau_D=32)
    h = R.rsc_analyze(p.n, p.row_ptr, p.col_idx, p.val, None, o)
    R.rsc_factor(h, 0.0)
    x, it, rr = R.rsc_solve(h, p.b, 1e-8, 10)
    assert it <= 2 and rr <= 1e-8
    R.rsc_factor(h, 0.05)
    assert R.rsc_get_stats(h)["n_compressed"] >= 1
    x, it, rr = R.rsc_solve(h, p.b, 1e-8, 500)
    assert rr <= 1e-8
    assert np.linalg.norm(p.b - p.scipy() @ x) / np.linalg.norm(p.b) <= 1e-8
