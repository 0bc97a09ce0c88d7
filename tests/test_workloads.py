"""Checks of the seeded input generators against closed forms (CPU).

The generators hold none of the method's arithmetic; these tests pin that the
synthetic systems are the PDE discretizations they stand for.
"""
import numpy as np
import scipy.sparse.linalg as sla

import workloads as W


def test_q1_element_stiffness_rigid_modes_and_energies():
    """Unit-cube trilinear element, E = 1, nu = 0.3: symmetric positive semidefinite of rank
    18 whose null space is the six rigid-body motions; a uniform stretch u_x = x stores
    u^T K u = lambda + 2 mu and a uniform shear u_x = y stores mu (linear fields are exact
    in the element and the 2x2x2 Gauss rule integrates the quadratic energy exactly)."""
    nu = 0.3
    K = W._q1_unit_stiffness(nu)
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    np.testing.assert_allclose(K, K.T, atol=1e-14)
    w = np.linalg.eigvalsh(K)
    assert w[:6].max() <= 1e-12 * w.max() and w[6] > 1e-3 * w.max() and w.min() > -1e-12
    X = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=np.float64)
    modes = []
    for ax in range(3):                                  # translations
        u = np.zeros((8, 3))
        u[:, ax] = 1.0
        modes.append(u.ravel())
    for om in np.eye(3):                                 # rotations omega x x
        modes.append(np.cross(om, X).ravel())
    for u in modes:
        assert np.abs(K @ u).max() <= 1e-12
    u = np.zeros((8, 3))
    u[:, 0] = X[:, 0]
    assert abs(u.ravel() @ K @ u.ravel() - (lam + 2 * mu)) <= 1e-12
    u = np.zeros((8, 3))
    u[:, 0] = X[:, 1]
    assert abs(u.ravel() @ K @ u.ravel() - mu) <= 1e-12


def test_poisson7_smallest_eigenvalue():
    """7-point Laplacian with Dirichlet boundary on an n1 x n2 x n3 grid: the smallest
    eigenvalue is sum over the axes of 2 - 2 cos(pi / (n_a + 1))."""
    p = W.poisson7(7, 5, 4)
    A = p.scipy()
    assert (A != A.T).nnz == 0
    lam = sla.eigsh(A, k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
    expect = sum(2 - 2 * np.cos(np.pi / (m + 1)) for m in (7, 5, 4))
    assert abs(lam - expect) <= 1e-10


def test_fv_diffusion_unit_conductivity_stencil():
    """k = 1 everywhere: interior faces have transmissibility 2 k k / (k + k) = 1 and a
    boundary face adds 2 k = 2, so an interior cell's diagonal is 6, a face cell's 7, an
    edge cell's 8 and a corner cell's 9; off-diagonals are -1."""
    n = 5
    p = W.fv_diffusion(np.ones((n, n, n)), 0)
    A = p.scipy().toarray()
    off = A - np.diag(np.diag(A))
    assert set(np.unique(off).tolist()) <= {-1.0, 0.0}
    x, y, z = p.coords[:, 0], p.coords[:, 1], p.coords[:, 2]
    nb = sum(((c == 0) | (c == n - 1)).astype(int) for c in (x, y, z))
    np.testing.assert_allclose(np.diag(A), 6 + nb)


def test_grf_moments_and_correlation_length():
    """Periodic Gaussian random field: mean 0 and standard deviation sigma exactly (it is
    normalised); its correlation at lag l along an axis follows exp(-l^2 / (2 L^2)) within
    the spread of one 64^3 realisation."""
    L, sigma = 6.0, 2.0
    g = W.grf((64, 64, 64), sigma, L, seed=1)
    assert abs(g.mean()) <= 1e-12 and abs(g.std() - sigma) <= 1e-12
    for lag in (3, 6, 9):
        c = np.mean(g * np.roll(g, lag, axis=0)) / sigma ** 2
        assert abs(c - np.exp(-lag ** 2 / (2 * L ** 2))) <= 0.12, (lag, c)


def test_fv_values_torch_function_matches_generator_and_differentiates():
    """FVValues(shape)(theta) is fv_diffusion(exp(theta)) entry for entry in CSR order, and
    its derivative in theta passes torch's finite-difference gradcheck (FP64, CPU)."""
    import pytest
    torch = pytest.importorskip("torch")
    shape = (3, 4, 5)
    theta = np.random.default_rng(7).standard_normal(shape)
    fv = W.FVValues(shape)
    ref = W.fv_diffusion(np.exp(theta), 0)
    np.testing.assert_array_equal(fv.row_ptr, ref.row_ptr)
    np.testing.assert_array_equal(fv.col_idx, ref.col_idx)
    vals = fv(torch.tensor(theta)).numpy()
    np.testing.assert_allclose(vals, ref.val, rtol=1e-13, atol=1e-13)
    small = W.FVValues((2, 2, 3))
    th = torch.tensor(np.random.default_rng(8).standard_normal((2, 2, 3)), requires_grad=True)
    assert torch.autograd.gradcheck(small, (th,), eps=1e-6, atol=1e-7)
