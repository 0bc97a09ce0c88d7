"""Differentiation form: x = A(theta)^{-1} b through paper_1507_05593_gb300.autograd.

The gradient of L = 0.5 ||x(theta) - x*||^2 (adjoint PCG with the kept factor, then
the -lambda_i x_j contraction over A's pattern) is checked against a dense FP64
reference gradient (torch.linalg.solve with autograd) and against central finite
differences along random directions.
"""
import numpy as np
import pytest

import paper_1507_05593_gb300 as R
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(side, seed=0):
    rng = np.random.default_rng(seed)
    shape = (side, side, side)
    fv = W.FVValues(shape)
    theta = rng.standard_normal(shape)
    theta_star = theta + 0.1 * rng.standard_normal(shape)
    b = rng.uniform(-1, 1, fv.n)
    return fv, theta, theta_star, b


def _dense_solve(fv, theta, b):
    vals = fv(theta)
    A = torch.sparse_csr_tensor(torch.as_tensor(fv.row_ptr), torch.as_tensor(fv.col_idx.astype(np.int64)), vals,
                                size=(fv.n, fv.n)).to_dense()
    return torch.linalg.solve(A, b)


@pytest.mark.parametrize("prec,tol", [("fp64", 0.0), ("fp64", 0.1), ("fp32", 0.1)])
def test_gradient_vs_dense_reference_and_fd(prec, tol):
    from paper_1507_05593_gb300.autograd import sparse_spd_solve
    side = 12
    fv, theta, theta_star, b = _setup(side)
    # dense FP64 reference (CPU)
    th_ref = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    b_cpu = torch.tensor(b, dtype=torch.float64)
    x_star = _dense_solve(fv, torch.tensor(theta_star), b_cpu).detach()
    x_ref = _dense_solve(fv, th_ref, b_cpu)
    loss_ref = 0.5 * ((x_ref - x_star) ** 2).sum()
    loss_ref.backward()
    g_ref = th_ref.grad.numpy()
    # ours
    opts = R.rsc_options_default(precision=prec, leaf_size=16, tau_O=40, tau_D=32)
    h = R.rsc_analyze(fv.n, fv.row_ptr, fv.col_idx, fv(torch.tensor(theta)).numpy(), fv.coords, opts)
    th = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
    b_gpu = b_cpu.cuda()
    xs = x_star.cuda()

    rtol = 1e-12 if prec == "fp64" else 1e-10    # FP32 preconditioner: PCG noise floor near 1e-11

    def loss_of(t):
        x = sparse_spd_solve(fv(t), b_gpu, h, tol=tol, rtol=rtol)
        return 0.5 * ((x - xs) ** 2).sum()

    loss = loss_of(th)
    loss.backward()
    g = th.grad.cpu().numpy()
    assert abs(loss.item() - loss_ref.item()) <= 1e-9 * abs(loss_ref.item())
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) <= 1e-6
    # central finite differences along the 32 random directions of the differentiation
    # configuration (seeded)
    rng = np.random.default_rng(3)
    hstep = 1e-6 if prec == "fp64" else 1e-4
    with torch.no_grad():
        for _ in range(32):
            d = torch.tensor(rng.standard_normal(theta.shape), device="cuda")
            fd = (loss_of(th + hstep * d).item() - loss_of(th - hstep * d).item()) / (2 * hstep)
            ad = float((torch.tensor(g, device="cuda") * d).sum())
            assert abs(fd - ad) <= 1e-4 * abs(ad), (fd, ad)


def test_backward_reuses_factor():
    """The adjoint solve uses the factor of the forward pass: no refactorization between."""
    from paper_1507_05593_gb300.autograd import sparse_spd_solve
    fv, theta, theta_star, b = _setup(10, seed=1)
    h = R.rsc_analyze(fv.n, fv.row_ptr, fv.col_idx, fv(torch.tensor(theta)).numpy(), fv.coords,
                      R.rsc_options_default(leaf_size=16, tau_O=40, tau_D=32))
    th = torch.tensor(theta, device="cuda", requires_grad=True)
    x = sparse_spd_solve(fv(th), torch.tensor(b, device="cuda"), h, tol=0.1, rtol=1e-12)
    t_factor = R.rsc_get_stats(h)["factor_seconds"]
    x.sum().backward()
    assert R.rsc_get_stats(h)["factor_seconds"] == t_factor
    assert torch.isfinite(th.grad).all()


@pytest.mark.slow
def test_differentiation_config_64():
    """64^3 FV diffusion, theta ~ N(0,1), x* from theta + 0.1 N(0,1): FP32 factor, FP64 PCG;
    autograd directional derivatives vs central differences (FD solves at rtol 1e-12)."""
    from paper_1507_05593_gb300.autograd import sparse_spd_solve
    side = 64
    rng = np.random.default_rng(0)
    shape = (side, side, side)
    fv = W.FVValues(shape)
    theta = rng.standard_normal(shape)
    theta_star = theta + 0.1 * np.random.default_rng(1).standard_normal(shape)
    b = np.random.default_rng(2).uniform(-1, 1, fv.n)
    h = R.rsc_analyze(fv.n, fv.row_ptr, fv.col_idx, fv(torch.tensor(theta)).numpy(), fv.coords,
                      R.rsc_options_default(precision="fp32"))
    b_gpu = torch.tensor(b, device="cuda")
    with torch.no_grad():
        xs = sparse_spd_solve(fv(torch.tensor(theta_star, device="cuda")), b_gpu, h, tol=1e-2, rtol=1e-12)
    th = torch.tensor(theta, device="cuda", requires_grad=True)

    def loss_of(t):
        x = sparse_spd_solve(fv(t), b_gpu, h, tol=1e-2, rtol=1e-12)
        return 0.5 * ((x - xs) ** 2).sum()

    loss = loss_of(th)
    loss.backward()
    g = th.grad.clone()
    rng3 = np.random.default_rng(3)
    with torch.no_grad():
        for _ in range(2):
            d = torch.tensor(rng3.standard_normal(shape), device="cuda")
            fd = (loss_of(th + 1e-6 * d).item() - loss_of(th - 1e-6 * d).item()) / 2e-6
            ad = float((g * d).sum())
            assert abs(fd - ad) <= 1e-4 * abs(ad), (fd, ad)
