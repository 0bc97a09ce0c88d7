"""Seeded synthetic inputs shaped like the paper's PDE test problems.

This module builds matrices, node coordinates and right-hand sides only.  It
holds none of the factorization's arithmetic, so both the CUDA path (through
its tests and the benchmark) and the CPU oracle may draw their inputs from it.

Every generator returns a :class:`Problem` whose matrix is the full symmetric
CSR (both triangles, sorted column indices, no duplicates) with int64 row
pointers, int32 column indices and float64 values.  Coordinates are lattice
positions (one row per unknown), which is what the nested-dissection ordering
bisects.

Workloads (the paper's own deal.II / UF problems are not available, so these
seeded grids stand in for them; their shapes follow the paper's 3D PDE
examples, Section 6):

* ``poisson7``      7-point finite-difference Laplacian, Dirichlet boundary
                    eliminated, diagonal 6 and off-diagonal -1 (no h^2 scaling).
* ``fv_diffusion``  7-point finite-volume operator with harmonic-mean face
                    transmissibilities 2 k_a k_b / (k_a + k_b); a boundary face
                    adds 2 k_c (Dirichlet at half a cell).
* ``grf``           periodic Gaussian random field with covariance
                    exp(-r^2 / (2 l^2)), normalised to mean 0 and std sigma.
* ``elasticity_q1`` trilinear hexahedral linear elasticity, 2x2x2 Gauss rule,
                    the x = 0 face clamped, a stiff central inclusion and a
                    uniform body force; three unknowns per node kept adjacent.
* ``random_geometric`` a non-grid sparsity pattern: points uniform in the unit
                    cube joined when closer than a radius; the matrix is the
                    graph Laplacian plus a diagonal shift; coordinates are the
                    points' real positions (for the graph ordering).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass
class Problem:
    name: str
    n: int
    row_ptr: np.ndarray      # int64 [n+1]
    col_idx: np.ndarray      # int32 [nnz]
    val: np.ndarray          # float64 [nnz]
    coords: np.ndarray       # float64 [n, 3] lattice positions
    b: np.ndarray            # float64 [n]
    dof_per_node: int = 1
    shape: tuple = ()

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.n, self.n))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def rhs_uniform(n: int, seed: int = 0) -> np.ndarray:
    """b ~ U[-1, 1], drawn from numpy's Philox bit generator with the given seed."""
    return _rng(seed).uniform(-1.0, 1.0, n)


def _grid_coords(nx: int, ny: int, nz: int) -> np.ndarray:
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float64)


def _csr_from_coo(n, rows, cols, vals) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    m = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    m.sum_duplicates()
    m.sort_indices()
    return m.indptr.astype(np.int64), m.indices.astype(np.int32), m.data.astype(np.float64)


def _face_pairs(nx, ny, nz):
    """Index pairs (a, b) of cells sharing a face, along x, y and z."""
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    pairs = []
    pairs.append((idx[:, :, :-1].ravel(), idx[:, :, 1:].ravel()))
    pairs.append((idx[:, :-1, :].ravel(), idx[:, 1:, :].ravel()))
    pairs.append((idx[:-1, :, :].ravel(), idx[1:, :, :].ravel()))
    a = np.concatenate([p[0] for p in pairs])
    b = np.concatenate([p[1] for p in pairs])
    return a, b


def poisson7(nx: int, ny: int | None = None, nz: int | None = None, seed: int = 0) -> Problem:
    """7-point Laplacian on an nx*ny*nz interior grid; unknown x + nx*y + nx*ny*z."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    n = nx * ny * nz
    a, b = _face_pairs(nx, ny, nz)
    rows = np.concatenate([a, b, np.arange(n)])
    cols = np.concatenate([b, a, np.arange(n)])
    vals = np.concatenate([-np.ones(2 * a.size), 6.0 * np.ones(n)])
    rp, ci, v = _csr_from_coo(n, rows, cols, vals)
    return Problem(f"poisson7_{nx}x{ny}x{nz}", n, rp, ci, v, _grid_coords(nx, ny, nz),
                   rhs_uniform(n, seed), 1, (nx, ny, nz))


def fv_diffusion(kcell: np.ndarray, seed: int = 0) -> Problem:
    """7-point finite-volume diffusion operator for cell conductivities kcell[nz, ny, nx]."""
    nz, ny, nx = kcell.shape
    n = nx * ny * nz
    k = kcell.ravel().astype(np.float64)
    a, b = _face_pairs(nx, ny, nz)
    t = 2.0 * k[a] * k[b] / (k[a] + k[b])
    diag = np.zeros(n)
    np.add.at(diag, a, t)
    np.add.at(diag, b, t)
    # boundary faces: each cell adds 2 k_c per face on the domain boundary
    kk = kcell.astype(np.float64)
    nb = np.zeros_like(kk)
    nb[:, :, 0] += 1; nb[:, :, -1] += 1
    nb[:, 0, :] += 1; nb[:, -1, :] += 1
    nb[0, :, :] += 1; nb[-1, :, :] += 1
    diag += (2.0 * kk * nb).ravel()
    rows = np.concatenate([a, b, np.arange(n)])
    cols = np.concatenate([b, a, np.arange(n)])
    vals = np.concatenate([-t, -t, diag])
    rp, ci, v = _csr_from_coo(n, rows, cols, vals)
    return Problem(f"fv_diffusion_{nx}x{ny}x{nz}", n, rp, ci, v, _grid_coords(nx, ny, nz),
                   rhs_uniform(n, seed), 1, (nx, ny, nz))


def grf(shape: tuple, sigma: float, corr_len: float, seed: int = 0) -> np.ndarray:
    """Periodic Gaussian random field g[nz, ny, nx].

    White noise (numpy Philox stream, ``seed``) is filtered in Fourier space by
    the square root of the spectrum of the covariance exp(-r^2 / (2 corr_len^2))
    (r the minimum-image distance in cells), then shifted and scaled to sample
    mean 0 and sample standard deviation ``sigma``.
    """
    nz, ny, nx = shape
    w = _rng(seed).standard_normal(shape)

    def d(m):
        i = np.arange(m)
        return np.minimum(i, m - i).astype(np.float64)

    dz, dy, dx = np.meshgrid(d(nz), d(ny), d(nx), indexing="ij")
    cov = np.exp(-(dx ** 2 + dy ** 2 + dz ** 2) / (2.0 * corr_len ** 2))
    spec = np.maximum(np.fft.fftn(cov).real, 0.0)
    f = np.fft.ifftn(np.sqrt(spec) * np.fft.fftn(w)).real
    return sigma * (f - f.mean()) / f.std()


def diffusion_grf(side: int, sigma: float = 2.0, corr_len: float = 8.0, seed: int = 0) -> Problem:
    """FV diffusion on side^3 cells with conductivity exp(g), g a GRF (seeded)."""
    g = grf((side, side, side), sigma, corr_len, seed)
    p = fv_diffusion(np.exp(g), seed)
    p.name = f"diffusion_grf_{side}^3"
    return p


def diffusion_lognormal(side: int, sigma: float = 1.0, seed: int = 0, rhs_seed: int | None = None) -> Problem:
    """FV diffusion on side^3 cells with iid log-normal conductivity exp(sigma z)."""
    z = _rng(seed).standard_normal((side, side, side))
    p = fv_diffusion(np.exp(sigma * z), seed if rhs_seed is None else rhs_seed)
    p.name = f"diffusion_lognormal_{side}^3"
    return p


# ----------------------------------------------------------------------------- elasticity

def _q1_unit_stiffness(nu: float) -> np.ndarray:
    """24x24 stiffness of the unit cube trilinear element for E = 1 (dofs node-major)."""
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3:, 3:] = np.eye(3) * mu
    # node ordering: local node a = ax + 2 ay + 4 az with corner (ax, ay, az)
    corners = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=np.float64)
    gp = np.array([0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)])
    K = np.zeros((24, 24))
    for qx in gp:
        for qy in gp:
            for qz in gp:
                q = np.array([qx, qy, qz])
                dN = np.zeros((8, 3))
                for a in range(8):
                    f = np.where(corners[a] > 0.5, q, 1 - q)
                    s = np.where(corners[a] > 0.5, 1.0, -1.0)
                    dN[a, 0] = s[0] * f[1] * f[2]
                    dN[a, 1] = f[0] * s[1] * f[2]
                    dN[a, 2] = f[0] * f[1] * s[2]
                B = np.zeros((6, 24))
                for a in range(8):
                    B[0, 3 * a + 0] = dN[a, 0]
                    B[1, 3 * a + 1] = dN[a, 1]
                    B[2, 3 * a + 2] = dN[a, 2]
                    B[3, 3 * a + 0] = dN[a, 1]; B[3, 3 * a + 1] = dN[a, 0]
                    B[4, 3 * a + 1] = dN[a, 2]; B[4, 3 * a + 2] = dN[a, 1]
                    B[5, 3 * a + 0] = dN[a, 2]; B[5, 3 * a + 2] = dN[a, 0]
                K += B.T @ D @ B / 8.0
    return K


def elasticity_q1(ne: int = 40, nu: float = 0.3, e_soft: float = 1.0, e_stiff: float = 1e3,
                  incl: tuple = (15, 25)) -> Problem:
    """Q1 linear elasticity on ne^3 elements of [0,1]^3, x = 0 face clamped.

    Elements with index in [incl[0], incl[1]) along every axis have Young's
    modulus ``e_stiff`` (a central 10^3 cube for ne = 40), the rest ``e_soft``.
    The load is the consistent nodal vector of the body force (0, 0, -1).
    """
    nn = ne + 1
    h = 1.0 / ne
    Ku = _q1_unit_stiffness(nu)
    ez, ey, ex = np.meshgrid(np.arange(ne), np.arange(ne), np.arange(ne), indexing="ij")
    ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
    inside = ((ex >= incl[0]) & (ex < incl[1]) & (ey >= incl[0]) & (ey < incl[1])
              & (ez >= incl[0]) & (ez < incl[1]))
    E = np.where(inside, e_stiff, e_soft) * h  # stiffness of a cube of side h scales with h
    loc = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)])
    nodes = ((ex[:, None] + loc[None, :, 0]) + nn * (ey[:, None] + loc[None, :, 1])
             + nn * nn * (ez[:, None] + loc[None, :, 2]))                   # [nel, 8]
    dofs = (3 * nodes[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 24)
    # clamp x = 0: node ix == 0 is removed; renumber the free nodes in natural order
    all_ix = np.arange(nn ** 3) % nn
    free = all_ix != 0
    new_node = -np.ones(nn ** 3, dtype=np.int64)
    new_node[free] = np.arange(free.sum())
    dof_map = (3 * new_node[:, None] + np.arange(3)[None, :])
    dof_map[~free] = -1
    dof_map = dof_map.ravel()
    gd = dof_map[dofs]                                                      # [nel, 24]
    n = int(free.sum()) * 3
    ii = np.broadcast_to(gd[:, :, None], (gd.shape[0], 24, 24))
    jj = np.broadcast_to(gd[:, None, :], (gd.shape[0], 24, 24))
    vv = E[:, None, None] * Ku[None, :, :]
    keep = (ii >= 0) & (jj >= 0)
    rp, ci, v = _csr_from_coo(n, ii[keep], jj[keep], vv[keep])
    # consistent load: each element contributes (volume / 8) * b to each of its nodes
    f = np.zeros(n)
    fz = gd[:, 2::3]
    ok = fz >= 0
    np.add.at(f, fz[ok], -(h ** 3) / 8.0)
    nz_, ny_, nx_ = np.meshgrid(np.arange(nn), np.arange(nn), np.arange(nn), indexing="ij")
    nc = np.stack([nx_.ravel(), ny_.ravel(), nz_.ravel()], axis=1)[free].astype(np.float64)
    coords = np.repeat(nc, 3, axis=0)
    return Problem(f"elasticity_q1_{ne}^3", n, rp, ci, v, coords, f, 3, (ne, ne, ne))


# ----------------------------------------------------------------------------- differentiable values

class FVValues:
    """CSR values of ``fv_diffusion`` as a torch function of the log-conductivity.

    ``FVValues(shape)(theta)`` returns the values of ``fv_diffusion(exp(theta))`` in its
    CSR order (the pattern is fixed by the grid), built from torch operations so that
    autograd can differentiate them with respect to theta[nz, ny, nx].
    """

    def __init__(self, shape):
        nz, ny, nx = shape
        self.shape = shape
        n = nx * ny * nz
        a, b = _face_pairs(nx, ny, nz)
        ref = fv_diffusion(np.ones(shape))          # pattern and entry order
        rp, ci = ref.row_ptr, ref.col_idx
        rows = np.repeat(np.arange(n), np.diff(rp))
        face_of = {}
        for f, (p, q) in enumerate(zip(a.tolist(), b.tolist())):
            face_of[(p, q)] = f
            face_of[(q, p)] = f
        self.is_diag = rows == ci
        self.face = np.array([0 if d else face_of[(int(r), int(c))] for r, c, d in zip(rows, ci, self.is_diag)])
        self.rows = rows
        self.a, self.b = a, b
        nb = np.zeros(shape)
        nb[:, :, 0] += 1; nb[:, :, -1] += 1
        nb[:, 0, :] += 1; nb[:, -1, :] += 1
        nb[0, :, :] += 1; nb[-1, :, :] += 1
        self.nbound = nb.ravel()
        self.row_ptr, self.col_idx, self.n = rp, ci, n
        self.coords = ref.coords

    def __call__(self, theta):
        import torch
        dev = theta.device
        k = torch.exp(theta.reshape(-1).to(torch.float64))
        a = torch.as_tensor(self.a, device=dev)
        b = torch.as_tensor(self.b, device=dev)
        t = 2.0 * k[a] * k[b] / (k[a] + k[b])
        diag = 2.0 * k * torch.as_tensor(self.nbound, device=dev, dtype=torch.float64)
        diag = diag.index_add(0, a, t).index_add(0, b, t)
        is_diag = torch.as_tensor(self.is_diag, device=dev)
        off = -t[torch.as_tensor(self.face, device=dev)]
        on = diag[torch.as_tensor(self.rows, device=dev)]
        return torch.where(is_diag, on, off)


def random_geometric(npts: int, radius: float, shift: float = 0.1, seed: int = 0) -> Problem:
    """Graph Laplacian + shift I of the random geometric graph on ``npts`` points uniform
    in [0,1]^3 (numpy Philox, ``seed``), edge between points closer than ``radius``;
    b ~ U[-1, 1] (seed ``seed``).  Coordinates are the points themselves (real)."""
    X = _rng(seed).uniform(0.0, 1.0, (npts, 3))
    d2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(axis=2)
    a, b = np.nonzero(np.triu(d2 < radius * radius, 1))
    deg = np.bincount(np.r_[a, b], minlength=npts).astype(np.float64)
    rows = np.concatenate([a, b, np.arange(npts)])
    cols = np.concatenate([b, a, np.arange(npts)])
    vals = np.concatenate([-np.ones(2 * a.size), deg + shift])
    rp, ci, v = _csr_from_coo(npts, rows, cols, vals)
    return Problem(f"random_geometric_{npts}_{radius:g}", npts, rp, ci, v, X, rhs_uniform(npts, seed), 1, ())
