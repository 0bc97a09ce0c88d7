"""Dense kernels written out as loops (oracle; test infrastructure).

These are the LAPACK/BLAS steps the paper's Algorithms call (Cholesky, the
triangular solves, the QR inside makeOrthonormal, Alg. 3) restated plainly so
that the oracle does not lean on the routines the pins compare against.
"""
from __future__ import annotations

import numpy as np


class NotPositiveDefinite(Exception):
    pass


def cholesky(S: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor by the column (Crout) recurrence; raises on a pivot <= 0."""
    n = S.shape[0]
    L = np.zeros_like(S, dtype=np.float64)
    for k in range(n):
        d = S[k, k] - L[k, :k] @ L[k, :k]
        if not d > 0.0:
            raise NotPositiveDefinite(f"pivot {k}: {d}")
        L[k, k] = np.sqrt(d)
        if k + 1 < n:
            L[k + 1:, k] = (S[k + 1:, k] - L[k + 1:, :k] @ L[k, :k]) / L[k, k]
    return L


def solve_lower(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X = L^{-1} B by forward substitution."""
    X = np.array(B, dtype=np.float64, copy=True)
    for i in range(L.shape[0]):
        X[i] = (X[i] - L[i, :i] @ X[:i]) / L[i, i]
    return X


def solve_lower_T(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X = L^{-T} B by backward substitution."""
    X = np.array(B, dtype=np.float64, copy=True)
    n = L.shape[0]
    for i in range(n - 1, -1, -1):
        X[i] = (X[i] - L[i + 1:, i] @ X[i + 1:]) / L[i, i]
    return X


def householder_q(Y: np.ndarray) -> np.ndarray:
    """Thin Q (m x b) of the Householder QR of Y (m x b, m >= b)."""
    R = np.array(Y, dtype=np.float64, copy=True)
    m, b = R.shape
    vs = []
    for k in range(b):
        x = R[k:, k]
        nx = np.sqrt(x @ x)
        v = x.copy()
        v[0] += nx if x[0] >= 0 else -nx
        nv = np.sqrt(v @ v)
        if nv == 0.0:
            v = np.zeros_like(x)
            v[0] = 1.0
            nv = 1.0
            # a zero column: reflect e1 onto itself (H = I - 2 e1 e1^T still orthogonal)
        v /= nv
        R[k:, k:] -= 2.0 * np.outer(v, v @ R[k:, k:])
        vs.append(v)
    Q = np.zeros((m, b))
    Q[np.arange(b), np.arange(b)] = 1.0
    for k in range(b - 1, -1, -1):
        v = vs[k]
        Q[k:, :] -= 2.0 * np.outer(v, v @ Q[k:, :])
    return Q
