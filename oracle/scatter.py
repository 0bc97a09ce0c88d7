"""scatterRows / gatherRows (oracle; test infrastructure), Section 2.1 (Eq. "scatterEx").

scatterRows(B, R1, R2): R1 is an ordered sub-list of the ordered list R2 and B has
|R1| rows; the result has |R2| rows, with row i of B placed at the position of
R1[i] inside R2 and zeros elsewhere.  gatherRows(C, R2, R1) undoes it: it returns
the rows of C at the positions of R1's entries inside R2.
"""
from __future__ import annotations

import numpy as np


def positions(R1, R2) -> np.ndarray:
    """Positions of the entries of R1 inside the ordered list R2 (R1 must be a subset)."""
    R1 = np.asarray(R1)
    R2 = np.asarray(R2)
    pos = np.searchsorted(R2, R1)
    if R1.size and (pos.max() >= R2.size or np.any(R2[pos] != R1)):
        raise ValueError("R1 is not a subset of R2")
    return pos


def scatter_rows(B, R1, R2) -> np.ndarray:
    B = np.asarray(B, dtype=np.float64)
    out = np.zeros((len(R2),) + B.shape[1:])
    out[positions(R1, R2)] = B
    return out


def gather_rows(C, R2, R1) -> np.ndarray:
    return np.asarray(C)[positions(R1, R2)]
