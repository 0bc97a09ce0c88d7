"""Symbolic analysis (oracle; test infrastructure), Section 2.1.

Follows the paper's definitions literally:

* column structure of L by the elimination tree: struct(L(:,p)) is the set of
  rows i > p of A(:,p) united with struct(L(:,c)) \\ {p} over the tree children c
  of p; the tree parent of p is the smallest row of struct(L(:,p));
* R_j (Eq. before "descendents"): rows after supernode j's columns with a
  nonzero in some column of C_j.  Reading: the paper also states (below Eq.
  "schurOffDiag") that a descendant k of j has R_k meeting the rows after C_j only
  inside R_j; when a supernode's columns are not one chain of the elimination tree
  (the graph ordering's separators and leaves may be disconnected), the union of
  the column structures can break that, so R_j is the smallest set that keeps it:
  the rows after C_j of A(:, C_j) united with R_k restricted to rows after C_j
  over every k in D_j (computed in supernode order).  It contains the union of the
  column structures and equals it whenever every supernode is an elimination-tree
  chain (every lattice ordering); the extra rows hold exact zeros;
* D_j (Eq. "descendents"): supernodes k < j with R_k meeting C_j;
* R^D_{k->j}, R^O_{k->j} (Eqs. "rowsDiagKtoJ", "rowsOffKtoJ"): positions in R_k of
  the rows that fall in C_j, resp. in R_j.

Exact column structures are kept per column, so this is meant for grids up to
about 40^3; larger problems are checked through properties (see the tests).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class Symbolic:
    def __init__(self):
        self.n = 0
        self.snode_ptr = None      # [M+1]
        self.snode_of = None       # [n] supernode of each column
        self.rows = []             # R_j, sorted global (permuted) row indices
        self.desc = []             # D_j as list of (k, pD, pO) with positions into R_k
        self.parent = None         # supernodal tree parent (-1 = root)
        self.etree = None          # column elimination tree parent (-1 = root)

    @property
    def nsuper(self):
        return len(self.snode_ptr) - 1


def symbolic(Ap: sp.csr_matrix, snode_ptr: np.ndarray) -> Symbolic:
    """Ap: permuted symmetric matrix (full pattern).  snode_ptr: supernode columns."""
    n = Ap.shape[0]
    M = len(snode_ptr) - 1
    csc = sp.csc_matrix(Ap)
    csc.sort_indices()
    snode_of = np.repeat(np.arange(M), np.diff(snode_ptr))
    etree = -np.ones(n, dtype=np.int64)
    children: list[list[int]] = [[] for _ in range(n)]
    struct: dict[int, np.ndarray] = {}
    R = []
    meets: list[list[int]] = [[] for _ in range(M)]   # k with R_k meeting C_j (D_j), filled as R_k is known
    for j in range(M):
        c0, c1 = int(snode_ptr[j]), int(snode_ptr[j + 1])
        acc = []
        for p in range(c0, c1):
            # column elimination tree (the column structures of L)
            col = csc.indices[csc.indptr[p]:csc.indptr[p + 1]]
            pieces = [col[col > p]]
            for c in children[p]:
                s = struct.pop(c)
                pieces.append(s[s != p])
            s = np.unique(np.concatenate(pieces)) if pieces else np.zeros(0, np.int64)
            s = s.astype(np.int64)
            if s.size:
                etree[p] = s[0]
                children[s[0]].append(p)
                struct[p] = s
            acc.append(col[col >= c1].astype(np.int64))   # rows after C_j of A(:, C_j)
        for k in meets[j]:                                   # R_k beyond C_j, k in D_j
            acc.append(R[k][R[k] >= c1])
        Rj = np.unique(np.concatenate(acc)).astype(np.int64) if acc else np.zeros(0, np.int64)
        R.append(Rj)
        for i in np.unique(snode_of[Rj]).tolist():
            meets[i].append(j)
    sym = Symbolic()
    sym.n = n
    sym.snode_ptr = np.asarray(snode_ptr, dtype=np.int64)
    sym.snode_of = snode_of
    sym.rows = R
    sym.etree = etree
    sym.parent = np.array([snode_of[r[0]] if r.size else -1 for r in R], dtype=np.int64)
    desc: list[list] = [[] for _ in range(M)]
    for k in range(M):
        if R[k].size == 0:
            continue
        for j in np.unique(snode_of[R[k]]):
            c0, c1 = snode_ptr[j], snode_ptr[j + 1]
            pD = np.nonzero((R[k] >= c0) & (R[k] < c1))[0]
            pO = np.nonzero(np.isin(R[k], R[j]))[0]
            desc[j].append((k, pD, pO))
    sym.desc = desc
    return sym
