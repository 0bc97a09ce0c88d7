"""Relaxed supernode amalgamation (oracle; test infrastructure), Section 3.1.

Section 3.1 groups the columns of small supernodes "by methods identical to CHOLMOD".  CHOLMOD
relaxes its fundamental supernodes by merging a child into its parent when the merged block
stays small or adds few explicit zeros, with three size thresholds and three zero fractions.
Reading used on both sides (the paper gives no parameters; CHOLMOD's defaults are taken):

* supernodes are visited in their order (a postorder of the supernodal tree); the groups built
  so far form a stack; group G (starting as one supernode) absorbs the group L on top of the
  stack while
    - L's supernodal parent lies in G (the first row of R_L is a column of G) -- L ends where
      G begins, since the order is a postorder;
    - neither is compressed: a separator with at least tau_O columns keeps its own supernode,
      and a merged separator must stay below tau_O columns;
    - with ns = c_L + c_G, R_M = R_G united with the rows of R_L after G's columns, stored
      entries s(X) = c (c + 1) / 2 + c |R| of a block with c columns and rows R, and
      z = 1 - (s(L) + s(G)) / s(M) the fraction of the merged block's entries that neither
      block stored before: ns <= 4, or ns <= 16 and z <= 0.8, or ns <= 48 and z <= 0.1, or
      z <= 0.05;
  the merged group has G's kind and R_M;
* the merged partition's supernodal structure is then computed as for any other.

Columns keep their order, so the factor it gives (with compression off) is the same Cholesky
factor; only the blocking changes.
"""
from __future__ import annotations

import numpy as np

NRELAX = (4, 16, 48)
ZRELAX = (0.8, 0.1, 0.05)


def _stored(c: int, r: int) -> int:
    return c * (c + 1) // 2 + c * r


def merge_ok(cL: int, rL: int, cG: int, rG: int, rM: int) -> bool:
    """The relaxation rule for merging a child block (cL columns, rL rows) into its parent
    (cG, rG) giving rM rows after the merged columns."""
    ns = cL + cG
    z = 1.0 - (_stored(cL, rL) + _stored(cG, rG)) / _stored(ns, rM)
    return (ns <= NRELAX[0] or (ns <= NRELAX[1] and z <= ZRELAX[0]) or (ns <= NRELAX[2] and z <= ZRELAX[1])
            or z <= ZRELAX[2])


def amalgamate(snode_ptr, kinds, rows, tau_O: int):
    """Merged partition: (snode_ptr, kinds, members), members[g] = the original supernodes of
    group g.  rows[j]: R_j of the unmerged partition (sorted permuted row indices)."""
    M = len(snode_ptr) - 1
    stack = []   # [first col, end col, R (array), kind, members]

    def compressed(kind, c):
        return kind == 1 and c >= tau_O

    for s in range(M):
        G = [int(snode_ptr[s]), int(snode_ptr[s + 1]), np.asarray(rows[s], dtype=np.int64), int(kinds[s]), [s]]
        while stack:
            L = stack[-1]
            RL = L[2]
            cL, cG = L[1] - L[0], G[1] - G[0]
            if RL.size == 0 or not (G[0] <= RL[0] < G[1]):
                break
            if compressed(L[3], cL) or compressed(G[3], cG) or compressed(G[3], cL + cG):
                break
            RM = np.union1d(G[2], RL[RL >= G[1]])
            if not merge_ok(cL, RL.size, cG, G[2].size, RM.size):
                break
            stack.pop()
            G = [L[0], G[1], RM, G[3], L[4] + G[4]]
        stack.append(G)
    ptr = np.array([stack[0][0]] + [g[1] for g in stack], dtype=np.int64)
    return ptr, [g[3] for g in stack], [g[4] for g in stack]
