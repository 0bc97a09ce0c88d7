"""Numeric factorization (oracle; test infrastructure).

Algorithm by algorithm, in the paper's order and notation:

* ``factor_supernode``          Alg. 1 (Section 2.1, Eqs. "schurDiag", "schurOffDiag").
* ``offdiag_multiply``          Alg. 2 (Section 3.4), with Eq. "lowRankMult" for
                                descendants stored as V_k U_k^T.
* ``offdiag_multiply_T``        (L^O_j)^T G.  The paper only says it has "similar
                                structure" (Section 3.4).  Reading: (L^O_j)^T =
                                (L^D_j)^{-1} (U^O_j)^T with U^O_j from Eq. "schurOffDiag":
                                W = A(R_j,C_j)^T G; for each k in D_j:
                                T = L^O_k(R^O,:)^T gatherRows(G, R_j, R^O_glob);
                                T = L^O_k(R^D,:) T; W -= scatterRows(T, R^D_glob, C_j);
                                then W <- diagonalSolve(j, W, transpose=false).
* ``approximate_offdiag``       Alg. 3 in adaptive form.  The paper fixes ranks by a
                                heuristic (Section 5.2) but notes adaptive tolerance
                                as an option; here the blocked adaptive range finder:
                                16-column passes, each projected twice against the
                                current basis U (CGS2); stop before appending when
                                ||Yhat||_F <= tol ||Y_1||_F (Y_1 = first pass), or when
                                rank reaches min(|C_j|, |R_j|).  makeOrthonormal is a
                                Householder QR, re-projected and re-orthonormalised
                                once so the new columns stay orthogonal to U; a pass
                                that would exceed min(|C_j|, |R_j|) keeps only its
                                first min(16, remaining) projected columns.
* ``diagonal_solve``            Alg. 4.  Reading: the printed branches are swapped;
                                L^{-1} solves G1 first, then G2 -= V_s (U_s^T G1), then
                                G2; L^{-T} solves G2 first, then G1 -= U_s (V_s^T G2),
                                then G1.
* ``diagonal_multiply(_T)``     Alg. 5 and its transpose (Section 4.2).
* ``factor_diagonal``           Alg. 6.  Readings: the descendant update uses L^O_k
                                (the printed L^D_k cannot be indexed by R_k), and the
                                loop over ancestors advances p <- parent(p).
* ``approximate_diagonal_block`` "nearly identical" to Alg. 3 (Section 4.2), with
                                tolerance tol_D.
* ``factor``                    Section 4.2's block order s = 1, 2, ... and the
                                indefinite restart of Section 5.3 in tolerance form:
                                tol_D <- tol_D / 1.25 per restart; after
                                ``max_restarts`` restarts diagonal compression is
                                switched off (Section 3.2 then guarantees success).
* ``factor_fixed_rank``         Section 5.2's fixed-rank form of Alg. 3: block B
                                (m x n) gets rank(B) = alpha sqrt(k) log2(k) + p,
                                k = min(m, n) (Eq. rankFunction), alpha^O for
                                off-diagonal and alpha^D for diagonal blocks.
                                Reading: the rank is ceil(alpha sqrt(k) log2 k) + p,
                                capped at k.  The samples are the same 16-column
                                passes as the adaptive form with the stopping test
                                off (tol = 0); in exact arithmetic span(U) equals
                                span((B^T B)^q B^T G) for G the first rank(B) sampled
                                columns, the one-shot form of Alg. 3.  Section 5.3's
                                restart: alpha^D <- 1.25 alpha^D, starting from 0.5.

* Interior blocks (Section 5.1, ``Options.interior_blocks``): every maximal subtree
  of the supernodal tree without a compressed supernode is one interior block B,
  contiguous in the ordering; only L_B = chol(A(C_B, C_B)) is kept (Eq.
  "interiorDiagonalDef", a dense Cholesky here) and L(R_B, C_B) is never stored.
  Where the factorization needs rows X of it, they are L(X, C_B) = A(X, C_B) L_B^{-T}
  (Eq. "interiorBlockClosedForm"), formed for the small Schur complements and
  dropped; products L(X, C_B) L(Y, C_B)^T G go through Eq. "interiorBlockMult":
  A(Y, C_B)^T G, two triangular solves with L_B, then A(X, C_B).  The preconditioner
  apply solves with L_B and uses the same closed form for the block's off-diagonal.

Low-rank descendants keep U_prod = U_k^T U_k literally (Eq. "lowRankMult").
Random test matrices come from ``oracle.philox.gaussian_block`` with block id
(j << 12) | s (s = 0 for the off-diagonal block, s = label for diagonal blocks).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
from scipy.sparse import csgraph

from . import dense
from .dense import NotPositiveDefinite
from .ordering import node_graph, spectral_coordinates
from .ordering import Ordering
from .ordering import order as nd_order
from .philox import gaussian_block
from .scatter import gather_rows, positions, scatter_rows
from .symbolic import symbolic
from .amalgamate import amalgamate


@dataclasses.dataclass
class Options:
    tau_O: int = 256
    tau_D: int = 256
    leaf_size: int = 64
    sample_block: int = 16
    power_iters: int = 0
    dof_per_node: int = 1
    max_restarts: int = 8
    seed: int = 0
    diag_compress: bool = True
    ordering: int = 0          # 0: lattice bisection; 1: graph nested dissection
    interior_blocks: bool = False   # Section 5.1: L(R_B, C_B) of interior blocks not stored
    amalgamate: bool = False   # Section 3.1: relaxed amalgamation of small supernodes (amalgamate.py)


class Analysis:
    """Ordering + symbolic structure of one matrix."""

    def __init__(self, n, row_ptr, col_idx, val, coords, opts: Options):
        self.opts = opts
        self.n = n
        A = sp.csr_matrix((val, col_idx, row_ptr), shape=(n, n))
        # connected components of the node graph (independent systems are ordered apart)
        dof = opts.dof_per_node
        Pn = sp.csr_matrix((np.ones(len(col_idx)), (np.repeat(np.arange(n), np.diff(row_ptr)) // dof,
                                                      np.asarray(col_idx) // dof)), shape=(n // dof, n // dof))
        ncomp, labels = csgraph.connected_components(Pn, directed=False)
        comps = labels if ncomp > 1 else None
        graph = None
        if opts.ordering == 1 or coords is None:
            graph = node_graph(n, row_ptr, col_idx, dof)
            if coords is None:   # Section 4.3: positions from the graph Laplacian
                coords = np.repeat(spectral_coordinates(graph[0], graph[1], comps), dof, axis=0)
        self.coords = coords
        self.ordering = nd_order(coords, dof, opts.leaf_size, opts.tau_O, opts.tau_D, comps, graph)
        p = self.ordering.perm
        self.A = A
        self.Ap = sp.csr_matrix(A[p][:, p])
        self.Ap.sort_indices()
        self.sym = symbolic(self.Ap, self.ordering.snode_ptr)
        if opts.amalgamate:
            od = self.ordering
            kint = [1 if k == "sep" else 0 for k in od.kinds]
            ptr, kinds, members = amalgamate(od.snode_ptr, kint, self.sym.rows, opts.tau_O)
            trees = [od.trees[m[0]] if len(m) == 1 else None for m in members]
            self.ordering = Ordering(od.perm, ptr, ["sep" if k == 1 else "leaf" for k in kinds], trees)
            self.sym = symbolic(self.Ap, ptr)

    @property
    def nsuper(self):
        return self.sym.nsuper

    def cols(self, j):
        return int(self.sym.snode_ptr[j]), int(self.sym.snode_ptr[j + 1])

    def A_block(self, rows, cols) -> np.ndarray:
        """Dense A(rows, cols) of the permuted matrix (rows/cols global index arrays)."""
        return self.Ap[rows][:, cols].toarray()


class DiagFactor:
    """L^D_j: dense, or hierarchical over a BlockTree (Section 4.1)."""

    def __init__(self, tree=None):
        self.tree = tree
        self.L = None          # dense case
        self.leafL = {}        # s -> dense leaf block
        self.V = {}            # s -> V_s
        self.U = {}            # s -> U_s

    @property
    def hierarchical(self):
        return self.tree is not None


class SupernodeFactor:
    def __init__(self):
        self.compressed = False
        self.D: DiagFactor | None = None
        self.LO = None         # dense L^O_j (uncompressed)
        self.V = None          # V_j (compressed)
        self.U = None          # U_j
        self.Uprod = None      # U_j^T U_j


def rank_heuristic(m: int, n: int, alpha: float, p: int) -> int:
    """Eq. rankFunction (Section 5.2): ceil(alpha sqrt(k) log2 k) + p with k = min(m, n),
    capped at k (a block of k independent columns has no larger rank)."""
    k = min(int(m), int(n))
    if k <= 0:
        return 0
    return min(k, int(np.ceil(alpha * np.sqrt(k) * np.log2(k))) + int(p))


class Factor:
    def __init__(self, an: Analysis):
        self.an = an
        self.sn = [SupernodeFactor() for _ in range(an.nsuper)]
        self.restarts = 0
        self.compress = False
        self.tol = 0.0
        self.tol_D = 0.0
        self.diag_compress = False
        self.fixed_rank = False    # Section 5.2 ranks instead of the adaptive stopping test
        self.alpha_O = 0.0
        self.alpha_D = 0.0
        self.p = 0
        self.iblock_of = None      # Section 5.1: interior block of each supernode (-1: none)
        self.iblocks = []          # per block: dict(first, last, c0, c1, RB, L)

    # ----------------------------------------------------------- Section 5.1
    def _find_interior_blocks(self):
        """Maximal subtrees of the supernodal tree with no compressed supernode; each is
        a contiguous run of supernodes first..last (postorder) ending at its root."""
        an = self.an
        M = an.nsuper
        parent = an.sym.parent
        self.iblock_of = -np.ones(M, dtype=np.int64)
        self.iblocks = []
        if not an.opts.interior_blocks:
            return
        bad = [self.is_compressed(j) for j in range(M)]
        first = list(range(M))
        for j in range(M):                       # children precede parents
            pj = int(parent[j])
            if pj >= 0:
                bad[pj] = bad[pj] or bad[j]
                first[pj] = min(first[pj], first[j])
        for j in range(M):
            pj = int(parent[j])
            if bad[j] or (pj >= 0 and not bad[pj]):
                continue                         # not the root of a maximal clean subtree
            f0 = first[j]
            assert all(not bad[k] for k in range(f0, j + 1)), "interior block not contiguous"
            c0, _ = an.cols(f0)
            _, c1 = an.cols(j)
            rows = [an.sym.rows[k] for k in range(f0, j + 1)]
            RB = np.unique(np.concatenate(rows)) if rows else np.zeros(0, np.int64)
            RB = RB[RB >= c1]
            self.iblock_of[f0:j + 1] = len(self.iblocks)
            self.iblocks.append(dict(first=f0, last=j, c0=c0, c1=c1, RB=RB, L=None))

    def _ib_L(self, b, rows):
        """Rows ``rows`` of L(:, C_B): A(rows, C_B) L_B^{-T} (Eq. interiorBlockClosedForm)."""
        B = self.iblocks[b]
        Arc = self.an.A_block(rows, np.arange(B["c0"], B["c1"]))
        return dense.solve_lower(B["L"], Arc.T).T

    def _ib_mult(self, b, rows_out, rows_in, G):
        """L(rows_out, C_B) L(rows_in, C_B)^T G by Eq. interiorBlockMult."""
        B = self.iblocks[b]
        CB = np.arange(B["c0"], B["c1"])
        T = self.an.A_block(rows_in, CB).T @ G
        T = dense.solve_lower(B["L"], T)
        T = dense.solve_lower_T(B["L"], T)
        return self.an.A_block(rows_out, CB) @ T

    def _split_desc(self, j):
        """D_j without interior supernodes, and the interior blocks that meet D_j."""
        if self.iblock_of is None or not self.iblocks:
            return self.an.sym.desc[j], []
        ib = self.iblock_of
        normal = [d for d in self.an.sym.desc[j] if ib[d[0]] < 0]
        blocks = sorted({int(ib[d[0]]) for d in self.an.sym.desc[j] if ib[d[0]] >= 0})
        return normal, blocks

    # ----------------------------------------------------------- descendant blocks
    def lo_rows(self, k, pos):
        """Rows `pos` of L^O_k (uncompressed) or of V_k (compressed)."""
        s = self.sn[k]
        return s.LO[pos] if not s.compressed else s.V[pos]

    def lo_pair_product(self, k, pa, pb):
        """L^O_k(pa,:) L^O_k(pb,:)^T, or V_k(pa,:) U_k^T U_k V_k(pb,:)^T (Eq. lowRankMult)."""
        s = self.sn[k]
        if not s.compressed:
            return s.LO[pa] @ s.LO[pb].T
        return s.V[pa] @ (s.Uprod @ s.V[pb].T)

    def lo_apply(self, k, pa, pb, G):
        """L^O_k(pa,:) (L^O_k(pb,:)^T G) with the low-rank form when k is compressed."""
        s = self.sn[k]
        if not s.compressed:
            return s.LO[pa] @ (s.LO[pb].T @ G)
        T = s.V[pb].T @ G
        T = s.Uprod @ T
        return s.V[pa] @ T

    # ----------------------------------------------------------- Alg. 4
    def diagonal_solve(self, j, G, transpose, s=None):
        D = self.sn[j].D
        if not D.hierarchical:
            return dense.solve_lower_T(D.L, G) if transpose else dense.solve_lower(D.L, G)
        t = D.tree
        s = t.root if s is None else s
        if t.leaf[s]:
            L = D.leafL[s]
            return dense.solve_lower_T(L, G) if transpose else dense.solve_lower(L, G)
        n1 = t.mid[s] - t.lo[s]
        G1, G2 = G[:n1], G[n1:]
        s1, s2 = t.left[s], t.right[s]
        if transpose:
            G2 = self.diagonal_solve(j, G2, True, s2)
            G1 = G1 - D.U[s] @ (D.V[s].T @ G2)
            G1 = self.diagonal_solve(j, G1, True, s1)
        else:
            G1 = self.diagonal_solve(j, G1, False, s1)
            G2 = G2 - D.V[s] @ (D.U[s].T @ G1)
            G2 = self.diagonal_solve(j, G2, False, s2)
        return np.vstack([G1, G2])

    # ----------------------------------------------------------- Alg. 2 / transpose
    def offdiag_multiply(self, j, G):
        """B = L^O_j G for G in R^{|C_j| x r} (Alg. 2)."""
        an = self.an
        c0, c1 = an.cols(j)
        Rj = an.sym.rows[j]
        Cj = np.arange(c0, c1)
        G = self.diagonal_solve(j, G, transpose=True)
        W = an.A_block(Rj, Cj) @ G
        normal, blocks = self._split_desc(j)
        for k, pD, pO in normal:
            Rk = an.sym.rows[k]
            G_sub = gather_rows(G, Cj, Rk[pD])
            T = self.lo_apply(k, pO, pD, G_sub)
            W -= scatter_rows(T, Rk[pO], Rj)
        for b in blocks:
            W -= self._ib_mult(b, Rj, Cj, G)
        return W

    def offdiag_multiply_T(self, j, G):
        """B = (L^O_j)^T G for G in R^{|R_j| x r}."""
        an = self.an
        c0, c1 = an.cols(j)
        Rj = an.sym.rows[j]
        Cj = np.arange(c0, c1)
        W = an.A_block(Rj, Cj).T @ G
        normal, blocks = self._split_desc(j)
        for k, pD, pO in normal:
            Rk = an.sym.rows[k]
            G_sub = gather_rows(G, Rj, Rk[pO])
            T = self.lo_apply(k, pD, pO, G_sub)
            W -= scatter_rows(T, Rk[pD], Cj)
        for b in blocks:
            W -= self._ib_mult(b, Cj, Rj, G)
        return self.diagonal_solve(j, W, transpose=False)

    # ----------------------------------------------------------- adaptive range finder
    def _range_finder(self, m, c, tol, block_id, mult, mult_T, cap=None):
        """Shared body of Alg. 3 and approximateDiagonalBlock: returns (V, U).
        cap: largest rank (fixed-rank form, tol = 0); None: min(m, c)."""
        opts = self.an.opts
        b = opts.sample_block
        maxr = min(m, c) if cap is None else min(m, c, cap)
        U = np.zeros((c, 0))
        y1 = None
        t = 0
        while U.shape[1] < maxr:
            G = gaussian_block(m, b, opts.seed, block_id, t, self.restarts)
            Y = mult_T(G)
            for _ in range(opts.power_iters):
                Y = mult_T(mult(Y))
            if y1 is None:
                y1 = np.linalg.norm(Y)
            Yh = Y - U @ (U.T @ Y)
            Yh = Yh - U @ (U.T @ Yh)
            if np.linalg.norm(Yh) <= tol * y1:
                break
            Q = dense.householder_q(Yh[:, :min(b, maxr - U.shape[1])])
            Q = Q - U @ (U.T @ Q)
            Q = dense.householder_q(Q)
            U = np.hstack([U, Q])
            t += 1
        V = mult(U)
        return V, U

    def approximate_offdiag(self, j):
        """Alg. 3 (adaptive): L^O_j ~= V_j U_j^T with orthonormal U_j."""
        an = self.an
        c0, c1 = an.cols(j)
        m = an.sym.rows[j].size
        cap = rank_heuristic(m, c1 - c0, self.alpha_O, self.p) if self.fixed_rank else None
        V, U = self._range_finder(m, c1 - c0, self.tol, (j << 12) | 0,
                                  lambda G: self.offdiag_multiply(j, G),
                                  lambda G: self.offdiag_multiply_T(j, G), cap)
        s = self.sn[j]
        s.V, s.U, s.Uprod = V, U, U.T @ U

    # ----------------------------------------------------------- Alg. 5 / transpose
    def _desc_rows_in(self, j, k, lo, hi):
        """Positions p in R_k whose row lies in global range [lo, hi) (inside C_j)."""
        Rk = self.an.sym.rows[k]
        return np.nonzero((Rk >= lo) & (Rk < hi))[0]

    def _ancestor_blocks(self, j, s):
        """Blocks p on the path from s to the root with p < s (they precede s)."""
        t = self.sn[j].D.tree
        p = t.parent[s]
        out = []
        while p:
            if p < s:
                out.append(p)
            p = t.parent[p]
        return out

    def diagonal_multiply(self, j, s, G):
        """L^D_{j,s} G for internal block s (Alg. 5); G has |C^D_{j,s}| rows."""
        an = self.an
        D = self.sn[j].D
        t = D.tree
        c0, _ = an.cols(j)
        r0, r1 = t.rows(s)
        q0, q1 = t.cols(s)
        G = self.diagonal_solve(j, G, True, t.left[s])
        W = an.A_block(np.arange(c0 + r0, c0 + r1), np.arange(c0 + q0, c0 + q1)) @ G
        normal, blocks = self._split_desc(j)
        for b in blocks:
            W -= self._ib_mult(b, np.arange(c0 + r0, c0 + r1), np.arange(c0 + q0, c0 + q1), G)
        for k, _, _ in normal:
            Rk = an.sym.rows[k]
            pr = self._desc_rows_in(j, k, c0 + r0, c0 + r1)
            pc = self._desc_rows_in(j, k, c0 + q0, c0 + q1)
            if pr.size and pc.size:
                T = self.lo_apply(k, pr, pc, G[Rk[pc] - (c0 + q0)])
                W[Rk[pr] - (c0 + r0)] -= T
        for p in self._ancestor_blocks(j, s):
            pr0, _ = t.rows(p)
            Rsub = np.arange(r0, r1) - pr0                       # alignSet(R^D_s, R^D_p)
            Csub = np.arange(q0, q1) - pr0                       # alignSet(C^D_s, R^D_p)
            Up = D.U[p].T @ D.U[p]
            T = D.V[p][Csub].T @ G
            T = Up @ T
            W -= D.V[p][Rsub] @ T
        return W

    def diagonal_multiply_T(self, j, s, G):
        """(L^D_{j,s})^T G for internal block s; G has |R^D_{j,s}| rows."""
        an = self.an
        D = self.sn[j].D
        t = D.tree
        c0, _ = an.cols(j)
        r0, r1 = t.rows(s)
        q0, q1 = t.cols(s)
        W = an.A_block(np.arange(c0 + r0, c0 + r1), np.arange(c0 + q0, c0 + q1)).T @ G
        normal, blocks = self._split_desc(j)
        for b in blocks:
            W -= self._ib_mult(b, np.arange(c0 + q0, c0 + q1), np.arange(c0 + r0, c0 + r1), G)
        for k, _, _ in normal:
            Rk = an.sym.rows[k]
            pr = self._desc_rows_in(j, k, c0 + r0, c0 + r1)
            pc = self._desc_rows_in(j, k, c0 + q0, c0 + q1)
            if pr.size and pc.size:
                T = self.lo_apply(k, pc, pr, G[Rk[pr] - (c0 + r0)])
                W[Rk[pc] - (c0 + q0)] -= T
        for p in self._ancestor_blocks(j, s):
            pr0, _ = t.rows(p)
            Rsub = np.arange(r0, r1) - pr0
            Csub = np.arange(q0, q1) - pr0
            Up = D.U[p].T @ D.U[p]
            T = D.V[p][Rsub].T @ G
            T = Up @ T
            W -= D.V[p][Csub] @ T
        return self.diagonal_solve(j, W, False, t.left[s])

    def approximate_diagonal_block(self, j, s):
        D = self.sn[j].D
        t = D.tree
        r0, r1 = t.rows(s)
        q0, q1 = t.cols(s)
        cap = rank_heuristic(r1 - r0, q1 - q0, self.alpha_D, self.p) if self.fixed_rank else None
        V, U = self._range_finder(r1 - r0, q1 - q0, self.tol_D, (j << 12) | s,
                                  lambda G: self.diagonal_multiply(j, s, G),
                                  lambda G: self.diagonal_multiply_T(j, s, G), cap)
        D.V[s], D.U[s] = V, U

    # ----------------------------------------------------------- Alg. 6
    def factor_diagonal(self, j, s):
        an = self.an
        D = self.sn[j].D
        t = D.tree
        c0, _ = an.cols(j)
        r0, r1 = t.rows(s)
        gl = np.arange(c0 + r0, c0 + r1)
        S = an.A_block(gl, gl)
        normal, blocks = self._split_desc(j)
        for b in blocks:                                     # a sub-block of L(R_B, C_B), dropped after
            Lr = self._ib_L(b, gl)
            S -= Lr @ Lr.T
        for k, _, _ in normal:
            Rk = an.sym.rows[k]
            pr = self._desc_rows_in(j, k, c0 + r0, c0 + r1)
            if pr.size:
                loc = Rk[pr] - (c0 + r0)
                S[np.ix_(loc, loc)] -= self.lo_pair_product(k, pr, pr)
        for p in self._ancestor_blocks(j, s):
            pr0, _ = t.rows(p)
            Rsub = np.arange(r0, r1) - pr0
            Up = D.U[p].T @ D.U[p]
            S -= D.V[p][Rsub] @ (Up @ D.V[p][Rsub].T)
        D.leafL[s] = dense.cholesky(S)

    # ----------------------------------------------------------- Alg. 1
    def schur_blocks(self, j, with_offdiag=True):
        """U^D_j and U^O_j (Eqs. schurDiag / schurOffDiag)."""
        an = self.an
        c0, c1 = an.cols(j)
        Cj = np.arange(c0, c1)
        Rj = an.sym.rows[j]
        UD = an.A_block(Cj, Cj)
        UO = an.A_block(Rj, Cj) if with_offdiag else None
        normal, blocks = self._split_desc(j)
        for b in blocks:                                     # sub-blocks of L(R_B, C_B), dropped after
            Lc = self._ib_L(b, Cj)
            UD -= Lc @ Lc.T
            if with_offdiag and Rj.size:
                UO -= self._ib_L(b, Rj) @ Lc.T
        for k, pD, pO in normal:
            Rk = an.sym.rows[k]
            dloc = positions(Rk[pD], Cj)                         # scatter(., R^D_glob, C_j, R^D_glob, C_j)
            UD[np.ix_(dloc, dloc)] -= self.lo_pair_product(k, pD, pD)
            if with_offdiag and pO.size:
                oloc = positions(Rk[pO], Rj)                     # scatter(., R^O_glob, R_j, R^D_glob, C_j)
                UO[np.ix_(oloc, dloc)] -= self.lo_pair_product(k, pO, pD)
        return UD, UO

    def factor_supernode(self, j):
        """Alg. 1: L^D_j = chol(U^D_j), L^O_j = U^O_j (L^D_j)^{-T}."""
        UD, UO = self.schur_blocks(j)
        s = self.sn[j]
        s.D = DiagFactor()
        s.D.L = dense.cholesky(UD)
        s.LO = dense.solve_lower(s.D.L, UO.T).T

    def factor_compressed(self, j):
        an = self.an
        s = self.sn[j]
        s.compressed = True
        tree = an.ordering.trees[j]
        if self.diag_compress and tree is not None:
            s.D = DiagFactor(tree)
            for b in range(1, tree.nblocks + 1):
                if tree.leaf[b]:
                    self.factor_diagonal(j, b)
                else:
                    self.approximate_diagonal_block(j, b)
        else:
            UD, _ = self.schur_blocks(j, with_offdiag=False)
            s.D = DiagFactor()
            s.D.L = dense.cholesky(UD)
        if an.sym.rows[j].size:
            self.approximate_offdiag(j)
        else:
            c = an.cols(j)[1] - an.cols(j)[0]
            s.V, s.U, s.Uprod = np.zeros((0, 0)), np.zeros((c, 0)), np.zeros((0, 0))

    def is_compressed(self, j):
        an = self.an
        c0, c1 = an.cols(j)
        return self.compress and an.ordering.kinds[j] == "sep" and (c1 - c0) >= an.opts.tau_O

    def run(self):
        self.sn = [SupernodeFactor() for _ in range(self.an.nsuper)]
        self._find_interior_blocks()
        for j in range(self.an.nsuper):
            b = int(self.iblock_of[j])
            if b >= 0:
                B = self.iblocks[b]
                if j == B["last"]:                           # Eq. interiorDiagonalDef
                    CB = np.arange(B["c0"], B["c1"])
                    B["L"] = dense.cholesky(self.an.A_block(CB, CB))
                continue
            if self.is_compressed(j):
                self.factor_compressed(j)
            else:
                self.factor_supernode(j)


def _restart_loop(f: Factor, loosen) -> Factor:
    """Section 5.3: on an indefinite diagonal block, make diagonal compression more
    accurate (``loosen``) and factor again; after max_restarts restarts, switch it off."""
    attempt = 0
    while True:
        f.restarts = attempt
        try:
            f.run()
            return f
        except NotPositiveDefinite:
            if not f.diag_compress:
                raise
            attempt += 1
            if attempt <= f.an.opts.max_restarts:
                loosen(f)
            else:
                f.diag_compress = False


def factor(an: Analysis, tol: float) -> Factor:
    """Factor with the Section 5.3 restart loop (tolerance form: tol_D <- tol_D / 1.25)."""
    f = Factor(an)
    f.compress = tol > 0
    f.tol = tol if tol > 0 else 0.0
    f.tol_D = f.tol
    f.diag_compress = bool(an.opts.diag_compress and f.compress)

    def loosen(g):
        g.tol_D = g.tol_D / 1.25
    return _restart_loop(f, loosen)


def factor_fixed_rank(an: Analysis, alpha_O: float, alpha_D: float = 0.5, p: int = 8) -> Factor:
    """Factor with the ranks of Eq. rankFunction (Section 5.2) and the Section 5.3 restart
    alpha^D <- 1.25 alpha^D."""
    if not (alpha_O >= 0 and alpha_D >= 0 and p >= 0):
        raise ValueError("alpha_O, alpha_D and p must be >= 0")
    f = Factor(an)
    f.compress = True
    f.fixed_rank = True
    f.alpha_O, f.alpha_D, f.p = float(alpha_O), float(alpha_D), int(p)
    f.diag_compress = bool(an.opts.diag_compress)

    def loosen(g):
        g.alpha_D = g.alpha_D * 1.25
    return _restart_loop(f, loosen)


# ----------------------------------------------------------------------------- solve

def apply_preconditioner(f: Factor, r: np.ndarray) -> np.ndarray:
    """z = P (L L^T)^{-1} P^T r with the approximate factor: forward, then backward
    substitution over supernodes (Section 1: "two triangular solves")."""
    an = f.an
    perm = an.ordering.perm
    y = np.array(r[perm], dtype=np.float64)
    M = an.nsuper
    ib = f.iblock_of if f.iblock_of is not None else -np.ones(M, dtype=np.int64)
    for j in range(M):
        c0, c1 = an.cols(j)
        Rj = an.sym.rows[j]
        if ib[j] >= 0:                                       # interior block, once at its first supernode
            B = f.iblocks[int(ib[j])]
            if j == B["first"]:
                b0, b1 = B["c0"], B["c1"]
                y[b0:b1] = dense.solve_lower(B["L"], y[b0:b1, None])[:, 0]
                if B["RB"].size:
                    t = dense.solve_lower_T(B["L"], y[b0:b1, None])
                    y[B["RB"]] -= (an.A_block(B["RB"], np.arange(b0, b1)) @ t)[:, 0]
            continue
        y[c0:c1] = f.diagonal_solve(j, y[c0:c1, None], transpose=False)[:, 0]
        if Rj.size:
            s = f.sn[j]
            if s.compressed:
                y[Rj] -= s.V @ (s.U.T @ y[c0:c1])
            else:
                y[Rj] -= s.LO @ y[c0:c1]
    for j in range(M - 1, -1, -1):
        c0, c1 = an.cols(j)
        Rj = an.sym.rows[j]
        if ib[j] >= 0:                                       # interior block, once at its root
            B = f.iblocks[int(ib[j])]
            if j == B["last"]:
                b0, b1 = B["c0"], B["c1"]
                if B["RB"].size:
                    t = an.A_block(B["RB"], np.arange(b0, b1)).T @ y[B["RB"], None]
                    y[b0:b1] -= dense.solve_lower(B["L"], t)[:, 0]
                y[b0:b1] = dense.solve_lower_T(B["L"], y[b0:b1, None])[:, 0]
            continue
        if Rj.size:
            s = f.sn[j]
            if s.compressed:
                y[c0:c1] -= s.U @ (s.V.T @ y[Rj])
            else:
                y[c0:c1] -= s.LO.T @ y[Rj]
        y[c0:c1] = f.diagonal_solve(j, y[c0:c1, None], transpose=True)[:, 0]
    z = np.empty_like(y)
    z[perm] = y
    return z


def pcg(A: sp.csr_matrix, b: np.ndarray, precond, rtol: float = 1e-8, max_iter: int = 1000):
    """Hestenes-Stiefel PCG from x0 = 0 (Section 6.1 uses PCG to a relative l2
    residual).  Stops when the recursive ||r||/||b|| <= rtol and the true residual
    ||b - A x||/||b|| confirms it.  Returns (x, iterations, true relative residual,
    converged) with iterations = number of CG steps (products with A)."""
    x = np.zeros_like(b)
    r = b.copy()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, 0.0, True
    z = precond(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, max_iter + 1):
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        if np.linalg.norm(r) / nb <= rtol:
            true_rel = np.linalg.norm(b - A @ x) / nb
            if true_rel <= rtol:
                return x, it, true_rel, True
        z = precond(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, max_iter, np.linalg.norm(b - A @ x) / nb, False


def analyze(n, row_ptr, col_idx, val, coords, opts: Options | None = None) -> Analysis:
    return Analysis(n, row_ptr, col_idx, val, coords, opts or Options())


def solve(an: Analysis, f: Factor, b: np.ndarray, rtol=1e-8, max_iter=1000):
    return pcg(an.A, b, lambda r: apply_preconditioner(f, r), rtol, max_iter)


def factor_bytes(f: Factor) -> int:
    """Bytes of the stored factor in FP64 (dense blocks, V and U factors)."""
    tot = 0
    an = f.an
    for j, s in enumerate(f.sn):
        if f.iblock_of is not None and f.iblock_of[j] >= 0:
            # Section 5.1: only the in-block part of the supernodal panel is stored
            B = f.iblocks[int(f.iblock_of[j])]
            c0, c1 = an.cols(j)
            Rj = an.sym.rows[j]
            tot += (c1 - c0) * (c1 - c0 + 1) // 2 + (c1 - c0) * int(np.sum(Rj < B["c1"]))
            continue
        D = s.D
        if D.hierarchical:
            tot += sum(L.size for L in D.leafL.values())
            tot += sum(D.V[b].size + D.U[b].size for b in D.V)
        else:
            tot += D.L.shape[0] * (D.L.shape[0] + 1) // 2
        if s.compressed:
            tot += s.V.size + s.U.size
        else:
            tot += s.LO.size
    return 8 * tot
