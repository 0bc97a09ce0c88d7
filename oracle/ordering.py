"""Fill-reducing ordering and within-separator ordering (oracle; test infrastructure).

* Nested dissection, Section 2.2 / 3.1: separators are ordered after the two
  subdomains they separate; every nested-dissection tree node (leaf subdomain or
  separator) becomes one supernode.  The paper does not name its partitioner;
  the reading here is recursive coordinate bisection of lattice points:

  - a point set with at most ``leaf_size`` nodes is a leaf;
  - otherwise split on the axis of largest bounding-box extent (ties: lowest
    axis), at plane ``m = lo + ext // 2`` with ``ext = max - min + 1``; points
    with coordinate < m form the left part, == m the separator, > m the right;
  - postorder numbering: left subtree, right subtree, separator;
  - inside a leaf or separator, nodes are in lexicographic (z, y, x) order,
    ties by original index.

* Within-separator geometric ordering, Section 4.1 (Fig. "diagOrdering"): for a
  separator whose diagonal block is compressed, sort its nodes stably along the
  longest bounding-box axis (ties: lowest axis), split into halves (the left gets
  floor(n/2) nodes) and recurse until a part has at most ``tau_D`` unknowns.  The
  leaves become contiguous runs of the separator's columns.

* The block tree of a hierarchically compressed diagonal block, Section 4.1
  (Eq. "ldjLabel"): tree nodes are labelled by an in-order traversal.  Leaves are
  dense diagonal blocks; an internal node s is the off-diagonal block with the
  rows of its right subtree and the columns of its left subtree.  Reading: the
  paper's 7-block example names the root's children "3 and 6"; the block layout
  it draws makes them 2 and 6, which is what an in-order labelling gives.

* Graph nested dissection (general sparsity; the paper's partitioner is unnamed, and
  its non-grid examples need one that does not assume a lattice).  Reading: recursive
  bisection of the node graph guided by real node positions X (given, or the spectral
  coordinates below):

  - a node set with at most ``leaf_size`` nodes is a leaf;
  - otherwise take the axis of largest bounding-box extent of X (ties: lowest axis),
    sort the nodes by (X[axis], node id) and cut at the median: L = the first
    floor(size/2) nodes, R = the rest;
  - the vertex separator is the boundary of the cut on one side: S_L = nodes of L
    with a neighbour in R, S_R = nodes of R with a neighbour in L; S = S_L if
    |S_L| <= |S_R| else S_R (removing S leaves no edge between the two halves);
  - recurse on L minus S and R minus S, then the separator (postorder); inside a leaf or
    separator, nodes are in ascending id order.

* Spectral coordinates, Section 4.3: where no positions are given, node i sits at
  (v1_i, v2_i, v3_i) for the three lowest eigenvectors of the node graph's Laplacian
  (off-diagonal -1 per edge, diagonal = degree).  Reading: per connected component,
  skipping that component's constant null vector (it carries no position); the
  oracle solves the dense eigenproblem.

Unknowns: with ``dof`` unknowns per node, node i owns unknowns dof*i .. dof*i+dof-1,
which stay adjacent.  ``tau_D`` and supernode sizes count unknowns; the leaf
rule counts nodes.
"""
from __future__ import annotations

import numpy as np


def nested_dissection(coords: np.ndarray, leaf_size: int = 64, dof: int = 1, components=None):
    """Return (node_order, parts): node_order lists node ids in elimination order and
    parts is a list of (kind, node_ids) per supernode, kind in {"leaf", "sep"}.

    ``components`` (optional, one label per node): the nodes of each connected
    component of the matrix graph are dissected on their own, components in order of
    their smallest node id (a block-diagonal stack of independent systems becomes a
    forest of elimination trees)."""
    P = np.rint(np.asarray(coords)[::dof]).astype(np.int64)
    parts: list[tuple[str, np.ndarray]] = []

    def lex(ids):
        pts = P[ids]
        return ids[np.lexsort((ids, pts[:, 0], pts[:, 1], pts[:, 2]))]

    def rec(ids):
        if ids.size == 0:
            return
        if ids.size <= leaf_size:
            parts.append(("leaf", lex(ids)))
            return
        pts = P[ids]
        lo = pts.min(axis=0)
        ext = pts.max(axis=0) - lo + 1
        ax = int(np.argmax(ext))                    # first maximum = lowest axis on ties
        m = lo[ax] + ext[ax] // 2
        rec(ids[pts[:, ax] < m])
        rec(ids[pts[:, ax] > m])
        sep = ids[pts[:, ax] == m]
        if sep.size:
            parts.append(("sep", lex(sep)))

    if components is None:
        rec(np.arange(P.shape[0], dtype=np.int64))
    else:
        comp = np.asarray(components)
        first = {}
        for i, c in enumerate(comp.tolist()):
            first.setdefault(c, i)
        for c in sorted(first, key=first.get):
            rec(np.nonzero(comp == c)[0].astype(np.int64))
    order = np.concatenate([p[1] for p in parts])
    return order, parts


def _component_order(nnodes, components):
    """Node id arrays of the connected components, in order of their smallest node."""
    if components is None:
        return [np.arange(nnodes, dtype=np.int64)]
    comp = np.asarray(components)
    first = {}
    for i, c in enumerate(comp.tolist()):
        first.setdefault(c, i)
    return [np.nonzero(comp == c)[0].astype(np.int64) for c in sorted(first, key=first.get)]


def graph_nested_dissection(adj_ptr, adj_idx, X, leaf_size: int = 64, components=None):
    """Graph nested dissection of the node graph (CSR adjacency without self loops,
    symmetric) guided by node positions X (nodes x 3, real).  Returns parts as
    ``nested_dissection`` does."""
    adj_ptr = np.asarray(adj_ptr)
    adj_idx = np.asarray(adj_idx)
    X = np.asarray(X, dtype=np.float64)
    nnodes = X.shape[0]
    parts: list[tuple[str, np.ndarray]] = []
    side = np.zeros(nnodes, dtype=np.int8)      # scratch: 1 = in L, 2 = in R

    def boundary(A, other):
        """Nodes of A with a neighbour marked ``other``."""
        out = []
        for v in A.tolist():
            nb = adj_idx[adj_ptr[v]:adj_ptr[v + 1]]
            if np.any(side[nb] == other):
                out.append(v)
        return np.array(out, dtype=np.int64)

    def rec(ids):
        if ids.size == 0:
            return
        if ids.size <= leaf_size:
            parts.append(("leaf", np.sort(ids)))
            return
        pts = X[ids]
        ext = pts.max(axis=0) - pts.min(axis=0)
        ax = int(np.argmax(ext))                    # first maximum = lowest axis on ties
        srt = ids[np.lexsort((ids, pts[:, ax]))]    # by (X[ax], id)
        h = ids.size // 2
        L, R = srt[:h], srt[h:]
        side[L] = 1
        side[R] = 2
        SL, SR = boundary(L, 2), boundary(R, 1)
        side[ids] = 0
        S = SL if SL.size <= SR.size else SR
        inS = np.zeros(nnodes, dtype=bool)
        inS[S] = True
        rec(np.sort(L[~inS[L]]))
        rec(np.sort(R[~inS[R]]))
        if S.size:
            parts.append(("sep", np.sort(S)))

    for ids in _component_order(nnodes, components):
        rec(ids)
    order = np.concatenate([p[1] for p in parts]) if parts else np.zeros(0, dtype=np.int64)
    return order, parts


def spectral_coordinates(adj_ptr, adj_idx, components=None) -> np.ndarray:
    """Section 4.3: positions from the three lowest non-constant eigenvectors of the
    graph Laplacian, per connected component (dense eigensolver: small graphs only).
    Components with fewer than 4 nodes keep the missing coordinates at 0."""
    adj_ptr = np.asarray(adj_ptr)
    adj_idx = np.asarray(adj_idx)
    nnodes = adj_ptr.size - 1
    X = np.zeros((nnodes, 3))
    for ids in _component_order(nnodes, components):
        m = ids.size
        if m < 2:
            continue
        if m > 6000:
            raise NotImplementedError("the oracle's dense eigensolver is for small graphs")
        loc = -np.ones(nnodes, dtype=np.int64)
        loc[ids] = np.arange(m)
        Lap = np.zeros((m, m))
        for a, v in enumerate(ids.tolist()):
            nb = loc[adj_idx[adj_ptr[v]:adj_ptr[v + 1]]]
            Lap[a, nb] = -1.0
            Lap[a, a] = nb.size
        w, V = np.linalg.eigh(Lap)
        k = min(3, m - 1)
        X[ids, :k] = V[:, 1:1 + k]                 # column 0: the constant null vector
    return X


def node_graph(n, row_ptr, col_idx, dof: int = 1):
    """CSR adjacency (sorted, no self loops) of the node graph: nodes u != v adjacent
    when some unknown of u couples with some unknown of v in A's pattern."""
    rp = np.asarray(row_ptr)
    ci = np.asarray(col_idx)
    rows = np.repeat(np.arange(n), np.diff(rp)) // dof
    cols = ci // dof
    keep = rows != cols
    pairs = np.unique(np.stack([rows[keep], cols[keep]], axis=1), axis=0)
    nn = n // dof
    ptr = np.zeros(nn + 1, dtype=np.int64)
    np.add.at(ptr, pairs[:, 0] + 1, 1)
    return np.cumsum(ptr), pairs[:, 1].astype(np.int64)


class BlockTree:
    """In-order labelled binary tree over the columns of one diagonal block.

    For label s (1-based): ``leaf[s]``; ``lo[s], hi[s]`` the local column range of
    the subtree; for internal s, ``mid[s]`` splits it into the left range
    [lo, mid) (the block's columns) and the right range [mid, hi) (its rows);
    ``left[s]``, ``right[s]``, ``parent[s]`` (0 = none)."""

    def __init__(self):
        self.leaf = {}
        self.lo = {}
        self.hi = {}
        self.mid = {}
        self.left = {}
        self.right = {}
        self.parent = {}
        self.root = 0
        self.nblocks = 0

    def rows(self, s):
        """Local row range of block s (Section 4.1: R^D_{j,s})."""
        return (self.lo[s], self.hi[s]) if self.leaf[s] else (self.mid[s], self.hi[s])

    def cols(self, s):
        """Local column range of block s (C^D_{j,s})."""
        return (self.lo[s], self.hi[s]) if self.leaf[s] else (self.lo[s], self.mid[s])


def geometric_split(node_ids: np.ndarray, coords: np.ndarray, tau_D: int, dof: int = 1):
    """Reorder one separator's nodes (Section 4.1) and build its block tree.

    Returns (new_node_order, BlockTree) with ranges counted in unknowns."""
    P = np.asarray(coords)[::dof]
    leaves: list[np.ndarray] = []
    tree = BlockTree()
    counter = [0]

    def rec(ids, lo):
        """Split recursively; returns (label, hi). Labels assigned in-order."""
        if ids.size * dof <= tau_D:
            counter[0] += 1
            s = counter[0]
            leaves.append(ids)
            tree.leaf[s] = True
            tree.lo[s], tree.hi[s] = lo, lo + ids.size * dof
            tree.left[s] = tree.right[s] = 0
            return s, tree.hi[s]
        pts = P[ids]
        ext = pts.max(axis=0) - pts.min(axis=0)
        ax = int(np.argmax(ext))
        srt = ids[np.argsort(pts[:, ax], kind="stable")]
        h = ids.size // 2
        sl, mid = rec(srt[:h], lo)
        counter[0] += 1
        s = counter[0]
        sr, hi = rec(srt[h:], mid)
        tree.leaf[s] = False
        tree.lo[s], tree.mid[s], tree.hi[s] = lo, mid, hi
        tree.left[s], tree.right[s] = sl, sr
        tree.parent[sl] = s
        tree.parent[sr] = s
        return s, hi

    root, _ = rec(np.asarray(node_ids), 0)
    tree.root = root
    tree.parent[root] = 0
    tree.nblocks = counter[0]
    return np.concatenate(leaves), tree


class Ordering:
    """perm[new] = old unknown; snode_ptr[M+1] column boundaries; kinds; block trees
    (None unless the supernode's diagonal block may be hierarchically compressed)."""

    def __init__(self, perm, snode_ptr, kinds, trees):
        self.perm = perm
        self.snode_ptr = snode_ptr
        self.kinds = kinds
        self.trees = trees

    @property
    def nsuper(self):
        return len(self.snode_ptr) - 1


def order(coords: np.ndarray, dof: int = 1, leaf_size: int = 64, tau_O: int = 256,
          tau_D: int = 256, components=None, graph=None) -> Ordering:
    """Nested dissection, then the Section 4.1 reorder of every separator that will
    be compressed (>= tau_O unknowns, Section 3.1: "at least tau_O") and whose
    diagonal block is larger than tau_D.

    graph: None for the lattice bisection; (adj_ptr, adj_idx) of the node graph for
    graph nested dissection guided by ``coords`` (one row per unknown, as for the
    lattice form)."""
    if graph is None:
        _, parts = nested_dissection(coords, leaf_size, dof, components)
    else:
        _, parts = graph_nested_dissection(graph[0], graph[1], np.asarray(coords)[::dof], leaf_size,
                                           components)
    node_blocks = []
    trees = []
    for kind, ids in parts:
        nc = ids.size * dof
        if kind == "sep" and nc >= tau_O and nc > tau_D:
            ids, tree = geometric_split(ids, coords, tau_D, dof)
            trees.append(tree)
        else:
            trees.append(None)
        node_blocks.append(ids)
    nodes = np.concatenate(node_blocks)
    perm = (dof * nodes[:, None] + np.arange(dof)[None, :]).ravel()
    sizes = np.array([b.size * dof for b in node_blocks], dtype=np.int64)
    snode_ptr = np.concatenate([[0], np.cumsum(sizes)])
    return Ordering(perm, snode_ptr, [p[0] for p in parts], trees)
