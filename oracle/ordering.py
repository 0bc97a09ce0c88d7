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
          tau_D: int = 256, components=None) -> Ordering:
    """Nested dissection, then the Section 4.1 reorder of every separator that will
    be compressed (>= tau_O unknowns, Section 3.1: "at least tau_O") and whose
    diagonal block is larger than tau_D."""
    _, parts = nested_dissection(coords, leaf_size, dof, components)
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
