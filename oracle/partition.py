"""Multilevel partition for spaND on grid problems (oracle side).

Test infrastructure only (see ``oracle/__init__``).

The paper's spaND partitioning (§3) splits the unknowns, level by level, into
*interiors* -- eliminated by block Cholesky at that level -- and *interfaces*,
small subsets that separate the interiors and are scaled and sparsified.  The
paper defines it on the graph of A and defers the details to the spaND paper;
for grid problems given with coordinates this module builds the geometric
equivalent:

Nested dissection.  The grid box is bisected recursively down to
depth ``ell-1``.  The node at depth ``d`` cuts coordinate ``d mod D`` at the
``floor(cnt/2)``-th smallest distinct coordinate value present in its box;
vertices on the cut plane form the node's separator, vertices strictly below /
above go to the lower / upper child.  Nodes are numbered heap-style (children
of ``i`` are ``2i+1`` and ``2i+2``), so node ids are in breadth-first order
with the lower child first.  A separator of a depth-``d`` node has level
``ell-1-d``; the leaves (depth ``ell-1``) have level 0.

Clusters.  At stage ``k`` every vertex of level ``>= k`` is live.
A vertex of level ``k`` belongs to the single interior cluster of its node.  A
vertex ``v`` of level ``m > k`` on the separator of node ``S`` is classified
by walking down the lower-child subtree of ``S`` while the node depth is
``< ell-1-k``: at a node whose cut is parallel to ``S`` the walk goes to the
upper child (the side that touches ``S``) and records nothing; otherwise it
records the comparison of ``v``'s coordinate with the cut (0: below, 1: on,
2: above), goes to the lower child on 0, the upper child on 2, and stops on 1
(``v`` lies on the crossing line or point with that descendant separator,
which makes it its own small cluster).  The cluster is ``(S, key)``, where
``key[j]`` is the comparison recorded at depth ``j`` or -1.  Cluster ids at a
stage are the lexicographic order of ``(S, key)``.

Because the cut dimension cycles and sibling boxes have equal extents in all
non-cut dimensions, the walk in the lower subtree sees the same non-parallel
cuts as the upper subtree would, so a cluster touches at most one sub-box on
each side of ``S``.  Stage ``k+1`` clusters are unions of stage ``k`` clusters
(the key only loses its deepest entries).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def node_depth(i: int) -> int:
    """Depth of heap-numbered node ``i`` (root 0 has depth 0)."""
    return int(np.floor(np.log2(i + 1) + 1e-12))


@dataclass
class NDTree:
    """Geometric nested-dissection tree to depth ``nlevels - 1``."""

    nlevels: int
    dim: int
    coords: np.ndarray
    cut_dim: dict = field(default_factory=dict)  # internal node -> coordinate index
    cut_val: dict = field(default_factory=dict)  # internal node -> cut value
    node_of: np.ndarray | None = None  # vertex -> node (separator node or leaf)
    level_of: np.ndarray | None = None  # vertex -> level

    @property
    def depth_max(self) -> int:
        return self.nlevels - 1


def nested_dissection(coords: np.ndarray, nlevels: int) -> NDTree:
    """Recursive coordinate bisection; raises ValueError on an empty box."""
    coords = np.asarray(coords, dtype=np.float64)
    n, dim = coords.shape
    if nlevels < 1:
        raise ValueError("nlevels must be >= 1")
    tree = NDTree(nlevels=nlevels, dim=dim, coords=coords)
    node_of = np.full(n, -1, dtype=np.int64)
    level_of = np.full(n, -1, dtype=np.int64)
    dmax = nlevels - 1
    frontier = [(0, np.arange(n, dtype=np.int64))]
    for depth in range(dmax + 1):
        nxt = []
        for node, verts in frontier:
            if verts.size == 0:
                raise ValueError(f"empty nested-dissection box at node {node}")
            if depth == dmax:
                node_of[verts] = node
                level_of[verts] = 0
                continue
            c = depth % dim
            x = coords[verts, c]
            vals = np.unique(x)
            cut = vals[len(vals) // 2]
            tree.cut_dim[node] = c
            tree.cut_val[node] = cut
            sep = verts[x == cut]
            node_of[sep] = node
            level_of[sep] = dmax - depth
            nxt.append((2 * node + 1, verts[x < cut]))
            nxt.append((2 * node + 2, verts[x > cut]))
        frontier = nxt
    tree.node_of = node_of
    tree.level_of = level_of
    return tree


def cluster_keys(tree: NDTree, k: int):
    """Cluster key of every live vertex at stage ``k``.

    Returns ``(live, keys)``: the live vertices (level >= k, ascending) and an
    int64 array of shape ``(len(live), 1 + ell)`` whose row is
    ``(node, key[0], ..., key[ell-1])``.  Rows compare lexicographically in the
    same order as the tuples ``(node, key)``.
    """
    ell = tree.nlevels
    nint = 2 ** (ell - 1) - 1  # internal nodes have ids < nint
    cut_dim = np.full(max(nint, 1), -1, dtype=np.int64)
    cut_val = np.zeros(max(nint, 1), dtype=np.float64)
    for node, c in tree.cut_dim.items():
        cut_dim[node] = c
        cut_val[node] = tree.cut_val[node]
    limit = ell - 1 - k  # the walk visits nodes of depth < limit

    def depth(i):
        return np.floor(np.log2(i + 1.0) + 1e-12).astype(np.int64)

    live = np.nonzero(tree.level_of >= k)[0].astype(np.int64)
    nodes = tree.node_of[live]
    key = np.full((live.size, ell), -1, dtype=np.int64)
    walk = tree.level_of[live] > k
    sdim = np.where(walk, cut_dim[np.where(walk, nodes, 0)], -1)
    cur = 2 * nodes + 1
    active = walk & (depth(cur) < limit)
    while active.any():
        idx = np.nonzero(active)[0]
        c = cur[idx]
        cd = cut_dim[c]
        par = cd == sdim[idx]  # cut parallel to the separator: go to the side touching it
        x = tree.coords[live[idx], cd]
        cv = cut_val[c]
        cmp = np.where(x < cv, 0, np.where(x > cv, 2, 1))
        cmp[par] = 2
        rec = ~par
        key[idx[rec], depth(c[rec])] = cmp[rec]
        cur[idx] = np.where(cmp == 0, 2 * c + 1, 2 * c + 2)
        stop = rec & (cmp == 1)
        active[idx[stop]] = False
        active[idx] &= depth(cur[idx]) < limit
    return live, np.concatenate([nodes[:, None], key], axis=1)


@dataclass
class StageClusters:
    """Clusters of one stage: sorted keys and vertex membership."""

    keys: list  # sorted cluster keys, each a tuple (node, key[0..ell-1])
    members: dict  # key -> ascending np.array of original vertices
    level: dict  # key -> level of its node


def stage_clusters(tree, k: int) -> StageClusters:
    """All live clusters at stage ``k``, in id (lexicographic key) order."""
    live, rows = tree_cluster_keys(tree, k)
    uniq, inv = np.unique(rows, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    order = np.argsort(inv, kind="stable")
    bounds = np.searchsorted(inv[order], np.arange(uniq.shape[0] + 1))
    keys = [tuple(int(t) for t in row) for row in uniq]
    members = {}
    level = {}
    for i, key in enumerate(keys):
        verts = live[order[bounds[i]:bounds[i + 1]]]
        members[key] = verts  # already ascending: live is ascending, sort is stable
        level[key] = int(tree.level_of[verts[0]])
    return StageClusters(keys=keys, members=members, level=level)


def greedy_colouring(order: list, adjacency: dict) -> dict:
    """Smallest-free-colour greedy colouring in the given vertex order."""
    colour: dict = {}
    for p in order:
        used = {colour[q] for q in adjacency.get(p, ()) if q in colour}
        c = 0
        while c in used:
            c += 1
        colour[p] = c
    return colour


# ---------------------------------------------------------------------------
# Algebraic nested dissection (general sparse SPD input, no coordinates).
#
# The node at depth d bisects its vertex set V by a breadth-first level
# structure of the subgraph of A induced on V: starting from the smallest
# vertex index, one sweep finds a far vertex (the smallest index at the
# largest distance), and the levels are the BFS distances from it.  With the
# vertices ordered by (distance, index) and unreached vertices (other
# components) last, the level L* of the median (position floor(|V|/2)) is the
# separator; smaller distances go to the lower child, larger distances and
# unreached vertices to the upper child.  (No edge joins the two children:
# BFS distances of adjacent vertices differ by at most one.)  If the median is
# unreached, the separator is empty and the reached vertices form the lower
# child.  Node numbering and levels are those of the geometric tree.
#
# Clusters.  Interfaces are keyed by the subdomains they touch: the reach
# R(v) of a separator vertex v is the set of leaves connected to v through
# vertices of strictly lower level (for a neighbour u of lower level, u's own
# leaf if u is a leaf vertex, else R(u)).  At stage k, with subdomains the
# subtrees of the depth ell-1-k nodes, an interface vertex v of node S has
# key = the sorted set of depth-(ell-1-k) ancestors of the leaves in R(v);
# its cluster is (S, key).  The key at stage k+1 is the set of parents of the
# key at stage k, so stage k+1 clusters are unions of stage k clusters.
# ---------------------------------------------------------------------------


@dataclass
class GraphNDTree:
    """Algebraic nested-dissection tree to depth ``nlevels - 1``."""

    nlevels: int
    node_of: np.ndarray  # vertex -> node (separator node or leaf)
    level_of: np.ndarray  # vertex -> level
    reach: list  # vertex -> sorted tuple of leaf ids (separator vertices; () for leaves)
    width: int  # largest reach set (>= 1): the padded key width

    @property
    def depth_max(self) -> int:
        return self.nlevels - 1


def bfs_levels(rowptr, colind, inset: np.ndarray, root: int) -> np.ndarray:
    """BFS distance from ``root`` of every vertex in the subgraph induced on
    ``inset`` (boolean mask); -1 for vertices not reached."""
    lev = np.full(inset.size, -1, dtype=np.int64)
    lev[root] = 0
    front = np.array([root], dtype=np.int64)
    d = 0
    while front.size:
        nb = np.concatenate([colind[rowptr[v]:rowptr[v + 1]] for v in front])
        nb = np.unique(nb)
        nb = nb[inset[nb] & (lev[nb] < 0)]
        d += 1
        lev[nb] = d
        front = nb.astype(np.int64)
    return lev


def graph_bisect(rowptr, colind, verts: np.ndarray):
    """(separator, lower, upper) of the ascending vertex array ``verts``."""
    n = rowptr.size - 1
    inset = np.zeros(n, dtype=bool)
    inset[verts] = True
    lev = bfs_levels(rowptr, colind, inset, int(verts[0]))
    lv = lev[verts]
    far = lv.max()
    r1 = int(verts[lv == far].min())
    lev = bfs_levels(rowptr, colind, inset, r1)
    lv = lev[verts]
    big = np.iinfo(np.int64).max
    key = np.where(lv < 0, big, lv)
    order = np.lexsort((verts, key))  # by (distance, index)
    med = key[order[verts.size // 2]]
    if med == big:
        return verts[:0], verts[lv >= 0], verts[lv < 0]
    return verts[key == med], verts[key < med], verts[key > med]


def graph_nested_dissection(rowptr, colind, nlevels: int) -> GraphNDTree:
    """Algebraic ND on the graph of a symmetric CSR pattern; raises ValueError
    on an empty leaf or subdomain."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    colind = np.asarray(colind, dtype=np.int64)
    n = rowptr.size - 1
    if nlevels < 1:
        raise ValueError("nlevels must be >= 1")
    node_of = np.full(n, -1, dtype=np.int64)
    level_of = np.full(n, -1, dtype=np.int64)
    dmax = nlevels - 1
    frontier = [(0, np.arange(n, dtype=np.int64))]
    for depth in range(dmax + 1):
        nxt = []
        for node, verts in frontier:
            if verts.size == 0:
                raise ValueError(f"empty nested-dissection subdomain at node {node}")
            if depth == dmax:
                node_of[verts] = node
                level_of[verts] = 0
                continue
            sep, lo, hi = graph_bisect(rowptr, colind, verts)
            node_of[sep] = node
            level_of[sep] = dmax - depth
            nxt.append((2 * node + 1, lo))
            nxt.append((2 * node + 2, hi))
        frontier = nxt
    reach = [()] * n
    for lvl in range(1, nlevels):
        for v in np.nonzero(level_of == lvl)[0]:
            s = set()
            for u in colind[rowptr[v]:rowptr[v + 1]]:
                if level_of[u] == 0:
                    s.add(int(node_of[u]))
                elif level_of[u] < lvl:
                    s.update(reach[u])
            reach[v] = tuple(sorted(s))
    width = max([1] + [len(r) for r in reach])
    return GraphNDTree(nlevels=nlevels, node_of=node_of, level_of=level_of, reach=reach,
                       width=width)


def ancestor(i: int, depth: int) -> int:
    """The ancestor at ``depth`` of heap-numbered node ``i`` (i itself if not deeper)."""
    while node_depth(i) > depth:
        i = (i - 1) // 2
    return i


def graph_cluster_keys(tree: GraphNDTree, k: int):
    """Cluster key of every live vertex at stage ``k`` (algebraic tree): like
    ``cluster_keys``, rows ``(node, key[0], ..., key[width-1])`` with the key's
    sorted subdomain ids padded with -1."""
    ell = tree.nlevels
    dk = ell - 1 - k
    live = np.nonzero(tree.level_of >= k)[0].astype(np.int64)
    rows = np.full((live.size, 1 + tree.width), -1, dtype=np.int64)
    rows[:, 0] = tree.node_of[live]
    for i, v in enumerate(live):
        if tree.level_of[v] > k:
            key = sorted({ancestor(leaf, dk) for leaf in tree.reach[v]})
            rows[i, 1:1 + len(key)] = key
    return live, rows


def build_tree(coords, nlevels: int, rowptr=None, colind=None):
    """The multilevel tree: geometric with coordinates, algebraic (from the
    CSR pattern) when ``coords`` is None."""
    if coords is None:
        return graph_nested_dissection(rowptr, colind, nlevels)
    return nested_dissection(coords, nlevels)


def tree_cluster_keys(tree, k: int):
    """``cluster_keys`` for either kind of tree."""
    if isinstance(tree, GraphNDTree):
        return graph_cluster_keys(tree, k)
    return cluster_keys(tree, k)
