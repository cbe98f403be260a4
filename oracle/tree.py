"""Domain tree (Section 2, Definition "Domain tree"; ideal domains by
recursive 2^d partition, Section 2 after that definition).

Test infrastructure: part of the oracle package.

A node is a subdomain; its children partition it; the root is the whole
point set.  On an ideal d-dimensional domain the paper partitions each node
into 2^d children by halving every coordinate direction.  The split used
here halves the node's points axis by axis (x, then y, then z): sort by
(coordinate, original index) and give the first floor(n/2) points to the
lower half.  On an n^d grid of cell centres with n a power of two this is
exactly the paper's uniform geometric 2^d partition; on other point sets it
is the balanced (median) version of the same partition, which still
satisfies the definition (children partition the parent).

Children are numbered c = b_0 + 2 b_1 (+ 4 b_2), b_a = 1 for the upper
half along axis a, and are laid out in that order, so every node owns a
contiguous range [begin, end) of the tree order.

Box coordinates.  A node of level l is the subdomain
prod_a [q_a h, (q_a + 1) h] of the ideal domain [0, 1]^d, h = 2^-l, with
q = 2 q_parent + (b_0, b_1, b_2): the geometry the admissibility
conditions are stated on (on the grids it is the points' own cell).

Depth.  The leaves are all at depth L, the smallest L >= 0 with
ceil(N / 2^(d L)) <= leaf_size (the paper leaves the leaf size open; the
workloads use 64).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Node:
    level: int
    index: int            # position among the nodes of its level, tree order
    begin: int            # tree-order range [begin, end)
    end: int
    children: list = field(default_factory=list)
    parent: "Node | None" = None
    child_id: int = 0     # c = b_0 + 2 b_1 + 4 b_2 inside the parent
    coords: tuple = ()    # box coordinates q: the subdomain prod [q_a h, (q_a + 1) h], h = 2^-level

    @property
    def size(self) -> int:
        return self.end - self.begin

    def is_leaf(self) -> bool:
        return not self.children


@dataclass
class DomainTree:
    d: int
    N: int
    leaf_size: int
    depth: int                       # L: leaves are at level L
    perm: np.ndarray                 # perm[tree position] = original point index
    levels: list                     # levels[l] = list of Node in tree order

    @property
    def root(self) -> Node:
        return self.levels[0][0]

    def ancestor(self, pos: int, level: int) -> Node:
        """The node at `level` whose range contains tree position `pos`."""
        nodes = self.levels[level]
        begins = np.fromiter((n.begin for n in nodes), dtype=np.int64, count=len(nodes))
        j = int(np.searchsorted(begins, pos, side="right")) - 1
        while nodes[j].size == 0 or not (nodes[j].begin <= pos < nodes[j].end):
            j -= 1
        return nodes[j]


def tree_depth(N: int, d: int, leaf_size: int) -> int:
    """Smallest L >= 0 with ceil(N / 2^(dL)) <= leaf_size."""
    if leaf_size <= 0:
        raise ValueError("leaf_size must be positive")
    L = 0
    while -(-N // (1 << (d * L))) > leaf_size:
        L += 1
    return L


def _split_half(points: np.ndarray, idx: np.ndarray, axis: int):
    """Lower / upper halves of `idx` along `axis`, ties broken by index."""
    order = np.lexsort((idx, points[idx, axis]))   # primary key: coordinate
    srt = idx[order]
    h = len(srt) // 2
    return srt[:h], srt[h:]


def build_tree(points: np.ndarray, leaf_size: int) -> DomainTree:
    """Domain tree of `points` (N x d float64), children by 2^d partition."""
    points = np.asarray(points, dtype=np.float64)
    N, d = points.shape
    L = tree_depth(N, d, leaf_size)
    perm_parts: list[np.ndarray] = []
    levels: list[list[Node]] = [[] for _ in range(L + 1)]

    def recurse(idx: np.ndarray, level: int, begin: int, parent, child_id):
        if parent is None:
            coords = (0,) * d
        else:
            coords = tuple(2 * parent.coords[a] + ((child_id >> a) & 1) for a in range(d))
        node = Node(level, len(levels[level]), begin, begin + len(idx),
                    parent=parent, child_id=child_id, coords=coords)
        levels[level].append(node)
        if level == L:
            perm_parts.append(idx)
            return node
        parts = [idx]
        for axis in range(d):                       # halve along x, then y, then z
            nxt = []
            for p in parts:
                lo, hi = _split_half(points, p, axis)
                nxt.extend([lo, hi])
            parts = nxt
        # Halving appends (lo, hi) for every part, so the list position, read
        # in binary, is b_0 b_1 ... b_{d-1} with b_0 most significant.
        # Reorder to the child id c = b_0 + 2 b_1 + 4 b_2.
        children_idx = [None] * (1 << d)
        for pos, p in enumerate(parts):
            bits = [(pos >> (d - 1 - a)) & 1 for a in range(d)]   # b_a
            c = sum(b << a for a, b in enumerate(bits))
            children_idx[c] = p
        off = begin
        for c in range(1 << d):
            ch = recurse(children_idx[c], level + 1, off, node, c)
            node.children.append(ch)
            off += len(children_idx[c])
        return node

    recurse(np.arange(N, dtype=np.int64), 0, 0, None, 0)
    perm = np.concatenate(perm_parts) if perm_parts else np.zeros(0, dtype=np.int64)
    return DomainTree(d, N, leaf_size, L, perm, levels)
