"""Reverse Cuthill-McKee ordering and the symmetric permutation P A P^T.
Test infrastructure only (see ``oracle/__init__.py``).

The paper reduces the bandwidth of matrices that are not already
bandwidth-reduced with an RCM reordering [Cuthill 1969] before translating
them to DA-CSR (Section 2, Example 2; Section 3).  It names no start vertex,
no tie-break rule and no treatment of disconnected graphs, and notes that its
own RCM yields a different bandwidth from SuiteSparse's on the same matrix.
RCM is therefore not unique; this oracle fixes one reading, and the CUDA
library's ordering must reproduce it bit for bit:

1. G is the pattern of A + A^T without self loops; deg(v) is the number of
   distinct neighbours of v.
2. Connected components are processed in the order of their smallest vertex.
3. Inside a component the start vertex is a pseudo-peripheral vertex found by
   the George-Liu iteration: begin at the component's vertex of minimum
   degree (ties: smaller index); build the BFS level structure; take the
   vertex of minimum degree in the last level (ties: smaller index); move to
   it while its eccentricity is strictly larger, else stop.
4. Cuthill-McKee: breadth-first from the start vertex; when a vertex is
   dequeued, its unvisited neighbours are appended in order of increasing
   degree, ties by increasing index.
5. The component orders are concatenated and the whole sequence is reversed.
   The result ``perm`` maps new index -> old index.
6. P A P^T: new row i is old row perm[i]; each column c becomes iperm[c]; each
   row is then sorted by new column (entries with equal columns keep their
   stored order).
"""
from __future__ import annotations

from collections import deque

import numpy as np

from .dacsr import entry_rows


def symmetric_graph(n: int, rowptr, col):
    """Adjacency (CSR, neighbours ascending) of pattern(A) + pattern(A^T)
    without self loops, and the degree of every vertex."""
    r = entry_rows(n, rowptr)
    c = np.asarray(col, dtype=np.int64)
    a = np.concatenate([r, c])
    b = np.concatenate([c, r])
    keep = a != b
    key = np.unique(a[keep] * n + b[keep])
    src = key // n
    dst = key - src * n
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=ptr[1:])
    deg = np.diff(ptr)
    return ptr, dst, deg


def level_structure(start: int, ptr, adj):
    """Rooted level structure: list of BFS levels (each a list of vertices)."""
    seen = {start}
    levels = [[start]]
    while True:
        nxt = []
        for v in levels[-1]:
            for u in adj[ptr[v]:ptr[v + 1]].tolist():
                if u not in seen:
                    seen.add(u)
                    nxt.append(u)
        if not nxt:
            return levels
        levels.append(nxt)


def pseudo_peripheral(start: int, ptr, adj, deg) -> int:
    """George-Liu: walk to a min-degree vertex of the last BFS level while the
    eccentricity grows."""
    v = start
    levels = level_structure(v, ptr, adj)
    while True:
        last = levels[-1]
        u = min(last, key=lambda t: (int(deg[t]), t))
        lu = level_structure(u, ptr, adj)
        if len(lu) > len(levels):
            v, levels = u, lu
        else:
            return v


def cuthill_mckee_from(start: int, ptr, adj, deg, visited) -> list:
    order = [start]
    visited[start] = True
    queue = deque([start])
    while queue:
        v = queue.popleft()
        nbrs = [u for u in adj[ptr[v]:ptr[v + 1]].tolist() if not visited[u]]
        nbrs.sort(key=lambda t: (int(deg[t]), t))
        for u in nbrs:
            visited[u] = True
            order.append(u)
            queue.append(u)
    return order


def rcm_order(n: int, rowptr, col) -> np.ndarray:
    """RCM permutation perm (new index -> old index), int32[n]."""
    ptr, adj, deg = symmetric_graph(n, rowptr, col)
    visited = np.zeros(n, dtype=bool)
    comp_seen = np.zeros(n, dtype=bool)
    order = []
    for v0 in range(n):
        if visited[v0]:
            continue
        # the component of v0, to pick its minimum-degree vertex
        comp = [v0]
        comp_seen[v0] = True
        q = deque([v0])
        while q:
            v = q.popleft()
            for u in adj[ptr[v]:ptr[v + 1]].tolist():
                if not comp_seen[u]:
                    comp_seen[u] = True
                    comp.append(u)
                    q.append(u)
        s = min(comp, key=lambda t: (int(deg[t]), t))
        p = pseudo_peripheral(s, ptr, adj, deg)
        order.extend(cuthill_mckee_from(p, ptr, adj, deg, visited))
    return np.asarray(order[::-1], dtype=np.int32)


def inverse_permutation(perm) -> np.ndarray:
    perm = np.asarray(perm, dtype=np.int64)
    iperm = np.empty_like(perm)
    iperm[perm] = np.arange(len(perm), dtype=np.int64)
    return iperm


def permute_symmetric(n: int, rowptr, col, val, perm):
    """B = P A P^T with B[i, j] = A[perm[i], perm[j]]: every entry (r, c, v)
    of A becomes (iperm[r], iperm[c], v); rows sorted by column, equal
    columns in stored order."""
    iperm = inverse_permutation(perm)
    r = iperm[entry_rows(n, rowptr)]
    c = iperm[np.asarray(col, dtype=np.int64)]
    pos = np.arange(len(c), dtype=np.int64)
    order = np.lexsort((pos, c, r))
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=rp[1:])
    return rp.astype(np.int32), c[order].astype(np.int32), np.asarray(val)[order]
