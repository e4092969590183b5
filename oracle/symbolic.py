"""Symbolic part of the oracle (test infrastructure): Section 2 of the paper.

* aggregate sparsity pattern E of (C, A_1..A_m)             -- Section 3 (Eq. PrimalSDP)
* chordal extension E' by exact minimum-degree elimination  -- Section 2.1
* maximal cliques C_1..C_p, members in natural order        -- Section 2.1
* entry selectors H_k = E_Ck (x) E_Ck as index maps          -- Section 3.1
* D = H^T H (clique overlap count per entry)                -- Section 4.3

Readings (the paper names no extension method and no tie-break):
  * exact minimum degree on the elimination graph, ties to the smallest
    original vertex index; no clique merging;
  * the candidate clique of v is {v} U (alive neighbours of v when v is
    eliminated); the maximal cliques are the candidates contained in no other
    candidate, ordered by the elimination step of their defining vertex, and
    each clique lists its members ascending ("natural ordering");
  * E' is the union of the clique lower triangles, stored column-major lower
    (CSC lower: by column, then row);
  * the clique-local packed order is column-major lower: (a,b) for
    b = 0..c-1, a = b..c-1.

Everything here is integer work and is compared bit-exactly with the C++
host analysis of the library.
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass

import numpy as np


@dataclass
class Structure:
    n: int
    order: np.ndarray          # int32 [n]   elimination order (vertex eliminated at step t)
    cliques: list              # list of int32 arrays, members ascending
    pat_row: np.ndarray        # int32 [N]   CSC-lower pattern E' (row >= col)
    pat_col: np.ndarray        # int32 [N]
    pat_colptr: np.ndarray     # int32 [n+1]
    gather: np.ndarray         # int32 [P]   clique packed entry -> pattern position
    clique_ptr: np.ndarray     # int32 [p+1] offsets of clique members
    clique_idx: np.ndarray     # int32 [sum c_k]
    packed_ptr: np.ndarray     # int64 [p+1] offsets of packed clique storage
    D: np.ndarray              # int32 [N]   number of cliques containing each entry

    @property
    def N(self):
        return int(self.pat_row.shape[0])

    @property
    def p(self):
        return len(self.cliques)

    @property
    def P(self):
        return int(self.packed_ptr[-1])

    @property
    def n_d(self):
        return int(sum(len(c) ** 2 for c in self.cliques))


def aggregate_pattern(prob) -> set:
    """Lower pairs (i, j), i >= j, of supp(C) U supp(A_i) U diag (Section 2.2
    assumes (i,i) in E for every node)."""
    pat = set()
    for r, c in zip(prob.C_row.tolist(), prob.C_col.tolist()):
        pat.add((r, c))
    for r, c in zip(prob.A_row.tolist(), prob.A_col.tolist()):
        pat.add((r, c))
    for i in range(prob.n):
        pat.add((i, i))
    return pat


def minimum_degree(n: int, lower_pairs) -> tuple[list, list]:
    """Exact minimum-degree elimination (Section 2.1 chordal extension).

    Returns (order, candidates): order[t] is the vertex eliminated at step t and
    candidates[t] the set {v} U N(v) of its alive neighbours at that moment.
    Eliminating v turns its alive neighbourhood into a clique (the fill)."""
    adj = [set() for _ in range(n)]
    for (i, j) in lower_pairs:
        if i != j:
            adj[i].add(j)
            adj[j].add(i)
    alive = [True] * n
    heap = [(len(adj[v]), v) for v in range(n)]
    heapq.heapify(heap)
    order, cand = [], []
    while heap:
        d, v = heapq.heappop(heap)
        if not alive[v] or d != len(adj[v]):
            continue
        nb = adj[v]
        order.append(v)
        cand.append(frozenset(nb | {v}))
        alive[v] = False
        for u in nb:
            adj[u].discard(v)
            adj[u] |= nb
            adj[u].discard(u)
        for u in nb:
            heapq.heappush(heap, (len(adj[u]), u))
        adj[v] = set()
    return order, cand


def maximal_cliques(order, cand) -> list:
    """Candidates contained in no other candidate, in elimination order.

    A candidate K_v can only sit inside K_w for a w eliminated before v that
    had v as an alive neighbour, so only those are tested."""
    step = {v: t for t, v in enumerate(order)}
    earlier = [[] for _ in range(len(order))]
    for t, K in enumerate(cand):
        v = order[t]
        for u in K:
            if u != v:
                earlier[step[u]].append(t)
    out = []
    for t, K in enumerate(cand):
        if any(K <= cand[s] for s in earlier[t]):
            continue
        out.append(np.array(sorted(K), dtype=np.int32))
    return out


def analyze(prob) -> Structure:
    n = prob.n
    pat = aggregate_pattern(prob)
    order, cand = minimum_degree(n, pat)
    cliques = maximal_cliques(order, cand)
    lower = set()
    for mem in cliques:
        ml = mem.tolist()
        for b in range(len(ml)):
            for a in range(b, len(ml)):
                lower.add((ml[a], ml[b]))
    ent = sorted(lower, key=lambda rc: (rc[1], rc[0]))
    pat_row = np.array([r for r, _ in ent], dtype=np.int32)
    pat_col = np.array([c for _, c in ent], dtype=np.int32)
    colptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(colptr, pat_col + 1, 1)
    colptr = np.cumsum(colptr).astype(np.int32)
    pos = {rc: e for e, rc in enumerate(ent)}
    gather, packed_ptr = [], [0]
    for mem in cliques:
        ml = mem.tolist()
        for b in range(len(ml)):
            for a in range(b, len(ml)):
                gather.append(pos[(ml[a], ml[b])])
        packed_ptr.append(len(gather))
    gather = np.array(gather, dtype=np.int32)
    D = np.bincount(gather, minlength=len(ent)).astype(np.int32)
    clique_ptr = np.zeros(len(cliques) + 1, dtype=np.int32)
    clique_ptr[1:] = np.cumsum([len(c) for c in cliques])
    clique_idx = (np.concatenate(cliques) if cliques else np.zeros(0)).astype(np.int32)
    return Structure(n, np.array(order, dtype=np.int32), cliques, pat_row, pat_col, colptr,
                     gather, clique_ptr, clique_idx, np.array(packed_ptr, dtype=np.int64), D)
