"""Pins of the oracle's symbolic analysis (Section 2.1-2.2, Section 3.1, Section 4.3).

Each pin comes from outside the oracle: closed-form clique structure of
block-arrow patterns (golden file), minimum-degree eliminations written here
from the definition (a brute-force one for small graphs, a heap-based one
for the 2000-vertex grids), networkx's chordality test and maximal-clique
enumeration.
"""
import json
import os
import random

import numpy as np
import pytest

nx = pytest.importorskip("networkx")

import synth
from oracle import symbolic

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "structure_pins.json")))


def _brute_md(n, pairs):
    """Minimum degree straight from the definition: at every step recount the
    degree of every alive vertex in the current elimination graph."""
    E = set()
    for i, j in pairs:
        if i != j:
            E.add((min(i, j), max(i, j)))
    alive = set(range(n))
    order, cand = [], []
    while alive:
        def deg(v):
            return sum(1 for u in alive if u != v and (min(u, v), max(u, v)) in E)
        v = min(alive, key=lambda v: (deg(v), v))
        nb = {u for u in alive if u != v and (min(u, v), max(u, v)) in E}
        for a in nb:
            for b in nb:
                if a < b:
                    E.add((a, b))
        order.append(v)
        cand.append(frozenset(nb | {v}))
        alive.remove(v)
    return order, cand


def _random_problem(n, n_edges, seed):
    rng = np.random.default_rng(seed)
    r, c = [], []
    for _ in range(n_edges):
        i, j = rng.integers(0, n, 2)
        if i != j:
            r.append(max(i, j)); c.append(min(i, j))
    key = sorted(set(zip(r, c)))
    rr = np.array([k[0] for k in key] + list(range(n)), np.int32)
    cc = np.array([k[1] for k in key] + list(range(n)), np.int32)
    return synth.Problem("rand", n, 0, rr, cc, np.ones(len(rr)), np.zeros(1, np.int64),
                         np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0), np.zeros(0))


@pytest.mark.parametrize("seed", range(8))
def test_minimum_degree_matches_brute_force(seed):
    n = 9 + seed
    p = _random_problem(n, 2 * n, seed)
    pat = symbolic.aggregate_pattern(p)
    order, cand = symbolic.minimum_degree(n, pat)
    o2, c2 = _brute_md(n, pat)
    assert order == o2
    assert cand == c2


def _filled_graph(st):
    G = nx.Graph()
    G.add_nodes_from(range(st.n))
    for r, c in zip(st.pat_row.tolist(), st.pat_col.tolist()):
        if r != c:
            G.add_edge(r, c)
    return G


@pytest.mark.parametrize("seed", range(6))
def test_cliques_against_networkx(seed):
    n = 40 + 10 * seed
    p = _random_problem(n, 3 * n, 100 + seed)
    st = symbolic.analyze(p)
    G = _filled_graph(st)
    assert nx.is_chordal(G)
    # the extension contains the original pattern
    for r, c in symbolic.aggregate_pattern(p):
        assert r == c or G.has_edge(r, c)
    ours = {frozenset(c.tolist()) for c in st.cliques}
    theirs = {frozenset(c) for c in nx.find_cliques(G)}
    assert ours == theirs
    assert ours == {frozenset(c) for c in nx.chordal_graph_cliques(G)}
    # members in natural (ascending) order
    for c in st.cliques:
        assert np.all(np.diff(c) > 0)


def test_block_arrow_closed_form():
    g = GOLD["block_arrow_l8_d6_h2"]
    p = synth.block_arrow_n50()
    st = symbolic.analyze(p)
    assert st.p == g["p"] and all(len(c) == g["c"] for c in st.cliques)
    assert st.N == g["N"] and st.n_d == g["n_d"] and st.P == g["P"]
    # zero fill: cliques are block_j U arrow
    want = {frozenset(c) for c in synth.block_arrow_cliques(8, 6, 2)}
    assert {frozenset(c.tolist()) for c in st.cliques} == want
    # E' equals the aggregate pattern (no fill)
    assert set(zip(st.pat_row.tolist(), st.pat_col.tolist())) == symbolic.aggregate_pattern(p)


@pytest.mark.parametrize("l,d,h", [(3, 4, 2), (10, 5, 3), (7, 2, 1)])
def test_block_arrow_shapes(l, d, h):
    p = synth.block_arrow(l, d, h, 2 * l, np.random.default_rng(1))
    st = symbolic.analyze(p)
    assert {frozenset(c.tolist()) for c in st.cliques} == {frozenset(c) for c in synth.block_arrow_cliques(l, d, h)}


def _heap_md_cliques(n, pairs):
    """Minimum degree (ties: smallest vertex) on the elimination graph, from
    the definition, with adjacency sets and a lazily invalidated heap of
    (degree, vertex); returns the maximal cliques among the candidates
    {v} U (alive neighbours of v) as sorted tuples."""
    import heapq
    adj = [set() for _ in range(n)]
    for i, j in pairs:
        if i != j:
            adj[i].add(j)
            adj[j].add(i)
    heap = [(len(adj[v]), v) for v in range(n)]
    heapq.heapify(heap)
    done = [False] * n
    cands = []
    while heap:
        d, v = heapq.heappop(heap)
        if done[v] or d != len(adj[v]):
            continue
        nb = sorted(adj[v])
        done[v] = True
        cands.append(tuple(sorted(nb + [v])))
        for u in nb:
            adj[u].discard(v)
        for a in range(len(nb)):
            for b in range(a + 1, len(nb)):
                x, y = nb[a], nb[b]
                if y not in adj[x]:
                    adj[x].add(y)
                    adj[y].add(x)
        for u in nb:
            heapq.heappush(heap, (len(adj[u]), u))
    # maximal: not a subset of another candidate (a candidate can only lie
    # inside the candidate of one of its own members)
    sets = [frozenset(c) for c in cands]
    by_member = {}
    for k, c in enumerate(sets):
        for u in c:
            by_member.setdefault(u, []).append(k)
    out = []
    for k, c in enumerate(sets):
        if not any(j != k and len(sets[j]) > len(c) and c <= sets[j] for u in c for j in by_member[u]):
            out.append(cands[k])
    return out


def test_heap_md_matches_brute_force_on_small_graphs():
    for seed in range(4):
        n = 12 + seed
        p = _random_problem(n, 2 * n, 100 + seed)
        pat = symbolic.aggregate_pattern(p)
        _, cand = _brute_md(n, pat)
        brute = {frozenset(c) for c in cand if not any(c < d for d in cand)}
        assert {frozenset(c) for c in _heap_md_cliques(n, pat)} == brute


@pytest.mark.parametrize("R,K", [(20, 100), (10, 100)])
def test_grid_structure_matches_independent_elimination(R, K):
    # the max-cut grids of the benchmark workloads: p, clique sizes,
    # n_d = sum c^2 (Section 3.2) and P = sum c (c + 1) / 2
    p = synth.maxcut_grid(R, K, synth.rng_for(1))
    st = symbolic.analyze(p)
    want = _heap_md_cliques(p.n, symbolic.aggregate_pattern(p))
    sz = sorted(len(c) for c in want)
    got = sorted(len(c) for c in st.cliques)
    assert st.p == len(want) and got == sz
    assert {tuple(sorted(c.tolist())) for c in st.cliques} == set(want)
    assert st.n_d == sum(c * c for c in sz)
    assert st.P == sum(c * (c + 1) // 2 for c in sz)


def test_index_maps_and_D():
    p = _random_problem(60, 150, 7)
    st = symbolic.analyze(p)
    pos = {(r, c): e for e, (r, c) in enumerate(zip(st.pat_row.tolist(), st.pat_col.tolist()))}
    # CSC-lower order
    keys = list(zip(st.pat_col.tolist(), st.pat_row.tolist()))
    assert keys == sorted(keys) and all(r >= c for r, c in pos)
    assert np.array_equal(np.diff(st.pat_colptr), np.bincount(st.pat_col, minlength=st.n))
    D = np.zeros(st.N, np.int64)
    t = 0
    for k, mem in enumerate(st.cliques):
        ml = mem.tolist()
        assert st.packed_ptr[k] == t
        for b in range(len(ml)):
            for a in range(b, len(ml)):
                assert st.gather[t] == pos[(ml[a], ml[b])]
                D[pos[(ml[a], ml[b])]] += 1
                t += 1
    assert np.array_equal(D, st.D)
    # D counts cliques containing both endpoints, counted directly
    for e, (r, c) in enumerate(zip(st.pat_row.tolist(), st.pat_col.tolist())):
        assert st.D[e] == sum(1 for mem in st.cliques if r in mem and c in mem)


def test_perfect_elimination_order():
    p = _random_problem(50, 120, 3)
    st = symbolic.analyze(p)
    G = _filled_graph(st)
    step = {v: t for t, v in enumerate(st.order.tolist())}
    for v in G.nodes:
        later = [u for u in G.neighbors(v) if step[u] > step[v]]
        for a in later:
            for b in later:
                if a < b:
                    assert G.has_edge(a, b)
