"""Pins of the box-QP relaxation workload (the qpG-type rows of Table 1):
the SDP relaxation of min x^T L_w x over x in [-1, 1]^n1 with the box
written by slacks, X = [[X1, .], [., S]], X1_ii + S_ii = 1.

* Two vertices and one edge of weight w: <L_w, X1> = w (X1_11 + X1_22 -
  2 X1_12) over PSD X1 with diagonal at most 1.  For w < 0 the optimum is
  4w (X1 = [[1, -1], [-1, 1]]); for w > 0 it is 0 (X1 = 0, S = I), both
  forms of the iteration (reading P7).
* Structure: the slack diagonal has no off-diagonal pattern entry, so each
  slack vertex is a clique of its own (Section 2.1: the maximal cliques of
  the chordal pattern); the chordal extension of the graph part is checked
  by networkx (is_chordal, its maximal cliques).
* X = I/2 satisfies every constraint (feasibility by construction).
"""
import networkx as nx
import numpy as np
import pytest

import synth
from oracle import hsde, symbolic

FORMS = {"literal": dict(alpha=1.0, scaling=False), "relaxed_scaled": dict(alpha=1.8, scaling=True)}


def _two_vertex(w):
    """The box QP on one edge of weight w (vertices 0, 1; slacks 2, 3)."""
    C_row = np.array([0, 1, 1], np.int32)
    C_col = np.array([0, 0, 1], np.int32)
    C_val = np.array([w, -w, w])
    A_ptr = np.array([0, 2, 4], np.int64)
    A_row = np.array([0, 2, 1, 3], np.int32)
    return synth.Problem("box_qp_2", 4, 2, C_row, C_col, C_val, A_ptr, A_row, A_row.copy(), np.ones(4), np.ones(2))


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("w", [-1.0, 1.0, -0.4])
def test_two_vertex_box_qp_closed_form(w, form):
    res = hsde.HSDE(_two_vertex(w), **FORMS[form]).solve(eps=1e-8, max_iter=50000)
    assert res.status == hsde.SOLVED
    want = 4.0 * w if w < 0 else 0.0
    assert abs(res.info["pobj"] - want) <= 1e-5
    assert abs(res.info["dobj"] - want) <= 1e-5


def test_generator_matches_the_two_vertex_form():
    """synth.box_qp on two vertices and one edge builds the same data as the
    hand-written instance above (up to the weight's sign)."""
    p = synth.box_qp(2, 1, np.random.default_rng(0))
    w = float(p.C_val[(p.C_row == 0) & (p.C_col == 0)][0])
    q = _two_vertex(w)
    for k in ("C_row", "C_col", "C_val", "A_ptr", "A_row", "A_col", "A_val", "b"):
        assert np.array_equal(np.asarray(getattr(p, k)), np.asarray(getattr(q, k))), k


@pytest.mark.parametrize("n1,E,seed", [(40, 90, 1), (300, 1400, 7)])
def test_box_qp_structure(n1, E, seed):
    p = synth.box_qp(n1, E, np.random.default_rng(seed))
    st = symbolic.analyze(p)
    cliques = [list(c) for c in st.cliques]
    singles = sorted(c[0] for c in cliques if len(c) == 1 and c[0] >= n1)
    assert singles == list(range(n1, 2 * n1))            # every slack vertex alone
    assert all(max(c) < n1 for c in cliques if not (len(c) == 1 and c[0] >= n1))
    G = nx.Graph()
    G.add_nodes_from(range(n1))
    pr, pc = np.asarray(st.pat_row), np.asarray(st.pat_col)
    for r, c in zip(pr, pc):
        if r != c and r < n1:
            G.add_edge(int(r), int(c))
    assert nx.is_chordal(G)
    want = {frozenset(c) for c in nx.chordal_graph_cliques(G)}
    got = {frozenset(c) for c in cliques if max(c) < n1}
    assert got == want


def test_half_identity_is_feasible():
    p = synth.box_qp(50, 120, np.random.default_rng(3))
    X = 0.5 * np.eye(p.n)
    for i in range(p.m):
        a, b = int(p.A_ptr[i]), int(p.A_ptr[i + 1])
        val = sum(p.A_val[k] * X[p.A_row[k], p.A_col[k]] * (1 if p.A_row[k] == p.A_col[k] else 2) for k in range(a, b))
        assert val == pytest.approx(p.b[i])
