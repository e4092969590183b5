"""Pins of the oracle's cone projection (Eq. Step2) and affine step (Eq. Step1).

* PSD projection: closed forms (diagonal input, 2x2 eigenvalues written out),
  the variational inequality that characterises a Euclidean projection onto a
  closed convex cone, Moreau's decomposition, a brute-force minimisation on
  2x2 blocks, and non-symmetric input (reading P8).
* Affine step: skew-symmetry of Q (Section 3.2), the block-eliminated path of
  Sections 4.2-4.3 against a dense LU solve of the literal (I + Q), the block
  form of Eq. ThirdBlkElm against I + Ahat^T Ahat (reading P2), and the
  restriction of x to the chordal pattern against the full n^2 space (P1).
"""
import numpy as np
import pytest
import scipy.optimize as so

import synth
from oracle import dense, hsde, symbolic


def _rand_sym(rng, c):
    G = rng.standard_normal((c, c))
    return 0.5 * (G + G.T)


def test_psd_diagonal_closed_form():
    d = np.array([3.0, -1.0, 0.0, 2.5, -7.0])
    assert np.allclose(hsde.project_psd(np.diag(d)), np.diag(np.maximum(d, 0)), atol=1e-15)


def test_psd_2x2_closed_form():
    rng = np.random.default_rng(0)
    for _ in range(50):
        a, b, c = rng.standard_normal(3)
        # eigenvalues of [[a,b],[b,c]] written out
        tr, det = a + c, a * c - b * b
        disc = np.sqrt(tr * tr / 4 - det)
        l1, l2 = tr / 2 + disc, tr / 2 - disc
        X = np.array([[a, b], [b, c]])
        P = hsde.project_psd(X)
        if l2 >= 0:
            want = X
        elif l1 <= 0:
            want = np.zeros((2, 2))
        else:
            # rank one: l1 * v v^T, v the eigenvector of l1
            v = np.array([b, l1 - a]) if abs(b) > 1e-12 else (np.array([1.0, 0]) if a > c else np.array([0, 1.0]))
            v /= np.linalg.norm(v)
            want = l1 * np.outer(v, v)
        assert np.allclose(P, want, atol=1e-12)


@pytest.mark.parametrize("c", [2, 3, 5, 8])
def test_psd_variational_inequality_and_moreau(c):
    rng = np.random.default_rng(c)
    for _ in range(20):
        X = _rand_sym(rng, c)
        P = hsde.project_psd(X)
        N = hsde.project_psd(-X)
        assert np.linalg.eigvalsh(P).min() >= -1e-12
        assert np.allclose(X, P - N, atol=1e-12)                 # Moreau
        assert abs(np.sum(P * N)) <= 1e-12                        # orthogonality
        for _ in range(10):
            G = rng.standard_normal((c, c))
            Y = G @ G.T
            assert np.sum((X - P) * (Y - P)) <= 1e-10             # projection characterisation


def test_psd_brute_force_2x2():
    rng = np.random.default_rng(5)
    for _ in range(10):
        X = _rand_sym(rng, 2)
        f = lambda L: np.sum((np.array([[L[0], 0], [L[1], L[2]]]) @ np.array([[L[0], L[1]], [0, L[2]]]) - X) ** 2)
        best = min((so.minimize(f, x0, method="BFGS", options=dict(gtol=1e-12)) for x0 in rng.standard_normal((6, 3))),
                   key=lambda r: r.fun)
        L = np.array([[best.x[0], 0], [best.x[1], best.x[2]]])
        assert np.allclose(L @ L.T, hsde.project_psd(X), atol=1e-5)


def test_psd_nonsymmetric_input_is_projection_in_Rc2():
    rng = np.random.default_rng(9)
    for _ in range(20):
        X = rng.standard_normal((4, 4))          # not symmetric
        P = hsde.project_psd(X)
        for _ in range(10):
            G = rng.standard_normal((4, 4))
            Y = G @ G.T
            assert np.sum((X - P) * (Y - P)) <= 1e-10


def _tiny(l=3, d=3, h=2, m=4, seed=0, dense_constraints=False):
    return synth.block_arrow(l, d, h, m, np.random.default_rng(seed), dense_constraints=dense_constraints,
                             kappa=50.0)


def test_Q_is_skew():
    hs = hsde.HSDE(_tiny())
    Q = dense.build_Q(hs)
    assert np.array_equal(Q, -Q.T)
    u = np.random.default_rng(1).standard_normal(hs.dim)
    assert abs(u @ Q @ u) < 1e-10


@pytest.mark.parametrize("prob", ["tiny", "tiny_dense", "arrow_n50", "arrow_n50_inf", "grid"])
def test_affine_matches_dense_solve(prob):
    p = {"tiny": lambda: _tiny(), "tiny_dense": lambda: _tiny(dense_constraints=True, seed=3),
         "arrow_n50": synth.block_arrow_n50, "arrow_n50_inf": lambda: synth.block_arrow_n50(True),
         "grid": lambda: synth.maxcut_grid(3, 4, np.random.default_rng(2))}[prob]()
    for scaling in (False, True):
        _affine_vs_dense(hsde.HSDE(p, scaling=scaling))


def _affine_vs_dense(hs):
    Q = dense.build_Q(hs)
    rng = np.random.default_rng(11)
    for _ in range(3):
        om = rng.standard_normal(hs.dim)
        a = hs.affine(om)
        b = dense.affine_dense(hs, om, Q)
        assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)


def test_third_block_elimination_matrix():
    """Eq. ThirdBlkElm is I + Ahat^T Ahat (not I + Ahat Ahat^T): reading P2."""
    hs = hsde.HSDE(_tiny(m=3))
    Ah = hs.Ahat.toarray()
    A = hs.A.toarray(); H = hs.V.H.toarray()      # the (scaled) data the iteration uses
    D = np.diag(hs.D)
    nd = hs.nd
    blk = np.block([[np.eye(hs.nF) + D + A.T @ A, -H.T], [-H, 2 * np.eye(nd)]])
    assert np.allclose(np.eye(Ah.shape[1]) + Ah.T @ Ah, blk)
    assert (Ah @ Ah.T).shape != blk.shape
    # and the factored matrix of Eq. FactorizationMatrix
    g = np.random.default_rng(0).standard_normal(hs.nF)
    M = np.eye(hs.nF) + 0.5 * D + A.T @ A
    assert np.allclose(hs.solve_factor(g), np.linalg.solve(M, g), atol=1e-12)


@pytest.mark.parametrize("alpha,scaling", [(1.0, False), (1.8, True)])
def test_dense_iterates_match_eliminated_iterates(alpha, scaling):
    p = synth.block_arrow_n50()
    hs = hsde.HSDE(p, alpha=alpha, scaling=scaling)
    Q = dense.build_Q(hs)
    u, nu = hs.initial()
    u2, nu2 = u.copy(), nu.copy()
    for _ in range(25):
        u, nu, _ = hs.step(u, nu)
        u2, nu2, _ = dense.step_dense(hs, u2, nu2, Q)
    # rounding of two different FP64 solves accumulates over the iterations
    assert np.linalg.norm(u - u2) <= 1e-7 * np.linalg.norm(u2)
    assert np.linalg.norm(nu - nu2) <= 1e-7 * max(1.0, np.linalg.norm(nu2))


def test_pattern_restriction_equals_full_space():
    """Reading P1: entries of vec(X) outside E' stay exactly 0 and the
    E'-restricted iteration equals the one on all of R^{n^2}."""
    p = synth.block_arrow(2, 2, 1, 3, np.random.default_rng(4), kappa=20.0)
    st = symbolic.analyze(p)
    full = hsde.HSDE(p, st, full_space=True)
    rest = hsde.HSDE(p, st)
    uf, nf = full.initial()
    ur, nr = rest.initial()
    for _ in range(30):
        uf, nf, _ = full.step(uf, nf)
        ur, nr, _ = rest.step(ur, nr)
    xf = uf[:full.nF]
    on = np.zeros(full.nF, bool)
    for rc in rest.V.ent:
        on[full.V.fpos[rc]] = True
    assert np.all(xf[~on] == 0.0)
    xr = ur[:rest.nF]
    assert np.allclose(np.array([xf[full.V.fpos[rc]] for rc in rest.V.ent]), xr, atol=1e-12)
    assert np.allclose(uf[full.nF:], ur[rest.nF:], atol=1e-12)


def test_packed_layout_roundtrip():
    hs = hsde.HSDE(synth.block_arrow_n50())
    rng = np.random.default_rng(0)
    xl = rng.standard_normal(hs.V.st.N)
    assert np.array_equal(hs.V.x_to_lower(hs.V.x_from_lower(xl)), xl)
    sp_ = rng.standard_normal(hs.V.st.P)
    assert np.array_equal(hs.V.s_to_packed(hs.V.s_from_packed(sp_)), sp_)
