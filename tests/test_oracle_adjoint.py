"""Pins of the oracle's reverse-mode gradient of f(C, b) = c^T x_K / tau_K
after K unrolled ADMM iterations: central finite differences of the oracle's
own forward (step 1e-6, FP64) on random directions, a finite-difference check
of the Daleckii-Krein product alone, and the literal sparse Q against the
dense one."""
import numpy as np
import pytest

import synth
from oracle import adjoint, dense, hsde


def _perturbed(p, dC_lower_vals, db, t):
    q = synth.Problem(**{**p.__dict__})
    q.C_val = p.C_val + t * dC_lower_vals
    q.b = p.b + t * db
    return q


def _C_on_pattern(p, st):
    """Give C an explicit entry on every pattern position (zeros allowed) so
    that perturbations can touch all of them."""
    pos = {(r, c): e for e, (r, c) in enumerate(zip(p.C_row.tolist(), p.C_col.tolist()))}
    vals = np.zeros(st.N)
    for e, (r, c) in enumerate(zip(st.pat_row.tolist(), st.pat_col.tolist())):
        if (r, c) in pos:
            vals[e] = p.C_val[pos[(r, c)]]
    q = synth.Problem(**{**p.__dict__})
    q.C_row, q.C_col, q.C_val = st.pat_row.copy(), st.pat_col.copy(), vals
    return q


def test_dk_vjp_matches_finite_differences():
    rng = np.random.default_rng(0)
    for c in (2, 4, 7):
        A = rng.standard_normal((c, c)); A = A + A.T
        G = rng.standard_normal((c, c)); G = G + G.T
        D = rng.standard_normal((c, c)); D = D + D.T
        h = 1e-6
        fd = (np.sum(G * hsde.project_psd(A + h * D)) - np.sum(G * hsde.project_psd(A - h * D))) / (2 * h)
        assert abs(fd - np.sum(adjoint.dk_vjp(A, G) * D)) <= 1e-6 * (1 + abs(fd))


def test_sparse_Q_equals_dense_Q():
    hs = hsde.HSDE(synth.block_arrow_n50(), alpha=1.0, scaling=False)
    assert np.array_equal(adjoint.sparse_Q(hs).toarray(), dense.build_Q(hs))


@pytest.mark.parametrize("case", ["grid", "arrow"])
def test_unrolled_gradient_matches_central_differences(case):
    rng = np.random.default_rng(3)
    if case == "grid":
        p0 = synth.maxcut_grid(3, 5, np.random.default_rng(1))
        K = 40
    else:
        p0 = synth.block_arrow(3, 3, 2, 5, np.random.default_rng(2), kappa=30.0, assign="roundrobin")
        K = 30
    st = hsde.HSDE(p0, alpha=1.0, scaling=False).V.st
    p = _C_on_pattern(p0, st)
    hs = hsde.HSDE(p, alpha=1.0, scaling=False)
    f, cbar, bbar = adjoint.gradient(hs, K)
    assert f == pytest.approx(adjoint.objective(hs, K), rel=1e-12)
    G = adjoint.grad_C_lower(hs, cbar)
    w = np.where(st.pat_row == st.pat_col, 1.0, 2.0)
    for _ in range(4):
        dC = rng.standard_normal(st.N)
        db = rng.standard_normal(p.m)
        h = 1e-6
        fp = adjoint.objective(hsde.HSDE(_perturbed(p, dC, db, h), alpha=1.0, scaling=False), K)
        fm = adjoint.objective(hsde.HSDE(_perturbed(p, dC, db, -h), alpha=1.0, scaling=False), K)
        fd = (fp - fm) / (2 * h)
        an = float(np.sum(w * G * dC) + bbar @ db)
        assert abs(fd - an) <= 1e-5 * (1 + abs(fd)), (fd, an)


@pytest.mark.parametrize("rel,h,expect_half", [
    (0.0, 1e-6, True),        # exactly zero: a central difference sees 1/2 (Moreau)
    (1e-12, 1e-6, True),      # below ZERO_REL: the step crosses it, so 1/2 again
    (1e-8, 1e-11, False),     # above ZERO_REL, with a step that does not cross it: 1
])
def test_dk_zero_eigenvalue_threshold_against_differences(rel, h, expect_half):
    """The derivative of Pi_psd at an eigenvalue near zero (reading P13),
    checked against central differences of the projection itself: the
    Daleckii-Krein product with the 1e-10 threshold agrees with what a
    difference of the given step sees, and the diagonal factor of the
    near-zero direction is 1/2 or 1 accordingly."""
    rng = np.random.default_rng(7)
    c = 5
    Q, _ = np.linalg.qr(rng.standard_normal((c, c)))
    lam = np.array([2.0, 1.0, rel * 2.0, -1.0, -0.5])
    A = (Q * lam) @ Q.T
    G = rng.standard_normal((c, c)); G = 0.5 * (G + G.T)
    fd = (hsde.project_psd(A + h * G) - hsde.project_psd(A - h * G)) / (2 * h)
    dk = adjoint.dk_vjp(A, G)
    assert np.linalg.norm(dk - fd) <= 1e-4 * np.linalg.norm(fd)
    # the near-zero direction q: <q q^T, dPi[q q^T]> is its diagonal factor
    q = Q[:, 2]
    P = np.outer(q, q)
    g = float(np.sum(P * adjoint.dk_vjp(A, P)))
    assert g == pytest.approx(0.5 if expect_half else 1.0, abs=1e-6)


def test_dk_threshold_is_needed_at_that_step():
    """Without the threshold, an eigenvalue at 1e-12 of the largest would get
    the factor 1, which a central difference of step 1e-6 does not see."""
    rng = np.random.default_rng(8)
    Q, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    A = (Q * np.array([1.0, 2e-12, -0.3, 0.4])) @ Q.T
    P = np.outer(Q[:, 1], Q[:, 1])
    h = 1e-6
    fd = float(np.sum(P * (hsde.project_psd(A + h * P) - hsde.project_psd(A - h * P)))) / (2 * h)
    assert fd == pytest.approx(0.5, abs=1e-4)
    assert float(np.sum(P * adjoint.dk_vjp(A, P))) == pytest.approx(fd, abs=1e-4)
