"""Planted mistakes in the oracle must be caught by its pins.

Each case monkeypatches one plausible slip into the oracle (on the CPU) and
checks that the dense cross-check, a closed form or a verdict pin fails."""
import numpy as np
import pytest

import synth
from oracle import dense, hsde


def _affine_err(hs):
    Q = dense.build_Q(hs)
    om = np.random.default_rng(0).standard_normal(hs.dim)
    b = dense.affine_dense(hs, om, Q)
    return np.linalg.norm(hs.affine(om) - b) / np.linalg.norm(b)


def _tiny():
    return synth.block_arrow(3, 3, 2, 4, np.random.default_rng(0), kappa=50.0)


def test_dropped_rank_one_correction(monkeypatch):
    hs = hsde.HSDE(_tiny())
    def bad(self, omega):
        w12, w3 = omega[:-1], float(omega[-1])
        u12 = self.solve_M(w12 - w3 * self.zeta)           # no Sherman-Morrison term
        u3 = w3 + float(self.chat @ u12[:self.n1]) + float(self.bhat @ u12[self.n1:])
        return np.concatenate([u12, [u3]])
    monkeypatch.setattr(hsde.HSDE, "affine", bad)
    assert _affine_err(hs) > 1e-3


def test_wrong_half_in_factor(monkeypatch):
    hs = hsde.HSDE(_tiny())
    hs.Delta = 1.0 + hs.D                                   # D instead of D/2
    assert _affine_err(hs) > 1e-3


def test_printed_second_elimination_route_agrees():
    """The printed route (u2 from (I + Ahat Ahat^T) u2 = Ahat w1 + w2, then
    u1 = w1 - Ahat^T u2) is a valid elimination too and gives the same M^{-1};
    only the block matrix of Eq. ThirdBlkElm belongs to the other route."""
    hs = hsde.HSDE(_tiny())
    Ah = hs.Ahat.toarray()
    w = np.random.default_rng(1).standard_normal(hs.n1 + hs.n2)
    w1, w2 = w[:hs.n1], w[hs.n1:]
    u2 = np.linalg.solve(np.eye(Ah.shape[0]) + Ah @ Ah.T, Ah @ w1 + w2)
    printed = np.concatenate([w1 - Ah.T @ u2, u2])
    assert np.allclose(printed, hs.solve_M(w), atol=1e-10)


def test_wrong_sign_in_second_elimination(monkeypatch):
    hs = hsde.HSDE(_tiny())
    orig = hsde.HSDE.solve_M
    def bad(self, w):
        w = w.copy()
        w[self.n1:] *= -1.0                                 # u1 from w1 + Ahat^T w2
        out = orig(self, w)
        return out
    monkeypatch.setattr(hsde.HSDE, "solve_M", bad)
    hs.Minv_zeta = hs.solve_M(hs.zeta)
    hs.den = 1.0 + float(hs.zeta @ hs.Minv_zeta)
    assert _affine_err(hs) > 1e-3


def test_wrong_sign_nu_update(monkeypatch):
    def bad_step(self, u, nu):
        uhat = self.affine(u + nu)
        u_new = self.project_K(uhat - nu)
        return u_new, nu + uhat - u_new, uhat
    monkeypatch.setattr(hsde.HSDE, "step", bad_step)
    res = hsde.HSDE(synth.block_arrow_n50()).solve(max_iter=500)
    assert res.status != hsde.SOLVED


def test_missing_tau_clamp(monkeypatch):
    def bad_proj(self, w):
        out = w.copy()
        out[self.nF:self.nF + self.nd] = self.project_S(w[self.nF:self.nF + self.nd])
        return out                                          # tau not clamped at 0
    monkeypatch.setattr(hsde.HSDE, "project_K", bad_proj)
    res = hsde.HSDE(synth.block_arrow_n50(infeasible=True)).solve(max_iter=500)
    assert res.status != hsde.PRIMAL_INFEASIBLE


def test_transposed_clique_block(monkeypatch):
    """Flattening the projected block row-major instead of column-major is
    harmless for symmetric blocks; a missing symmetrisation is not."""
    orig = hsde.HSDE.project_S
    def bad(self, s):
        out = np.empty_like(s)
        for k, c in enumerate(self.cl_sizes):
            o = self.V.s_off[k]
            S = s[o:o + c * c].reshape((c, c), order="F")
            lam, V = np.linalg.eigh(S)                      # eigh reads one triangle only
            out[o:o + c * c] = ((V * np.maximum(lam, 0)) @ V.T).reshape(-1, order="F")
        return out
    monkeypatch.setattr(hsde.HSDE, "project_S", bad)
    hs = hsde.HSDE(synth.block_arrow_n50())
    rng = np.random.default_rng(3)
    s = rng.standard_normal(hs.nd)
    got = hs.project_S(s)
    monkeypatch.setattr(hsde.HSDE, "project_S", orig)
    want = hs.project_S(s)
    assert np.linalg.norm(got - want) > 1e-3


def test_unscaling_without_the_row_scaling(monkeypatch):
    """Forgetting D when mapping the scaled y back (y = y~/rho instead of
    D y~/rho) must break the hand-built optimum's verdict."""
    import tests.test_oracle_solve as tos
    def bad(self, u, nu):
        x, s, y, _, tau = self.split(u)
        z = nu[self.nF:self.nF + self.nd]
        return (x / self.sigma, s / self.sigma, y / self.rho, z / self.rho, tau, float(nu[-1]))
    p, Cm = tos._dense_trace_one(4, 3)
    hs = hsde.HSDE(p)
    assert not np.allclose(hs.d, 1.0)
    lam, V = np.linalg.eigh(Cm)
    X = np.outer(V[:, 0], V[:, 0]); Z = Cm - lam[0] * np.eye(4)
    vec = lambda M: np.array([M[i, j] for (i, j) in hs.V.ent])
    x, s, y, v, z = tos._to_scaled(hs, vec(X), hs.V.H @ vec(X), np.array([lam[0]]), hs.V.H @ vec(Z),
                                   hs.V.H @ vec(Z))
    u = np.concatenate([x, s, y, v, [1.0]])
    nu = np.concatenate([np.zeros(hs.nF), z, [0.0], np.zeros(hs.nd), [0.0]])
    assert hs.verdict(hs.residuals(u, nu), 1e-4) == hsde.SOLVED
    monkeypatch.setattr(hsde.HSDE, "unscale", bad)
    assert hs.verdict(hs.residuals(u, nu), 1e-4) != hsde.SOLVED


def test_relaxation_missing_in_the_dual_update(monkeypatch):
    """nu <- nu - u_hat + u_new (the relaxed point left out of Eq. Step3)
    must not solve the closed-form trace-one problem."""
    import tests.test_oracle_solve as tos
    def bad_step(self, u, nu):
        uhat = self.affine(u + nu)
        urel = self.alpha * uhat + (1.0 - self.alpha) * u
        u_new = self.project_K(urel - nu)
        return u_new, nu - uhat + u_new, uhat
    p, Cm = tos._dense_trace_one(5, 4)
    lam_min = np.linalg.eigvalsh(Cm).min()
    monkeypatch.setattr(hsde.HSDE, "step", bad_step)
    try:
        with np.errstate(all="ignore"):
            res = hsde.HSDE(p, alpha=1.8).solve(eps=1e-7, max_iter=5000)
    except np.linalg.LinAlgError:
        return                                              # diverged: caught
    assert not (res.status == hsde.SOLVED and abs(res.info["pobj"] - lam_min) <= 1e-4 * max(1.0, abs(lam_min)))
