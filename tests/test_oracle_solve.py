"""Pins of the oracle's whole solve: closed-form optima, hand-built points
for each verdict of the stopping rule (readings P5/P6), the constructed
infeasible instances with their certificates, and the Grone/Agler and
fixed-point invariants at convergence (Theorems 1-2, Eq. ADMMForm).

Every pin runs on the literal iteration (alpha = 1, no scaling) and on the
practical variant of reading P7 (over-relaxation and data scaling): the
closed forms and the verdicts must not depend on either.  The hand-built
points are written in the original variables and mapped into the scaled
ones by the definition of the scaling (x~ = sigma x, s~ = sigma s,
y~ = rho D^{-1} y, v~ = rho v, z~ = rho z), so a wrong unscaling in the
stopping rule fails them."""
import numpy as np
import pytest

import synth
from oracle import dense, hsde, symbolic


def _sym_from_lower(n, r, c, v):
    M = np.zeros((n, n))
    M[r, c] = v
    M[c, r] = v
    return M


def _random_C_on_block_arrow(l, d, h, seed):
    rng = np.random.default_rng(seed)
    r, c = [], []
    for mem in synth.block_arrow_cliques(l, d, h):
        for b in range(len(mem)):
            for a in range(b, len(mem)):
                r.append(mem[a]); c.append(mem[b])
    key = sorted(set(zip(r, c)), key=lambda t: (t[1], t[0]))
    r = np.array([k[0] for k in key], np.int32); c = np.array([k[1] for k in key], np.int32)
    return r, c, rng.standard_normal(len(r))


FORMS = {"literal": dict(alpha=1.0, scaling=False), "relaxed_scaled": dict(alpha=1.8, scaling=True)}


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("l,d,h,seed", [(3, 3, 2, 0), (4, 2, 1, 1), (2, 4, 2, 2)])
def test_trace_one_gives_lambda_min(l, d, h, seed, form):
    n = l * d + h
    r, c, v = _random_C_on_block_arrow(l, d, h, seed)
    p = synth.trace_one(r, c, v, n)
    lam_min = np.linalg.eigvalsh(_sym_from_lower(n, r, c, v)).min()
    res = hsde.HSDE(p, **FORMS[form]).solve(eps=1e-7, max_iter=50000)
    assert res.status == hsde.SOLVED
    assert abs(res.info["pobj"] - lam_min) <= 1e-4 * max(1.0, abs(lam_min))
    assert abs(res.info["dobj"] - lam_min) <= 1e-4 * max(1.0, abs(lam_min))


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("w", [1.0, -1.0, 2.5, -0.3])
def test_two_node_maxcut(w, form):
    """min <L_w, X> s.t. X_11 = X_22 = 1, X psd: 2w - 2|w| (X_12 = sign(w))."""
    p = synth.Problem("mc2", 2, 2, np.array([0, 1, 1], np.int32), np.array([0, 0, 1], np.int32),
                      np.array([w, -w, w]), np.array([0, 1, 2], np.int64), np.array([0, 1], np.int32),
                      np.array([0, 1], np.int32), np.ones(2), np.ones(2))
    res = hsde.HSDE(p, **FORMS[form]).solve(eps=1e-8, max_iter=50000)
    assert res.status == hsde.SOLVED
    assert abs(res.info["pobj"] - (2 * w - 2 * abs(w))) <= 1e-5


def _dense_trace_one(n, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n)); Cm = 0.5 * (G + G.T)
    ii, jj = np.tril_indices(n)
    order = np.lexsort((ii, jj))
    return synth.trace_one(ii[order], jj[order], Cm[ii[order], jj[order]], n), Cm


def _to_scaled(hs, x=None, s=None, y=None, v=None, z=None):
    """Original variables -> the scaled ones the iteration carries (by the
    definition of the scaling, not by the oracle's unscale())."""
    out = []
    for val, f in ((x, hs.sigma), (s, hs.sigma), (v, hs.rho), (z, hs.rho)):
        out.append(None if val is None else f * val)
    ys = None if y is None else hs.rho * y / hs.d
    return out[0], out[1], ys, out[2], out[3]


@pytest.mark.parametrize("form", list(FORMS))
def test_verdict_solved_on_hand_built_optimum(form):
    p, Cm = _dense_trace_one(4, 3)
    hs = hsde.HSDE(p, **FORMS[form])
    lam, V = np.linalg.eigh(Cm)
    X = np.outer(V[:, 0], V[:, 0]); Z = Cm - lam[0] * np.eye(4)
    vec = lambda M: np.array([M[i, j] for (i, j) in hs.V.ent])
    x, s, y, v, z = _to_scaled(hs, vec(X), hs.V.H @ vec(X), np.array([lam[0]]), hs.V.H @ vec(Z),
                               hs.V.H @ vec(Z))
    u = np.concatenate([x, s, y, v, [1.0]])
    nu = np.concatenate([np.zeros(hs.nF), z, [0.0], np.zeros(hs.nd), [0.0]])
    info = hs.residuals(u, nu)
    assert info["pres"] < 1e-12 and info["dres"] < 1e-12 and info["gap"] < 1e-12
    assert info["pobj"] == pytest.approx(lam[0], rel=1e-12)
    assert hs.verdict(info, 1e-4) == hsde.SOLVED
    # a wrong sign on y must not pass
    u_bad = u.copy(); u_bad[hs.nF + hs.nd] = -y[0]
    assert hs.verdict(hs.residuals(u_bad, nu), 1e-4) != hsde.SOLVED
    # nu = Q u at this point (Eq. ADMMForm), with kappa = 0
    assert np.allclose(dense.build_Q(hs) @ u, nu, atol=1e-12)


@pytest.mark.parametrize("form", list(FORMS))
def test_verdict_primal_infeasible_closed_form_certificate(form):
    """tr X = -1 appended: y = -e_{m+1}, z_k = diag(1/D) on each clique gives
    A^T y + H^T z = 0 and b^T y = 1."""
    p = synth.block_arrow_n50(infeasible=True)
    hs = hsde.HSDE(p, **FORMS[form])
    st = hs.V.st
    y = np.zeros(hs.m); y[-1] = -1.0
    Dfull = hs.D
    z = np.zeros(hs.nd)
    for k, mem in enumerate(st.cliques):
        c = len(mem)
        for a in range(c):
            e = hs.V.fpos[(int(mem[a]), int(mem[a]))]
            z[hs.V.s_off[k] + a + a * c] = 1.0 / Dfull[e]
    _, _, y, _, z = _to_scaled(hs, y=y, z=z)
    u = np.concatenate([np.zeros(hs.nF), np.zeros(hs.nd), y, np.zeros(hs.nd), [0.0]])
    nu = np.concatenate([np.zeros(hs.nF), z, np.zeros(hs.m), np.zeros(hs.nd), [1.0]])
    info = hs.residuals(u, nu)
    assert info["bty"] == pytest.approx(1.0)
    assert info["pinf_ratio"] < 1e-14
    assert hs.verdict(info, 1e-4) == hsde.PRIMAL_INFEASIBLE


@pytest.mark.parametrize("form", list(FORMS))
def test_verdict_dual_infeasible_hand_built_direction(form):
    base = synth.block_arrow(3, 3, 2, 5, synth.rng_for(9), kappa=50.0, assign="roundrobin")
    p = synth.make_dual_infeasible(base, np.random.default_rng(1))
    hs = hsde.HSDE(p, **FORMS[form])
    Dr, Dc, Dv = p.meta["Dd"]
    Dm = _sym_from_lower(p.n, Dr, Dc, Dv)
    x = np.array([Dm[i, j] for (i, j) in hs.V.ent])
    x, s, _, _, _ = _to_scaled(hs, x=x, s=hs.V.H @ x)
    u = np.concatenate([x, s, np.zeros(hs.m), np.zeros(hs.nd), [0.0]])
    nu = np.concatenate([np.zeros(hs.nF), np.zeros(hs.nd), np.zeros(hs.m), np.zeros(hs.nd), [1.0]])
    info = hs.residuals(u, nu)
    assert info["ctx"] == pytest.approx(-1.0)
    assert info["dinf_ratio"] < 1e-12
    assert hs.verdict(info, 1e-4) == hsde.DUAL_INFEASIBLE


@pytest.mark.parametrize("form", list(FORMS))
def test_block_arrow_n50_solution_invariants(form):
    p = synth.block_arrow_n50()
    hs = hsde.HSDE(p, **FORMS[form])
    res = hs.solve(eps=1e-6, max_iter=20000)
    assert res.status == hsde.SOLVED
    X, y, Z = hs.solution(res.u, res.nu)
    st = hs.V.st
    scale = np.abs(X).max()
    # Grone (Theorem 1): every clique block of X psd
    for mem in st.cliques:
        Xk = np.array([[X[hs.V.fpos[(int(a), int(b))]] for b in mem] for a in mem])
        assert np.linalg.eigvalsh(Xk).min() >= -1e-5 * scale
    # Agler (Theorem 2): Z = sum_k E_k^T Z_k E_k with psd Z_k (z is psd exactly)
    z = res.nu[hs.nF:hs.nF + hs.nd] / res.u[-1]
    for k, mem in enumerate(st.cliques):
        c = len(mem)
        Zk = z[hs.V.s_off[k]:hs.V.s_off[k] + c * c].reshape((c, c), order="F")
        assert np.linalg.eigvalsh(0.5 * (Zk + Zk.T)).min() >= -1e-9 * np.abs(Zk).max()
    # C - sum_i y_i A_i - Z ~ 0 on the pattern
    r = hs.V.c - hs.V.A.T @ y - Z
    assert np.linalg.norm(r) <= 1e-5 * (1 + np.linalg.norm(hs.V.c))
    # complementarity <s, z> ~ 0 and tau*kappa = 0
    s = res.u[hs.nF:hs.nF + hs.nd]
    assert abs(s @ res.nu[hs.nF:hs.nF + hs.nd]) <= 1e-6 * np.linalg.norm(s) * np.linalg.norm(res.nu[hs.nF:hs.nF + hs.nd]) + 1e-12
    assert res.u[-1] * res.nu[-1] == 0.0
    # fixed point of Eq. ADMMForm: nu ~ Q u
    Q = dense.build_Q(hs)
    assert np.linalg.norm(Q @ res.u - res.nu) <= 1e-4 * np.linalg.norm(res.u)


@pytest.mark.parametrize("form", list(FORMS))
def test_primal_infeasible_instance_gives_valid_certificate(form):
    p = synth.block_arrow_n50(infeasible=True)
    hs = hsde.HSDE(p, **FORMS[form])
    res = hs.solve()
    assert res.status == hsde.PRIMAL_INFEASIBLE
    y, Z = hs.certificate(res.u, res.nu, res.status)
    assert hs.V.b @ y == pytest.approx(1.0)
    assert np.linalg.norm(hs.V.A.T @ y + Z) <= 1e-4
    z = res.nu[hs.nF:hs.nF + hs.nd]
    for k, mem in enumerate(hs.V.st.cliques):
        c = len(mem)
        Zk = z[hs.V.s_off[k]:hs.V.s_off[k] + c * c].reshape((c, c), order="F")
        assert np.linalg.eigvalsh(0.5 * (Zk + Zk.T)).min() >= -1e-9 * np.abs(Zk).max()


@pytest.mark.parametrize("form", list(FORMS))
def test_dual_infeasible_instance_gives_valid_certificate(form):
    base = synth.block_arrow(4, 4, 2, 8, synth.rng_for(8), kappa=100.0, assign="roundrobin")
    p = synth.make_dual_infeasible(base, np.random.default_rng(2))
    hs = hsde.HSDE(p, **FORMS[form])
    res = hs.solve(max_iter=20000)
    assert res.status == hsde.DUAL_INFEASIBLE
    x, s = hs.certificate(res.u, res.nu, res.status)
    assert hs.V.c @ x == pytest.approx(-1.0)
    assert np.sqrt(np.sum((hs.V.A @ x) ** 2) + np.sum((hs.V.H @ x - s) ** 2)) <= 1e-4
    for k, mem in enumerate(hs.V.st.cliques):
        c = len(mem)
        Sk = s[hs.V.s_off[k]:hs.V.s_off[k] + c * c].reshape((c, c), order="F")
        assert np.linalg.eigvalsh(0.5 * (Sk + Sk.T)).min() >= -1e-9 * max(1e-30, np.abs(Sk).max())


@pytest.mark.parametrize("form", list(FORMS))
def test_feasible_block_arrow_n50_reaches_tolerance(form):
    res = hsde.HSDE(synth.block_arrow_n50(), **FORMS[form]).solve()
    assert res.status == hsde.SOLVED and res.iterations < 2000


def test_scaling_factors_normalise_the_rows_and_keep_the_b_to_c_ratio():
    hs = hsde.HSDE(synth.block_arrow_n50())
    A0 = hs.V.A.toarray()
    rows = np.linalg.norm(hs.A.toarray(), axis=1)
    assert np.allclose(rows, 1.0, rtol=1e-14)
    # b~ and c~ are the original b and c times one factor (times the dual
    # weight on c), so the scaled pair describes the same problem
    assert np.allclose(hs.b / hs.sigma, hs.d * hs.V.b, rtol=1e-14)
    assert np.allclose(hs.c / hs.rho, hs.V.c, rtol=1e-14)
    assert np.allclose(hs.A.toarray(), A0 * hs.d[:, None], rtol=1e-14)
    assert max(np.linalg.norm(hs.b), np.linalg.norm(hs.c) / hsde.DUAL_WEIGHT) == pytest.approx(hsde.SCALE_NORM)


@pytest.mark.parametrize("name", ["n50", "n50_inf"])
def test_relaxed_scaled_and_literal_forms_reach_the_same_point(name):
    """Reading P7 changes the path, not where it ends: the optimum (or the
    certificate) of the relaxed, scaled iteration equals the literal one."""
    p = synth.block_arrow_n50(infeasible=(name == "n50_inf"))
    a = hsde.HSDE(p, alpha=1.0, scaling=False)
    b = hsde.HSDE(p, alpha=1.8, scaling=True)
    ra = a.solve(eps=1e-8, max_iter=50000)
    rb = b.solve(eps=1e-8, max_iter=50000)
    assert ra.status == rb.status
    if ra.status == hsde.SOLVED:
        Xa, ya, Za = a.solution(ra.u, ra.nu)
        Xb, yb, Zb = b.solution(rb.u, rb.nu)
        for u, w in ((Xa, Xb), (ya, yb), (Za, Zb)):
            assert np.linalg.norm(u - w) <= 1e-4 * max(1.0, np.linalg.norm(u))
        assert rb.info["pobj"] == pytest.approx(ra.info["pobj"], rel=1e-6)
    else:
        ca, cb = a.certificate(ra.u, ra.nu, ra.status), b.certificate(rb.u, rb.nu, rb.status)
        # certificates are not unique; each must be valid
        for (y, Z) in (ca, cb):
            assert a.V.b @ y == pytest.approx(1.0)
            assert np.linalg.norm(a.V.A.T @ y + Z) <= 1e-6


def test_no_certificate_from_a_first_iterate_that_does_not_cancel():
    """Reading P6's cancellation condition: on the l = 500 block-arrow (feasible
    by construction, ||b|| ~ 5e5) the first iterate already has tau = 0 and
    ||A^T y + H^T z|| / b^T y below 1e-4, but A^T y and H^T z do not cancel;
    the ratio alone would call the instance primal infeasible."""
    hs = hsde.HSDE(synth.block_arrow_sweep(500, 10))
    u, nu = hs.initial()
    u, nu, _ = hs.step(u, nu)
    info = hs.residuals(u, nu)
    assert info["tau"] == 0.0 and info["bty"] > 0
    assert info["pinf_ratio"] <= 1e-4                   # the ratio alone passes
    assert info["pinf_cancel"] > 0.1                    # the terms do not cancel
    assert hs.verdict(info, 1e-4) == hsde.RUNNING
