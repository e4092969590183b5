"""HSDE-ADMM oracle (test infrastructure), FP64, literal and slow.

Follows the paper step by step:

* Section 3.1, Eqs. PrimalVectorForm / DualVectorForm: x = vec(X) with the
  usual column-stack vec, x_k = H_k x = vec(E_k X E_k^T), s = (x_1..x_p).
  Reading P1: entries of vec(X) outside the chordal pattern E' carry no data
  (A, c and D vanish there) and stay exactly zero from the zero start, so x is
  stored on BOTH triangles of E' only; all inner products and norms are then
  the plain Euclidean (Frobenius) ones.  ``Vectorised(full_space=True)`` keeps
  all n^2 entries instead and is used by the tests to pin this reading.
* Section 3.2, Eq. HomogeneousEmbedding / ADMMForm: u = (x, s, y, v, tau),
  nu = (h, z, r, w, kappa) (the paper calls the second vector v as well), and
  the cone K = R^{n^2} x S x R^m x R^{n_d} x R_+.
* Section 4.1, Eqs. Step1-Step3: the three ADMM steps.
* Section 4.2, Eqs. LinearSystem, MatrixInverse, FirstBlockElimination,
  MatrixInverseResult: first block elimination of the tau row and the rank-one
  correction with the cached M^{-1} zeta and 1 + zeta^T M^{-1} zeta.
* Section 4.3, Eqs. SecondBlockElimination, ThirdBlkElm, FactorizationMatrix:
  the inner system.  Reading P2: the printed second elimination (solve for
  u2 with I + Ahat Ahat^T) is a valid route, but the block matrix written in
  Eq. ThirdBlkElm is that of I + Ahat^T Ahat, which belongs to the other
  route: eliminate u2 = w2 + Ahat u1 and solve
  (I + Ahat^T Ahat) u1 = w1 - Ahat^T w2.  Only that route leads to Eq.
  FactorizationMatrix, so it is the one followed here.  Eliminating s from
  Eq. ThirdBlkElm leaves (I + D/2 + A^T A) x = r1 + H^T r2 / 2 and
  s = (r2 + H x)/2, solved with the matrix inversion lemma on
  Delta + A^T A, Delta = I + D/2: only S = I + A Delta^{-1} A^T (m x m) is
  factored (LAPACK Cholesky through scipy).
* Reading P4: u0 = (0,0,0,0,1), nu0 = (0,0,0,0,1).
* Readings P5/P6 (the paper only states eps_tol = 1e-4 and 2000 iterations):
  with xb = x/tau, sb = s/tau, yb = y/tau, zb = z/tau
    pres = ||(A xb - b, H xb - sb)|| / (1 + ||b||)
    dres = ||A^T yb + H^T zb - c|| / (1 + ||c||)
    gap  = |c^T xb - b^T yb| / (1 + |c^T xb| + |b^T yb|)
  SOLVED iff tau > 0 and all three <= eps; else PRIMAL_INFEASIBLE iff
  b^T y > 0 and ||A^T y + H^T z|| / b^T y <= eps and the two terms cancel,
  ||A^T y + H^T z|| <= CERT_CANCEL (||A^T y|| + ||H^T z||); else
  DUAL_INFEASIBLE iff c^T x < 0 and ||(A x, H x - s)|| / (-c^T x) <= eps and
  ||(A x, H x - s)|| <= CERT_CANCEL (||H x|| + ||s||).  Checked after every
  ``check_every``-th iteration; MAX_ITER when max_iter is reached.
  The cancellation condition is part of the reading: the ratio alone is not
  invariant to the scale of b (or c), and on block-arrows whose b is large
  (||b|| ~ 5e5) the first iterate, with tau already 0, has a ratio of 9e-5
  although the instance is feasible; its two terms do not cancel at all.
* Reading P7 (the paper applies the cited ADMM of O'Donoghue et al.
  "directly" and says nothing of its practical variants): optional
  over-relaxation and data scaling, both switched by arguments.
    - Relaxation: with u_hat = (I+Q)^{-1}(u + nu) and
      u_rel = alpha u_hat + (1 - alpha) u, the cone step projects u_rel - nu
      and the dual update is nu <- nu - u_rel + u_new.  alpha = 1 is the
      literal Eqs. Step1-Step3.
    - Scaling: the iteration runs on A~ = D A, b~ = sigma D b, c~ = rho c with
      D = diag(1 / ||A_i||) (every constraint row of unit full-vec norm) and
      scalars sigma, rho (see scaling_factors).  The constraint
      set x in K, the cliques and H are untouched: the scaled problem has
      x~ = sigma x, s~ = sigma s, y~ = rho D^{-1} y, z~ = rho z.  The stopping
      rule (P5/P6) is evaluated on the unscaled iterate against the original
      data, so verdicts mean the same with and without scaling.
* Reading P8: each clique block is symmetrised before its eigendecomposition;
  for a c^2-vector this IS the Euclidean projection onto vec(S^c_+).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import symbolic

RUNNING, SOLVED, PRIMAL_INFEASIBLE, DUAL_INFEASIBLE, MAX_ITER = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "running", 1: "solved", 2: "primal_infeasible", 3: "dual_infeasible",
                4: "max_iter"}

# Defaults of the practical variants (reading P7); the library's defaults are
# the same values.  They were chosen by running this oracle to the 1e-4
# verdict on the synthetic workloads (the n = 2000 max-cut grid, the n = 50
# and l = 100 block-arrows) over alpha in {1, 1.6, 1.8, 1.9}, the target norm
# in {0.1, 1, 10, 100} and the dual weight in {0.3, 1, 1.5, 2, 3, 10}.
ALPHA = 1.8
SCALE_NORM = 10.0
DUAL_WEIGHT = 1.5
# certificates must also cancel to this fraction of their terms (reading P6)
CERT_CANCEL = 1e-2


class Vectorised:
    """Section 3.1: vectorised data (c, A, H) of the decomposed primal-dual pair."""

    def __init__(self, prob, st: symbolic.Structure | None = None, full_space=False):
        self.prob = prob
        self.st = st if st is not None else symbolic.analyze(prob)
        n = prob.n
        self.n = n
        if full_space:
            ent = [(i, j) for j in range(n) for i in range(n)]
        else:
            ent = []
            for r, c in zip(self.st.pat_row.tolist(), self.st.pat_col.tolist()):
                ent.append((r, c))
                if r != c:
                    ent.append((c, r))
            ent.sort(key=lambda rc: (rc[1], rc[0]))        # column-stack vec order
        self.ent = ent
        self.fpos = {rc: i for i, rc in enumerate(ent)}
        nF = len(ent)
        self.nF = nF
        # H_k = E_Ck (x) E_Ck: row a + b*c of block k selects X(C_k(a), C_k(b))
        rows, cols = [], []
        off = 0
        self.s_off = []
        for mem in self.st.cliques:
            ml = mem.tolist()
            c = len(ml)
            self.s_off.append(off)
            for b in range(c):
                for a in range(c):
                    rows.append(off + a + b * c)
                    cols.append(self.fpos[(ml[a], ml[b])])
            off += c * c
        self.n_d = off
        self.H = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(off, nF))
        # A := [vec(A_1) ... vec(A_m)]^T  and c := vec(C)
        ar, ac, av = [], [], []
        for i in range(prob.m):
            s = slice(int(prob.A_ptr[i]), int(prob.A_ptr[i + 1]))
            for r, cc, v in zip(prob.A_row[s].tolist(), prob.A_col[s].tolist(), prob.A_val[s].tolist()):
                ar.append(i); ac.append(self.fpos[(r, cc)]); av.append(v)
                if r != cc:
                    ar.append(i); ac.append(self.fpos[(cc, r)]); av.append(v)
        self.A = sp.csr_matrix((av, (ar, ac)), shape=(prob.m, nF))
        cvec = np.zeros(nF)
        for r, cc, v in zip(prob.C_row.tolist(), prob.C_col.tolist(), prob.C_val.tolist()):
            cvec[self.fpos[(r, cc)]] += v
            if r != cc:
                cvec[self.fpos[(cc, r)]] += v
        self.c = cvec
        self.b = np.asarray(prob.b, dtype=np.float64).copy()
        self.m = prob.m

    # ----- conversions to the library's packed-lower layout (for parity tests) -----
    def x_to_lower(self, x):
        st = self.st
        return np.array([x[self.fpos[(r, c)]] for r, c in zip(st.pat_row.tolist(), st.pat_col.tolist())])

    def x_from_lower(self, xl):
        x = np.zeros(self.nF)
        st = self.st
        for e, (r, c) in enumerate(zip(st.pat_row.tolist(), st.pat_col.tolist())):
            x[self.fpos[(r, c)]] = xl[e]
            x[self.fpos[(c, r)]] = xl[e]
        return x

    def s_to_packed(self, s):
        out = []
        for k, mem in enumerate(self.st.cliques):
            c = len(mem)
            S = s[self.s_off[k]:self.s_off[k] + c * c].reshape((c, c), order="F")
            for b in range(c):
                out.extend(S[b:, b].tolist())
        return np.array(out)

    def s_from_packed(self, sp_):
        out = np.zeros(self.n_d)
        pp = self.st.packed_ptr
        for k, mem in enumerate(self.st.cliques):
            c = len(mem)
            S = np.zeros((c, c))
            seg = sp_[pp[k]:pp[k + 1]]
            t = 0
            for b in range(c):
                S[b:, b] = seg[t:t + c - b]
                t += c - b
            S = S + np.tril(S, -1).T
            out[self.s_off[k]:self.s_off[k] + c * c] = S.reshape(-1, order="F")
        return out


def project_psd(S):
    """Euclidean projection of a (possibly non-symmetric) square block onto the
    psd cone: symmetrise, eigendecompose, clamp eigenvalues at 0, rebuild."""
    S = 0.5 * (S + S.T)
    lam, V = np.linalg.eigh(S)
    return (V * np.maximum(lam, 0.0)) @ V.T


@dataclass
class Result:
    status: int
    iterations: int
    u: np.ndarray
    nu: np.ndarray
    info: dict
    history: list = field(default_factory=list)


def scaling_factors(V, enabled=True, target=None, dual_weight=None):
    """Reading P7: the data scaling (D, sigma, rho) of the vectorised pair V.

    D = diag(d), d_i = 1 / ||A_i|| (full-vec Frobenius norm of constraint i;
    1 for an all-zero row), so every scaled constraint row has unit norm.
    With M = max(||D b||, ||c||): sigma = target / M and
    rho = dual_weight * target / M (sigma = rho = 1 when M = 0).  One common
    factor keeps the ratio of ||b|| to ||c||; dual_weight > 1 gives the dual
    side a little more weight.  Disabled: D = I, sigma = rho = 1."""
    m = V.m
    if not enabled:
        return np.ones(m), 1.0, 1.0
    target = SCALE_NORM if target is None else float(target)
    dual_weight = DUAL_WEIGHT if dual_weight is None else float(dual_weight)
    rn = np.sqrt(np.asarray(V.A.multiply(V.A).sum(axis=1)).ravel()) if m > 0 else np.zeros(0)
    d = np.where(rn > 0, 1.0 / np.where(rn > 0, rn, 1.0), 1.0)
    nb = float(np.linalg.norm(d * V.b)) if m > 0 else 0.0
    nc = float(np.linalg.norm(V.c))
    mx = max(nb, nc)
    if mx == 0.0:
        return d, 1.0, 1.0
    return d, target / mx, dual_weight * target / mx


class HSDE:
    """The ADMM of Section 4 on the embedding of Section 3.2.

    alpha: over-relaxation (reading P7; 1 = the literal Eqs. Step1-Step3).
    scaling: run on the scaled data A~ = D A, b~ = sigma D b, c~ = rho c
    (reading P7).  The attributes A, b, c are the data the iteration uses
    (scaled or not); V keeps the original vectorised pair."""

    def __init__(self, prob, st=None, full_space=False, vec: Vectorised | None = None,
                 alpha=ALPHA, scaling=True, scale_norm=None, dual_weight=None):
        self.V = vec if vec is not None else Vectorised(prob, st, full_space)
        V = self.V
        self.alpha = float(alpha)
        self.scaled = bool(scaling)
        self.d, self.sigma, self.rho = scaling_factors(V, self.scaled, scale_norm, dual_weight)
        self.A = (sp.diags(self.d) @ V.A).tocsr() if V.m > 0 else V.A
        self.b = self.sigma * self.d * V.b
        self.c = self.rho * V.c
        A, H = self.A, V.H
        nF, nd, m = V.nF, V.n_d, V.m
        self.nF, self.nd, self.m = nF, nd, m
        self.n1 = nF + nd                      # length of u1 = (x, s)
        self.n2 = m + nd                       # length of u2 = (y, v)
        self.dim = self.n1 + self.n2 + 1
        # Section 4.3: D := H^T H is diagonal
        HtH = (H.T @ H).tocsr()
        self.D = HtH.diagonal().copy()
        off = HtH - sp.diags(self.D)
        assert abs(off).sum() == 0.0, "H^T H must be diagonal"
        # Section 4.2: Ahat, chat, bhat, M, zeta
        I_nd = sp.identity(nd, format="csr")
        self.Ahat = sp.bmat([[-A, None], [-H, I_nd]], format="csr")
        self.chat = np.concatenate([self.c, np.zeros(nd)])
        self.bhat = np.concatenate([-self.b, np.zeros(nd)])
        self.zeta = np.concatenate([self.chat, self.bhat])
        # Eq. FactorizationMatrix, I + D/2 + A^T A, through the matrix inversion lemma
        self.Delta = 1.0 + 0.5 * self.D
        Dinv = sp.diags(1.0 / self.Delta)
        S = (sp.identity(m) + A @ Dinv @ A.T).toarray() if m > 0 else np.zeros((0, 0))
        self.S_cho = sla.cho_factor(S, lower=True) if m > 0 else None
        # cached M^{-1} zeta and 1 + zeta^T M^{-1} zeta (Eq. MatrixInverseResult)
        self.Minv_zeta = self.solve_M(self.zeta)
        self.den = 1.0 + float(self.zeta @ self.Minv_zeta)
        # clique bookkeeping for the cone projection
        self.cl_sizes = [len(c) for c in V.st.cliques]

    # ---------------- affine projection, Eq. Step1 ----------------
    def solve_factor(self, g):
        """(Delta + A^T A)^{-1} g by the matrix inversion lemma,
        Delta^{-1} - Delta^{-1} A^T (I + A Delta^{-1} A^T)^{-1} A Delta^{-1}."""
        A = self.A
        h = g / self.Delta
        if self.m == 0:
            return h
        t = sla.cho_solve(self.S_cho, A @ h)
        return h - (A.T @ t) / self.Delta

    def solve_M(self, w):
        """M^{-1} w for M = [[I, Ahat^T], [-Ahat, I]] (Eq. SecondBlockElimination,
        eliminating u2 so that Eq. ThirdBlkElm's matrix I + Ahat^T Ahat appears)."""
        n1, nF = self.n1, self.nF
        H = self.V.H
        w1, w2 = w[:n1], w[n1:]
        rhs = w1 - self.Ahat.T @ w2                 # (I + Ahat^T Ahat) u1 = w1 - Ahat^T w2
        r1, r2 = rhs[:nF], rhs[nF:]
        x = self.solve_factor(r1 + 0.5 * (H.T @ r2))  # Eq. ThirdBlkElm with s eliminated
        s = 0.5 * (r2 + H @ x)
        u1 = np.concatenate([x, s])
        u2 = w2 + self.Ahat @ u1
        return np.concatenate([u1, u2])

    def affine(self, omega):
        """u_hat = (I+Q)^{-1} omega via Eqs. MatrixInverse, FirstBlockElimination
        and MatrixInverseResult."""
        w12, w3 = omega[:-1], float(omega[-1])
        t = self.solve_M(w12 - w3 * self.zeta)
        u12 = t - self.Minv_zeta * (float(self.zeta @ t) / self.den)
        u3 = w3 + float(self.chat @ u12[:self.n1]) + float(self.bhat @ u12[self.n1:])
        return np.concatenate([u12, [u3]])

    # ---------------- cone projection, Eq. Step2 ----------------
    def split(self, u):
        nF, nd, m = self.nF, self.nd, self.m
        x = u[:nF]
        s = u[nF:nF + nd]
        y = u[nF + nd:nF + nd + m]
        v = u[nF + nd + m:nF + 2 * nd + m]
        return x, s, y, v, float(u[-1])

    def project_S(self, s):
        """Projection onto S = S_1 x ... x S_p, each clique block separately
        (blocks of equal size are batched through one LAPACK call)."""
        out = np.empty_like(s)
        offs = self.V.s_off
        by_size = {}
        for k, c in enumerate(self.cl_sizes):
            by_size.setdefault(c, []).append(k)
        for c, ks in by_size.items():
            blocks = np.stack([s[offs[k]:offs[k] + c * c].reshape((c, c), order="F") for k in ks])
            blocks = 0.5 * (blocks + np.transpose(blocks, (0, 2, 1)))
            lam, Vv = np.linalg.eigh(blocks)
            P = np.einsum("kij,kj,klj->kil", Vv, np.maximum(lam, 0.0), Vv)
            for t, k in enumerate(ks):
                out[offs[k]:offs[k] + c * c] = P[t].reshape(-1, order="F")
        return out

    def project_K(self, w):
        """Pi_K for K = R^{n^2} x S x R^m x R^{n_d} x R_+."""
        nF, nd = self.nF, self.nd
        out = w.copy()
        out[nF:nF + nd] = self.project_S(w[nF:nF + nd])
        out[-1] = max(0.0, float(w[-1]))
        return out

    # ---------------- one ADMM iteration, Eqs. Step1-Step3 ----------------
    def initial(self):
        u = np.zeros(self.dim); u[-1] = 1.0
        nu = np.zeros(self.dim); nu[-1] = 1.0
        return u, nu

    def step(self, u, nu):
        uhat = self.affine(u + nu)                 # Eq. Step1
        urel = self.alpha * uhat + (1.0 - self.alpha) * u   # relaxation (reading P7)
        u_new = self.project_K(urel - nu)          # Eq. Step2
        nu_new = nu - urel + u_new                 # Eq. Step3
        return u_new, nu_new, uhat

    # ---------------- unscaling (reading P7) ----------------
    def unscale(self, u, nu):
        """The iterate of the original problem from that of the scaled one:
        x = x~/sigma, s = s~/sigma, y = D y~/rho, z = z~/rho (tau, kappa as they are)."""
        x, s, y, _, tau = self.split(u)
        z = nu[self.nF:self.nF + self.nd]
        return (x / self.sigma, s / self.sigma, self.d * y / self.rho, z / self.rho, tau, float(nu[-1]))

    # ---------------- stopping rule and certificates (P5/P6) ----------------
    def residuals(self, u, nu):
        """Readings P5/P6 on the unscaled iterate against the original data."""
        V = self.V
        A, H, c, b = V.A, V.H, V.c, V.b
        x, s, y, z, tau, kappa = self.unscale(u, nu)
        Ax = A @ x
        Hx_s = H @ x - s
        Aty_Htz = A.T @ y + H.T @ z
        ctx, bty = float(c @ x), float(b @ y)
        info = dict(tau=tau, kappa=kappa, ctx=ctx, bty=bty)
        if tau > 0:
            pres = np.sqrt(np.sum((Ax / tau - b) ** 2) + np.sum((Hx_s / tau) ** 2)) / (1 + np.linalg.norm(b))
            dres = np.linalg.norm(Aty_Htz / tau - c) / (1 + np.linalg.norm(c))
            gap = abs(ctx / tau - bty / tau) / (1 + abs(ctx / tau) + abs(bty / tau))
            info.update(pres=pres, dres=dres, gap=gap, pobj=ctx / tau, dobj=bty / tau)
        else:
            info.update(pres=np.inf, dres=np.inf, gap=np.inf, pobj=np.nan, dobj=np.nan)
        info["pinf_ratio"] = (np.linalg.norm(Aty_Htz) / bty) if bty > 0 else np.inf
        info["dinf_ratio"] = (np.sqrt(np.sum(Ax ** 2) + np.sum(Hx_s ** 2)) / (-ctx)) if ctx < 0 else np.inf
        # how far the two terms of each certificate cancel (scale-free)
        den_p = np.linalg.norm(A.T @ y) + np.linalg.norm(H.T @ z)
        den_d = np.linalg.norm(H @ x) + np.linalg.norm(s)
        info["pinf_cancel"] = np.linalg.norm(Aty_Htz) / den_p if den_p > 0 else np.inf
        info["dinf_cancel"] = np.sqrt(np.sum(Ax ** 2) + np.sum(Hx_s ** 2)) / den_d if den_d > 0 else np.inf
        return info

    def verdict(self, info, eps):
        if info["tau"] > 0 and info["pres"] <= eps and info["dres"] <= eps and info["gap"] <= eps:
            return SOLVED
        if info["bty"] > 0 and info["pinf_ratio"] <= eps and info["pinf_cancel"] <= CERT_CANCEL:
            return PRIMAL_INFEASIBLE
        if info["ctx"] < 0 and info["dinf_ratio"] <= eps and info["dinf_cancel"] <= CERT_CANCEL:
            return DUAL_INFEASIBLE
        return RUNNING

    def solve(self, eps=1e-4, max_iter=2000, check_every=1, u0=None, nu0=None, record=False):
        u, nu = self.initial() if u0 is None else (u0.copy(), nu0.copy())
        hist = []
        status = RUNNING
        it = 0
        info = {}
        while it < max_iter:
            u, nu, _ = self.step(u, nu)
            it += 1
            if it % check_every == 0 or it == max_iter:
                info = self.residuals(u, nu)
                if record:
                    hist.append(dict(it=it, **{k: info[k] for k in ("pres", "dres", "gap", "tau", "kappa")}))
                status = self.verdict(info, eps)
                if status != RUNNING:
                    break
        if status == RUNNING:
            status = MAX_ITER
        return Result(status, it, u, nu, info, hist)

    # ---------------- recovery ----------------
    def solution(self, u, nu):
        """X = x/tau, y/tau and the Agler sum Z = H^T z / tau (Theorem 2), unscaled."""
        x, s, y, z, tau, _ = self.unscale(u, nu)
        return x / tau, y / tau, (self.V.H.T @ z) / tau

    def certificate(self, u, nu, status):
        x, s, y, z, tau, _ = self.unscale(u, nu)
        if status == PRIMAL_INFEASIBLE:
            bty = float(self.V.b @ y)
            return y / bty, (self.V.H.T @ z) / bty
        if status == DUAL_INFEASIBLE:
            ctx = float(self.V.c @ x)
            return x / (-ctx), s / (-ctx)
        raise ValueError("no certificate for this status")
