"""Reverse-mode derivative of K unrolled ADMM iterations (test infrastructure).

The objective after K iterations from the standard start (reading P4) is
    f(C, b) = c^T x_K / (tau_K + kappa_K)
with c = vec(C) (Section 3.1).  It equals the primal objective c^T x_K/tau_K
once kappa_K = 0 and stays defined while the unscaled iteration still has
tau_K = 0 (the first few hundred iterations on max-cut grids).  The reverse
pass itself takes any upstream gradient on (x_K, y_K, tau_K, kappa_K).  Its gradient with respect to C (a symmetric
matrix on the chordal pattern, df = <G_C, dC>_F) and b is computed here by
plain reverse mode through the three steps of Section 4.1 (Eqs. Step1-Step3)
on the embedding of Section 3.2 (Eq. HomogeneousEmbedding):

* Eq. Step1, u_hat = (I + Q)^{-1} omega: since Q is skew-symmetric the
  adjoint is omega_bar = (I - Q)^{-1} u_hat_bar, solved here with a sparse LU
  of the literal I - Q; Q depends on (c, b), which contributes
  c_bar += -(omega_bar_x tau_hat - omega_bar_tau x_hat) and
  b_bar += omega_bar_y tau_hat - omega_bar_tau y_hat.
* Eq. Step2, the projection on K: identity on the free parts, the step
  function on tau, and on each clique block the Frechet derivative of the
  psd projection (Daleckii-Krein): for A = V diag(l) V^T,
      dPi[G] = V (Gamma o (V^T G V)) V^T,
      Gamma_ij = (max(l_i,0) - max(l_j,0)) / (l_i - l_j)  (l_i != l_j),
      Gamma_ij = 1, 1/2, 0 for l_i == l_j > 0, = 0, < 0,
  which is self-adjoint, so the same formula gives the vector-Jacobian
  product.  At an eigenvalue exactly 0 the projection is not differentiable;
  1/2 is the value a central difference sees (by Moreau, Pi(tM) - Pi(-tM) =
  tM), and exactly-zero eigenvalues do occur in the first iteration from the
  standard start.  Eigenvalues below 1e-10 of the block's largest one are
  taken as exactly zero, so that rounding in the eigensolver does not pick
  the derivative.  This derivative is not in the paper; it is textbook matrix
  analysis.
* Eq. Step3, nu = nu - u_hat + u: linear.

The free-cone parts h, r, w of nu are identically zero (Eq. Step3 resets
them every iteration whatever the inputs), so they carry no derivative.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import dense, hsde


ZERO_REL = 1e-10   # eigenvalues below this fraction of the block's largest are taken as 0


def _dk_gamma(lam):
    scale = np.abs(lam).max() if lam.size else 0.0
    lam = np.where(np.abs(lam) <= ZERO_REL * scale, 0.0, lam)
    lp = np.maximum(lam, 0.0)
    dl = lam[:, None] - lam[None, :]
    dp = lp[:, None] - lp[None, :]
    same = np.abs(dl) <= 1e-300
    with np.errstate(divide="ignore", invalid="ignore"):
        G = np.where(same, 0.0, dp / np.where(same, 1.0, dl))
    # coinciding eigenvalues: derivative of max(l, 0), 1/2 exactly at 0
    step = np.where(lam > 0, 1.0, np.where(lam < 0, 0.0, 0.5))
    return np.where(same, step[:, None] * np.ones_like(G), G)


def dk_vjp(A, Gbar):
    """Vector-Jacobian product of the psd projection at symmetric A."""
    A = 0.5 * (A + A.T)
    lam, V = np.linalg.eigh(A)
    B = V.T @ (0.5 * (Gbar + Gbar.T)) @ V
    return V @ (_dk_gamma(lam) * B) @ V.T


def _check_literal(hs):
    # the derivative is taken through the literal Eqs. Step1-Step3 on the
    # original data: no relaxation, no scaling (whose factors depend on b, c)
    if hs.alpha != 1.0 or hs.scaled:
        raise ValueError("reverse mode needs HSDE(..., alpha=1, scaling=False)")


def sparse_Q(hs):
    _check_literal(hs)
    V = hs.V
    A, H = V.A, V.H
    nF, nd, m = hs.nF, hs.nd, hs.m
    c = sp.csr_matrix(V.c.reshape(-1, 1))
    b = sp.csr_matrix(V.b.reshape(-1, 1))
    I = sp.identity(nd, format="csr")
    Z = None
    return sp.bmat([
        [Z, Z, -A.T, -H.T, c],
        [Z, Z, Z, I, Z],
        [A, Z, Z, Z, -b],
        [H, -I, Z, Z, Z],
        [-c.T, Z, b.T, Z, None],
    ], format="csc", dtype=float) if m > 0 else None


def objective(hs, K):
    _check_literal(hs)
    u, nu = hs.initial()
    for _ in range(K):
        u, nu, _ = hs.step(u, nu)
    x, s, y, v, tau = hs.split(u)
    return float(hs.V.c @ x) / (tau + float(nu[-1]))


def gradient(hs, K, seed=None):
    """Reverse mode through K iterations.

    Without `seed`: f = c^T x_K/(tau_K + kappa_K) and its gradient
    (f, cbar over full-vec entries (both triangles), bbar).
    With `seed = (xbar, ybar, taubar, kappabar)`: the gradient of
    <xbar, x_K> + <ybar, y_K> + taubar tau_K + kappabar kappa_K instead
    (f returned as that value)."""
    _check_literal(hs)
    nF, nd, m = hs.nF, hs.nd, hs.m
    dim = hs.dim
    Q = sparse_Q(hs)
    # literal Q built from the same blocks as oracle.dense (checked by the tests)
    ImQ = spla.splu((sp.identity(dim, format="csc") - Q).tocsc())
    # ---- forward, keeping what the reverse pass needs ----
    u, nu = hs.initial()
    tape = []
    for _ in range(K):
        uhat = hs.affine(u + nu)
        w = uhat - nu
        u_new = hs.project_K(w)
        tape.append((uhat, w))
        nu = nu - uhat + u_new
        u = u_new
    x, s, y, v, tau = hs.split(u)
    kappa = float(nu[-1])
    c = hs.V.c
    ubar = np.zeros(dim)
    nubar = np.zeros(dim)
    if seed is None:
        den = tau + kappa
        f = float(c @ x) / den
        ubar[:nF] = c / den
        ubar[-1] = -f / den
        nubar[-1] = -f / den
        cbar = x / den
    else:
        xb, yb, tb, kb = seed
        f = float(xb @ x + yb @ y + tb * tau + kb * kappa)
        ubar[:nF] = xb
        ubar[nF + nd:nF + nd + m] = yb
        ubar[-1] = tb
        nubar[-1] = kb
        cbar = np.zeros(nF)
    bbar = np.zeros(m)
    ix = slice(0, nF)
    is_ = slice(nF, nF + nd)
    iy = slice(nF + nd, nF + nd + m)
    for k in range(K - 1, -1, -1):
        uhat, w = tape[k]
        # nu' = nu - uhat + u'
        ubar_tot = ubar + nubar
        uhat_bar = -nubar.copy()
        nubar_prev = nubar.copy()
        # u' = Pi_K(w), w = uhat - nu
        wbar = ubar_tot.copy()
        sbar = ubar_tot[is_]
        wbar_s = np.zeros(nd)
        for kk, cs in enumerate(hs.cl_sizes):
            o = hs.V.s_off[kk]
            Ak = w[nF + o:nF + o + cs * cs].reshape((cs, cs), order="F")
            Gk = sbar[o:o + cs * cs].reshape((cs, cs), order="F")
            wbar_s[o:o + cs * cs] = dk_vjp(Ak, Gk).reshape(-1, order="F")
        wbar[is_] = wbar_s
        wbar[-1] = ubar_tot[-1] if w[-1] > 0 else 0.0
        uhat_bar += wbar
        nubar_prev -= wbar
        # uhat = (I+Q)^{-1} omega, omega = u + nu  ->  omega_bar = (I-Q)^{-1} uhat_bar
        obar = ImQ.solve(uhat_bar)
        xh, yh, th = uhat[ix], uhat[iy], float(uhat[-1])
        cbar += -(obar[ix] * th - obar[-1] * xh)
        bbar += obar[iy] * th - obar[-1] * yh
        ubar = obar.copy()
        nubar = nubar_prev + obar
        # h, r, w of nu are identically zero: no derivative flows into them
        nubar[ix] = 0.0
        nubar[iy] = 0.0
        nubar[nF + nd + m:nF + 2 * nd + m] = 0.0
    return f, cbar, bbar


def grad_C_lower(hs, cbar):
    """Symmetric-matrix gradient on the pattern (lower CSC order): the entry
    (i,j) collects both vec positions (i,j) and (j,i) as a matrix gradient
    G with df = <G, dC>_F, i.e. G_ij = (cbar_(i,j) + cbar_(j,i)) / 2."""
    V = hs.V
    st = V.st
    out = np.zeros(st.N)
    for e, (r, c) in enumerate(zip(st.pat_row.tolist(), st.pat_col.tolist())):
        out[e] = 0.5 * (cbar[V.fpos[(r, c)]] + cbar[V.fpos[(c, r)]])
    return out
