"""Literal dense embedding matrix Q (test infrastructure).

Builds Q of Section 3.2 (Eq. HomogeneousEmbedding) as a dense array for tiny
instances and solves (I + Q) u_hat = omega with a plain LU solve, to pin the
block-eliminated affine step of Sections 4.2-4.3 and the reading of the
garbled second elimination.
"""
from __future__ import annotations

import numpy as np


def build_Q(hs):
    """Q = [[0,0,-A^T,-H^T,c],[0,0,0,I,0],[A,0,0,0,-b],[H,-I,0,0,0],[-c^T,0,b^T,0,0]]
    in the variable order u = (x, s, y, v, tau), with the data the iteration
    uses (hs.A, hs.b, hs.c: scaled when the oracle scales, reading P7)."""
    A = hs.A.toarray()
    H = hs.V.H.toarray()
    nF, nd, m = hs.nF, hs.nd, hs.m
    ix = slice(0, nF)
    is_ = slice(nF, nF + nd)
    iy = slice(nF + nd, nF + nd + m)
    iv = slice(nF + nd + m, nF + 2 * nd + m)
    it = nF + 2 * nd + m
    Q = np.zeros((hs.dim, hs.dim))
    Q[ix, iy] = -A.T
    Q[ix, iv] = -H.T
    Q[ix, it] = hs.c
    Q[is_, iv] = np.eye(nd)
    Q[iy, ix] = A
    Q[iy, it] = -hs.b
    Q[iv, ix] = H
    Q[iv, is_] = -np.eye(nd)
    Q[it, ix] = -hs.c
    Q[it, iy] = hs.b
    return Q


def affine_dense(hs, omega, Q=None):
    Q = build_Q(hs) if Q is None else Q
    return np.linalg.solve(np.eye(Q.shape[0]) + Q, omega)


def step_dense(hs, u, nu, Q):
    uhat = affine_dense(hs, u + nu, Q)
    urel = hs.alpha * uhat + (1.0 - hs.alpha) * u
    u_new = hs.project_K(urel - nu)
    return u_new, nu - urel + u_new, uhat
