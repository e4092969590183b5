"""Element-by-element comparison of a library state with the oracle's.

A state is [x (N) | s (P) | y (m) | v (P) | tau | z (P) | kappa] (the layout
of include/hsde.h).  Each part is compared on its own, so that a wrong
scalar, a wrong constraint-space vector or one wrong clique block cannot hide
under the norm of the whole state:

* x and y: max |got - want| / (1 + max |want|) over the vector;
* s, v and z: the same measure per clique block; the worst block is named;
* tau and kappa: |got - want| / (1 + |want|), or against a caller-given
  scale: tau_hat = omega_tau + c~^T x_hat - b~^T y_hat is formed from inner
  products that can be many times tau itself, and its rounding is relative
  to them (scalar_scale = 1 + |c~^T x| + |b~^T y| of the reference state).

The failure message names the component and, for the clique parts, the
block (clique index and size).
"""
from __future__ import annotations

import numpy as np


def split(state, N, P, m):
    o = 0
    out = {}
    for name, ln in (("x", N), ("s", P), ("y", m), ("v", P), ("tau", 1), ("z", P), ("kappa", 1)):
        out[name] = np.asarray(state[o:o + ln], dtype=np.float64)
        o += ln
    return out


def _vec_err(g, w):
    if g.size == 0:
        return 0.0
    return float(np.max(np.abs(g - w)) / (1.0 + np.max(np.abs(w))))


def component_errors(got, want, N, P, m, packed_ptr, scalar_scale=None):
    """{component: (error, where)} for every part of the state."""
    g, w = split(got, N, P, m), split(want, N, P, m)
    out = {}
    for k in ("x", "y"):
        out[k] = (_vec_err(g[k], w[k]), "")
    for k in ("tau", "kappa"):
        sc = 1.0 + abs(w[k][0]) if scalar_scale is None else max(1.0 + abs(w[k][0]), scalar_scale)
        out[k] = (float(abs(g[k][0] - w[k][0]) / sc), "")
    pp = np.asarray(packed_ptr)
    for k in ("s", "v", "z"):
        worst, where = 0.0, ""
        for b in range(len(pp) - 1):
            e = _vec_err(g[k][pp[b]:pp[b + 1]], w[k][pp[b]:pp[b + 1]])
            if e > worst:
                size = int(round((np.sqrt(8 * (pp[b + 1] - pp[b]) + 1) - 1) / 2))
                worst, where = e, f"clique {b} (size {size})"
        out[k] = (worst, where)
    return out


def assert_state_close(got, want, N, P, m, packed_ptr, tol, label="", scalar_scale=None):
    errs = component_errors(got, want, N, P, m, packed_ptr, scalar_scale)
    bad = {k: v for k, v in errs.items() if not v[0] <= tol}
    summary = ", ".join(f"{k} {v[0]:.2e}{(' at ' + v[1]) if v[1] else ''}" for k, v in errs.items())
    assert not bad, f"{label} state differs beyond {tol:.1e}: " + "; ".join(
        f"{k}: {v[0]:.3e}{(' at ' + v[1]) if v[1] else ''}" for k, v in bad.items()) + f"  [all: {summary}]"
    return errs
