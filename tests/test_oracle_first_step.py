"""The first affine step from the standard start, a closed form of
Eq. MatrixInverseResult, and the rounding bound it sets.

From u0 = (0,0,0,0,1), nu0 = (0,0,0,0,1) (reading P4), omega = u0 + nu0 has
only omega_tau = 2, so omega_hat = -2 zeta, w = M^{-1} omega_hat = -2 M^{-1} zeta
and the Sherman-Morrison correction gives exactly

    u_hat_{1,2} = w - M^{-1}zeta (zeta^T w) / den = -2 M^{-1} zeta / den,
    den = 1 + zeta^T M^{-1} zeta.

The formula reaches this as the difference of two vectors about den times
larger than the result, so FP64 rounding leaves a relative error of order
eps * den: the bound every FP64 evaluation of the printed formula (this
oracle's and the GPU's alike) is held to on the first iterations.  den grows
with the unscaled data: ~1e7 for l = 100, ~1e9 for l = 500, ~1e11 for
l = 2000 on the block-arrow sweep.  The data scaling of reading P7 brings
||zeta|| to the scaling's target norm, and with it den to O(100): the same
closed form then holds to near machine precision.
"""
import numpy as np
import pytest

import synth
from oracle import hsde as ohsde

EPS = np.finfo(np.float64).eps


@pytest.mark.parametrize("l,d", [(20, 4), (100, 10), (500, 10)])
def test_first_step_is_minus_two_Minv_zeta_over_den(l, d):
    r = ohsde.HSDE(synth.block_arrow_sweep(l, d), alpha=1.0, scaling=False)
    u, nu = r.initial()
    uh = r.affine(u + nu)
    n = len(r.Minv_zeta)
    closed = -2.0 * r.Minv_zeta / r.den
    err = np.linalg.norm(uh[:n] - closed) / np.linalg.norm(closed)
    # within the cancellation bound, and well below it is impossible to ask
    assert err <= 10.0 * EPS * r.den, (err, r.den)
    # the tau row: tau_hat = omega_tau + c^T x_hat - b^T y_hat
    assert np.isfinite(uh[-1])


def test_first_step_closed_form_on_a_well_scaled_instance():
    # the n = 50 block-arrow has den small enough that the closed form holds
    # to near machine precision, which a dropped or mis-signed term of
    # Eq. MatrixInverseResult would break
    r = ohsde.HSDE(synth.block_arrow_n50(), alpha=1.0, scaling=False)
    u, nu = r.initial()
    uh = r.affine(u + nu)
    n = len(r.Minv_zeta)
    closed = -2.0 * r.Minv_zeta / r.den
    assert np.linalg.norm(uh[:n] - closed) / np.linalg.norm(closed) < max(1e-12, 10.0 * EPS * r.den)


@pytest.mark.parametrize("l,d", [(100, 10), (500, 10)])
def test_scaling_removes_the_cancellation(l, d):
    """With the data scaling of reading P7 den is O(100) and the first step
    meets the closed form to ~1e-13, where the unscaled data lose log10(den)
    digits."""
    r = ohsde.HSDE(synth.block_arrow_sweep(l, d))
    assert r.den < 1e3
    u, nu = r.initial()
    uh = r.affine(u + nu)
    n = len(r.Minv_zeta)
    closed = -2.0 * r.Minv_zeta / r.den
    assert np.linalg.norm(uh[:n] - closed) / np.linalg.norm(closed) < 1e-12
