"""GPU: the numerical-failure paths, provoked from the host.

* A NaN planted in the loaded state (hsde_set_state) must end that instance
  with HSDE_NUMERICAL_ERROR after one iteration, and leave the other
  instances of the same batch running exactly as they would alone.
* An eigensolve that runs out of sweeps is counted (hsde_info's
  jacobi_unconverged), not hidden: one sweep from a cold start is not enough
  for the 33-wide cliques of the block-arrow below; the default sweep limit is.
Nothing here faults the GPU: NaN arithmetic is ordinary arithmetic and every
loop of the kernels is bounded.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_01828_gb300 import hsde
    return hsde


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("part", ["s", "x", "y"])
def test_nan_in_the_state_gives_numerical_error(hs, prec, part):
    probs = [synth.block_arrow_n50(), synth.maxcut_grid(7, 9, np.random.default_rng(1))]
    with hs.Handle(probs[1], precision=prec) as H1:
        H1.hsde_iterate(8)
        alone = H1.hsde_get_state(0)
    with hs.Handle(probs, precision=prec) as H:
        H.hsde_iterate(3)
        sz = H.sizes[0]
        st = H.hsde_get_state(0)
        pos = {"x": 0, "s": sz.N, "y": sz.N + sz.P}[part]
        st[pos + 1] = np.nan
        H.hsde_set_state(0, st, 3)
        status = H.hsde_iterate(1)
        assert int(status[0]) == hs.NUMERICAL_ERROR
        assert int(status[1]) == hs.RUNNING
        assert H.hsde_get_info(0)["status"] == hs.NUMERICAL_ERROR
        H.hsde_iterate(4)
        assert np.array_equal(H.hsde_get_state(1), alone)
        assert int(H.hsde_iterate(1)[0]) == hs.NUMERICAL_ERROR   # it stays frozen


def test_unconverged_eigensolves_are_counted(hs):
    p = synth.block_arrow(3, 30, 3, 6, np.random.default_rng(3))        # cliques of 33
    with hs.Handle(p, precision="fp64", warm_start=0, jacobi_max_sweeps=1) as H:
        H.hsde_iterate(3)
        info = H.hsde_get_info(0)
    assert info["jacobi_unconverged"] == 3
    assert info["jacobi_unconverged_iterations"] == 3
    for prec in ("fp64", "mixed"):
        with hs.Handle(p, precision=prec) as H:
            H.hsde_iterate(20)
            info = H.hsde_get_info(0)
        assert info["jacobi_unconverged"] == 0 and info["jacobi_unconverged_iterations"] == 0, prec
