"""CPU: bit-exact symbolic analysis of the library (host C++) against the
oracle on a sample of the 256-instance batch (uneven sizes, both families,
infeasible variants)."""
import numpy as np
import pytest

import synth
from oracle import symbolic


@pytest.fixture(scope="module")
def hs():
    import os
    from paper_1611_01828_gb300 import _build
    if not os.path.exists(os.path.join(os.path.dirname(_build.__file__), "libhsde.so")):
        _build.build()
    from paper_1611_01828_gb300 import hsde
    return hsde


@pytest.mark.parametrize("i", [0, 1, 37, 64, 101, 128, 199, 255])
def test_serving_batch_instance_structure_bit_exact(hs, i):
    p = synth.serving_batch(select=[i])[0]
    got = hs.hsde_analyze(p)
    st = symbolic.analyze(p)
    for k in ("order", "clique_ptr", "clique_idx", "pat_colptr", "pat_row", "gather", "D"):
        assert np.array_equal(got[k], getattr(st, k)), k
