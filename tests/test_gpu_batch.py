"""GPU: batched serving of independent SDPs of uneven sizes in the same
launches (the config-3 generator), against the FP64 oracle per instance.

Tolerances: identical verdicts; SOLVED objectives within 1e-4 (1 + |obj|);
iteration counts within 10% (mixed precision changes the trajectory a little).
"""
import numpy as np
import pytest

import synth
from oracle import hsde as ohsde

pytestmark = pytest.mark.gpu

SEL = [2, 5, 6, 7, 11, 13]     # grids, block-arrows, one dual- and one primal-infeasible


@pytest.fixture(scope="module")
def hs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_01828_gb300 import hsde
    return hsde


@pytest.fixture(scope="module")
def batch():
    probs = synth.config3(B=16, n_lo=60, n_hi=160, select=SEL)
    refs = [ohsde.HSDE(p).solve(max_iter=3000) for p in probs]
    return probs, refs


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batched_verdicts_and_objectives(hs, batch, prec):
    probs, refs = batch
    kinds = {p.kind for p in probs}
    assert {"feasible", "primal_infeasible", "dual_infeasible"} <= kinds
    with hs.Handle(probs, precision=prec, max_iter=3000) as H:
        st = H.solve(chunk=100)
        infos = [H.hsde_get_info(i) for i in range(len(probs))]
    for p, r, s, inf in zip(probs, refs, st, infos):
        assert int(s) == r.status, (p.name, int(s), r.status)
        assert abs(inf["iterations"] - r.iterations) <= max(3, 0.1 * r.iterations), p.name
        if r.status == ohsde.SOLVED:
            assert abs(inf["pobj"] - r.info["pobj"]) <= 1e-4 * (1 + abs(r.info["pobj"])), p.name


def test_frozen_instances_do_not_move(hs, batch):
    """An instance that reached its verdict keeps its state while the rest iterate."""
    probs, refs = batch
    with hs.Handle(probs, precision="mixed", max_iter=3000) as H:
        st = H.solve(chunk=50)
        done = [H.hsde_get_state(i) for i in range(len(probs))]
        H.hsde_iterate(20)
        for i in range(len(probs)):
            assert np.array_equal(H.hsde_get_state(i), done[i])
