"""GPU: the allocation-free SPD inverse.

hsde_spd_inverse_noalloc serves callers that cannot allocate device memory
while they call it (graph capture under an allocator-restricted framework,
fixed-budget real-time hosts, pooled allocators).  It must give the same
inverse as the allocating hsde_spd_inverse, call after call, while reusing
its one static scratch array.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12   # same kernels, same order: the two results agree to rounding


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_01828_gb300 import hsde
    return torch, hsde


def _spd(m, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((m, m))
    return np.eye(m) + G @ G.T / m


def test_noalloc_matches_allocating_inverse_on_two_calls_in_a_row(env):
    torch, hsde = env
    stream = torch.cuda.current_stream().cuda_stream
    for m, seed in ((300, 11), (1000, 12)):
        S = _spd(m, seed)
        a = torch.from_numpy(S.copy()).cuda()
        b = a.clone()
        assert hsde.lib.hsde_spd_inverse(ctypes.c_void_p(a.data_ptr()), m, ctypes.c_void_p(stream)) == 0
        assert hsde.lib.hsde_spd_inverse_noalloc(ctypes.c_void_p(b.data_ptr()), m, ctypes.c_void_p(stream)) == 0
        torch.cuda.synchronize()
        want, got = a.cpu().numpy(), b.cpu().numpy()
        assert np.linalg.norm(got - want) <= TOL * np.linalg.norm(want)
        assert np.linalg.norm(got @ S - np.eye(m)) <= 1e-9 * m


def test_noalloc_rejects_sizes_beyond_its_limit(env):
    torch, hsde = env
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = hsde.lib.hsde_spd_inverse_noalloc(ctypes.c_void_p(t.data_ptr()), 8193, ctypes.c_void_p(0))
    assert rc == hsde.HSDE_ERANGE
    assert b"8192" in hsde.lib.hsde_last_error()
