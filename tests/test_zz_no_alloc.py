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


def _cudart():
    """The CUDA runtime library, to read the device's default memory pool
    (the pool cudaMallocAsync draws from); None if it cannot be found."""
    import glob
    import os
    cands = []
    try:
        import torch
        cands += glob.glob(os.path.join(os.path.dirname(torch.__file__), "lib", "libcudart.so*"))
    except Exception:
        pass
    cands += glob.glob("/usr/local/cuda/lib64/libcudart.so*") + ["libcudart.so"]
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


USED_MEM_HIGH = 8   # cudaMemPoolAttrUsedMemHigh


def test_noalloc_allocates_nothing(env):
    """The call itself must not allocate device memory: torch's allocator
    statistics and the default memory pool's high-water mark of used memory
    are unchanged across a call.  The allocating entry point is the control:
    the same probe sees its 2m-double scratch."""
    torch, hsde = env
    m = 2000
    stream = torch.cuda.current_stream().cuda_stream
    a = torch.from_numpy(_spd(m, 21)).cuda()
    b = a.clone()
    assert hsde.lib.hsde_spd_inverse_noalloc(ctypes.c_void_p(b.data_ptr()), m, ctypes.c_void_p(stream)) == 0
    torch.cuda.synchronize()                       # warm-up: the one-time symbol lookup
    rt = _cudart()
    pool = ctypes.c_void_p()
    have_pool = rt is not None and rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0

    def high_mark(call):
        if have_pool:
            zero = ctypes.c_uint64(0)
            assert rt.cudaMemPoolSetAttribute(pool, USED_MEM_HIGH, ctypes.byref(zero)) == 0
        alloc0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        assert call() == 0
        torch.cuda.synchronize()
        assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == alloc0
        if not have_pool:
            return None
        v = ctypes.c_uint64(0)
        assert rt.cudaMemPoolGetAttribute(pool, USED_MEM_HIGH, ctypes.byref(v)) == 0
        return v.value

    control = high_mark(lambda: hsde.lib.hsde_spd_inverse(ctypes.c_void_p(a.data_ptr()), m, ctypes.c_void_p(stream)))
    got = high_mark(lambda: hsde.lib.hsde_spd_inverse_noalloc(ctypes.c_void_p(b.data_ptr()), m,
                                                              ctypes.c_void_p(stream)))
    if have_pool:
        assert control >= 2 * m * 8          # the probe sees the allocating variant's scratch
        assert got == 0
