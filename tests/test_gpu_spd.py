"""GPU: the standalone SPD inverse (Gauss-Jordan, the cached factor of
Sections 4.2-4.3) against numpy.linalg.inv, FP64, relative 1e-10."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_01828_gb300 import hsde
    return torch, hsde


def spd(m, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((m, m))
    return np.eye(m) + G @ G.T / m


@pytest.mark.parametrize("m", [1, 2, 7, 64, 300, 1000])
def test_spd_inverse_matches_numpy(env, m):
    torch, hsde = env
    S = spd(m, m)
    d = torch.from_numpy(S.copy()).cuda()
    s = torch.cuda.current_stream()
    hsde.hsde_spd_inverse(d.data_ptr(), m, s.cuda_stream)
    torch.cuda.synchronize()
    got = d.cpu().numpy()
    want = np.linalg.inv(S)
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)


def test_spd_inverse_rejects_bad_args(env):
    torch, hsde = env
    with pytest.raises(hsde.HSDEError) as ei:
        hsde.hsde_spd_inverse(0, 4, 0)
    assert ei.value.code == hsde.HSDE_EINVAL
