"""GPU: gradient of f(C, b) = c^T x_K / (tau_K + kappa_K) after K unrolled
ADMM iterations through the library's reverse sweep.

* FP64 against the oracle's reverse mode (itself pinned by central
  differences): relative 1e-6.
* The max-cut n = 1000 workload (open 10 x 100 grid), K = 200, checkpoint
  every 20: against the oracle's reverse mode, relative 1e-6; and central
  differences of the GPU forward (step 1e-6, FP64) on 20 random directions
  in (C, b): median relative error 5e-3, maximum 5e-2.  The looser difference
  bounds are a property of the map, not of the gradient: 200 iterations
  through near-zero eigenvalues and the tau kink make it rough at that scale,
  and the oracle's own central differences move by ~1e-3 between steps 1e-5,
  1e-6 and 1e-7 while its analytic gradient agrees with this one to ~1e-9.
* Mixed precision (FP32 projections) against FP64 on the same instance:
  relative 2e-2 of the gradient norm.
"""
import numpy as np
import pytest

import synth
from oracle import adjoint, hsde as ohsde

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_01828_gb300 import hsde, unrolled
    return torch, hsde, unrolled


def _on_pattern(p, st):
    """Give C an explicit (possibly zero) entry on every pattern position."""
    pos = {(r, c): e for e, (r, c) in enumerate(zip(p.C_row.tolist(), p.C_col.tolist()))}
    vals = np.zeros(st.N)
    for e, (r, c) in enumerate(zip(st.pat_row.tolist(), st.pat_col.tolist())):
        if (r, c) in pos:
            vals[e] = p.C_val[pos[(r, c)]]
    q = synth.Problem(**{**p.__dict__})
    q.C_row, q.C_col, q.C_val = st.pat_row.copy(), st.pat_col.copy(), vals
    return q


def _grad(torch, hsde, unrolled, H, c, b, K, ckpt):
    ct = torch.tensor(c, dtype=torch.float64, requires_grad=True)
    bt = torch.tensor(b, dtype=torch.float64, requires_grad=True)
    f = unrolled.unrolled_objective(ct, bt, H, K, ckpt)
    f.backward()
    return float(f), ct.grad.numpy().copy(), bt.grad.numpy().copy()


@pytest.mark.parametrize("case", ["grid", "arrow", "arrow_n50"])
def test_fp64_gradient_matches_oracle(env, case):
    torch, hsde, unrolled = env
    if case == "grid":
        p0, K = synth.maxcut_grid(3, 5, np.random.default_rng(1)), 40
    elif case == "arrow":
        p0, K = synth.block_arrow(3, 3, 2, 5, np.random.default_rng(2), kappa=30.0, assign="roundrobin"), 30
    else:
        p0, K = synth.block_arrow_n50(), 25
    st = ohsde.HSDE(p0, alpha=1.0, scaling=False).V.st
    p = _on_pattern(p0, st)
    ref = ohsde.HSDE(p, alpha=1.0, scaling=False)
    f_r, cbar, bbar = adjoint.gradient(ref, K)
    w = np.where(st.pat_row == st.pat_col, 1.0, 2.0)
    gC_ref = w * adjoint.grad_C_lower(ref, cbar)
    with hsde.Handle(p, precision="fp64", **unrolled.LITERAL) as H:
        f, gC, gb = _grad(torch, hsde, unrolled, H, p.C_val, p.b, K, 7)
    assert f == pytest.approx(f_r, rel=1e-7)        # FP64 forward parity (rounding order)
    assert np.linalg.norm(gC - gC_ref) <= 1e-6 * np.linalg.norm(gC_ref)
    assert np.linalg.norm(gb - bbar) <= 1e-6 * max(1e-12, np.linalg.norm(bbar))


@pytest.fixture(scope="module")
def diff_grid(env):
    torch, hsde, unrolled = env
    p = synth.differentiation_maxcut_grid()
    H = hsde.Handle(p, precision="fp64", **unrolled.LITERAL)
    c0 = unrolled.pattern_values(H, p.C_row, p.C_col, p.C_val)
    yield p, H, c0
    H.close()


def test_diff_grid_gradient_central_differences(env, diff_grid):
    torch, hsde, unrolled = env
    p, H, c0 = diff_grid
    K, ckpt = 200, 20
    f0, gC, gb = _grad(torch, hsde, unrolled, H, c0, p.b, K, ckpt)
    w = torch.as_tensor(unrolled.pattern_weights(H))
    rng = np.random.default_rng(44)

    def fval(c, b):
        with torch.no_grad():
            return float(unrolled.unrolled_objective(torch.tensor(c), torch.tensor(b), H, K, ckpt, weights=w))

    h = 1e-6
    errs = []
    for _ in range(20):
        dC = rng.standard_normal(c0.shape[0])
        db = rng.standard_normal(p.m)
        fd = (fval(c0 + h * dC, p.b + h * db) - fval(c0 - h * dC, p.b - h * db)) / (2 * h)
        an = float(gC @ dC + gb @ db)
        errs.append(abs(fd - an) / max(abs(fd), 1e-12))
    errs = np.array(errs)
    print("max-cut 10x100 central-difference relative errors:", np.array2string(errs, precision=2))
    assert np.median(errs) <= 5e-3 and errs.max() <= 5e-2, errs


def test_diff_grid_gradient_matches_oracle(env, diff_grid):
    torch, hsde, unrolled = env
    p, H, c0 = diff_grid
    K, ckpt = 200, 20
    _, gC, gb = _grad(torch, hsde, unrolled, H, c0, p.b, K, ckpt)
    st = ohsde.HSDE(p, alpha=1.0, scaling=False).V.st
    q = _on_pattern(p, st)
    ref = ohsde.HSDE(q, alpha=1.0, scaling=False)
    f_r, cbar, bbar = adjoint.gradient(ref, K)
    w = np.where(st.pat_row == st.pat_col, 1.0, 2.0)
    gC_ref = w * adjoint.grad_C_lower(ref, cbar)
    assert np.linalg.norm(gC - gC_ref) <= 1e-6 * np.linalg.norm(gC_ref)
    assert np.linalg.norm(gb - bbar) <= 1e-6 * np.linalg.norm(bbar)


def test_diff_grid_mixed_gradient_close_to_fp64(env, diff_grid):
    torch, hsde, unrolled = env
    p, H, c0 = diff_grid
    K, ckpt = 200, 20
    _, gC64, gb64 = _grad(torch, hsde, unrolled, H, c0, p.b, K, ckpt)
    with hsde.Handle(p, precision="mixed", **unrolled.LITERAL) as Hm:
        _, gC32, gb32 = _grad(torch, hsde, unrolled, Hm, c0, p.b, K, ckpt)
    g64 = np.concatenate([gC64, gb64]); g32 = np.concatenate([gC32, gb32])
    assert np.linalg.norm(g32 - g64) <= 2e-2 * np.linalg.norm(g64)


def test_device_tensors_match_host_path(env, diff_grid):
    """CUDA tensors go to the library as device addresses; the C-ABI results
    are bitwise those of host arrays, and the autograd gradient agrees up to
    the order of the objective's sum."""
    torch, hsde, unrolled = env
    p, H, c0 = diff_grid
    K, ckpt = 60, 20
    H.hsde_set_data(0, c0, p.b)
    xh, yh, th, kh = H.hsde_unrolled_forward(K, ckpt)
    rng = np.random.default_rng(5)
    xb, yb = rng.standard_normal(xh.shape[0]), rng.standard_normal(yh.shape[0])
    gCh, gbh = H.hsde_unrolled_backward(xb, yb, 0.3, -0.7)

    dev = torch.device("cuda")
    cd = torch.tensor(c0, device=dev); bd = torch.tensor(p.b, device=dev)
    xd = torch.empty(xh.shape[0], dtype=torch.float64, device=dev)
    yd = torch.empty(yh.shape[0], dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    H.hsde_set_data(0, cd.data_ptr(), bd.data_ptr())
    _, _, td, kd = H.hsde_unrolled_forward(K, ckpt, x=xd.data_ptr(), y=yd.data_ptr())
    assert (td, kd) == (th, kh)
    assert np.array_equal(xd.cpu().numpy(), xh) and np.array_equal(yd.cpu().numpy(), yh)
    xbd, ybd = torch.tensor(xb, device=dev), torch.tensor(yb, device=dev)
    gCd = torch.empty_like(xd); gbd = torch.empty_like(yd)
    torch.cuda.synchronize()
    H.hsde_unrolled_backward(xbd.data_ptr(), ybd.data_ptr(), 0.3, -0.7, gC=gCd.data_ptr(), gb=gbd.data_ptr())
    assert np.array_equal(gCd.cpu().numpy(), gCh) and np.array_equal(gbd.cpu().numpy(), gbh)

    f_h, gC_h, gb_h = _grad(torch, hsde, unrolled, H, c0, p.b, K, ckpt)
    ct = torch.tensor(c0, device=dev, requires_grad=True)
    bt = torch.tensor(p.b, device=dev, requires_grad=True)
    f = unrolled.unrolled_objective(ct, bt, H, K, ckpt)
    f.backward()
    assert ct.grad.is_cuda and bt.grad.is_cuda
    assert float(f) == pytest.approx(f_h, rel=1e-12)
    assert np.linalg.norm(ct.grad.cpu().numpy() - gC_h) <= 1e-10 * np.linalg.norm(gC_h)
    assert np.linalg.norm(bt.grad.cpu().numpy() - gb_h) <= 1e-10 * np.linalg.norm(gb_h)


def test_set_data_from_device_memory_on_a_scaled_handle(env):
    """New data from device memory: the scaling sums are formed by kernels
    (another summation order), so the iterate after 30 iterations agrees
    with the host path's to rounding; a mix of host and device pointers is
    refused on the host."""
    torch, hsde, unrolled = env
    p = synth.maxcut_grid(4, 6, np.random.default_rng(3))
    rng = np.random.default_rng(8)
    with hsde.Handle(p, precision="fp64") as H:
        c1 = unrolled.pattern_values(H, p.C_row, p.C_col, p.C_val * (1.0 + 0.1 * rng.standard_normal(p.C_val.shape[0])))
        b1 = p.b * 1.3
        s0 = H.hsde_get_state(0)
        H.hsde_set_data(0, c1, b1)
        H.hsde_iterate(30)
        sh = H.hsde_get_state(0)
        H.hsde_set_state(0, s0)
        cd = torch.tensor(c1, device="cuda"); bd = torch.tensor(b1, device="cuda")
        torch.cuda.synchronize()
        H.hsde_set_data(0, cd.data_ptr(), bd.data_ptr())
        H.hsde_iterate(30)
        sd = H.hsde_get_state(0)
        assert np.max(np.abs(sd - sh)) <= 1e-10 * (1.0 + np.max(np.abs(sh)))
        with pytest.raises(hsde.HSDEError):
            H.hsde_set_data(0, cd.data_ptr(), b1)
