"""GPU parity of the tridiagonal QR eigensolver path (cliques above the Jacobi
bucket sizes: 112 in the mixed form, 80 in FP64; up to 1024), against the
FP64 oracle, element by element (tests/parity_util).

The path (Eq. Step2 on the large clique cones of Table 1's qpG-type rows):
Householder tridiagonalisation, implicit QR with the Wilkinson shift, and the
rebuild s = Q max(Lambda, 0) Q^T, by split-precision TF32 tensor-core
products in the mixed form.  Bars as for the Jacobi buckets: FP64 1e-8 (the
two sides differ by rounding order: Householder + QR against LAPACK), mixed
1e-4 (FP32 eigensolves, ~1e-6 of the block norm).
"""
import numpy as np
import pytest

import synth
from oracle import hsde as ohsde
from tests.test_gpu_parity import close, from_state, inner_product_scale, random_state, to_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_01828_gb300 import hsde
    return hsde


def small_box_qp():
    """Box-QP relaxation on 300 vertices, 1400 edges: 457 cliques of 1 to
    144 (5 above 112, 9 above 80), so the QR path runs beside the Jacobi
    buckets of both precisions."""
    return synth.box_qp(300, 1400, np.random.default_rng(7))


def _prec(hs, prec):
    return hs.FP64 if prec == "fp64" else hs.MIXED


@pytest.mark.parametrize("prec,c", [("mixed", 113), ("mixed", 200), ("mixed", 304), ("fp64", 81), ("fp64", 150)])
def test_qr_path_one_step_from_random_state(hs, prec, c):
    """Block-arrows whose cliques are all above the Jacobi sizes, one
    iteration from a random state against the oracle; the projection's
    residual partials and the ν update come out of the same kernel."""
    p = synth.block_arrow(2, c - 5, 5, 4, np.random.default_rng(c))
    ref = ohsde.HSDE(p)
    assert max(len(k) for k in ref.V.st.cliques) == c > hs.JACOBI_MAX[_prec(hs, prec)]
    state = random_state(ref, np.random.default_rng(11), f32=(prec == "mixed"))
    with hs.Handle(p, precision=prec, profile=1) as H:
        H.hsde_set_state(0, state, 0)
        H.hsde_iterate(1)
        got = H.hsde_get_state(0)
        sz = H.sizes[0]
        prof = H.hsde_get_profile()
        info = H.hsde_get_info(0)
    assert "cone_qr" in prof["phases"]
    assert info["jacobi_unconverged"] == 0
    u0, nu0 = from_state(ref, state, sz)
    u1, nu1, _ = ref.step(u0, nu0)
    close(ref, got, to_state(ref, u1, nu1), 1e-8 if prec == "fp64" else 1e-4, f"c = {c}, {prec}")


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_box_qp_one_step_from_random_state(hs, prec):
    """Uneven cliques (1 to 144) on the Jacobi buckets and the QR path in the
    same iteration."""
    p = small_box_qp()
    ref = ohsde.HSDE(p)
    sizes = [len(k) for k in ref.V.st.cliques]
    assert max(sizes) == 144 and min(sizes) == 1
    state = random_state(ref, np.random.default_rng(12), f32=(prec == "mixed"))
    with hs.Handle(p, precision=prec) as H:
        H.hsde_set_state(0, state, 0)
        H.hsde_iterate(1)
        got = H.hsde_get_state(0)
        sz = H.sizes[0]
    u0, nu0 = from_state(ref, state, sz)
    u1, nu1, _ = ref.step(u0, nu0)
    close(ref, got, to_state(ref, u1, nu1), 1e-8 if prec == "fp64" else 1e-4, f"box QP, {prec}")


def test_box_qp_first_iterations_fp64(hs):
    """The first 1, 5 and 20 iterations from the standard start, FP64."""
    p = small_box_qp()
    ref = ohsde.HSDE(p)
    u, nu = ref.initial()
    with hs.Handle(p, precision="fp64") as H:
        for k in (1, 4, 15):
            H.hsde_iterate(k)
            for _ in range(k):
                u, nu, _ = ref.step(u, nu)
            close(ref, H.hsde_get_state(0), to_state(ref, u, nu), 1e-8, f"box QP after {k}")


def test_box_qp_first_iterations_mixed(hs):
    """The first 20 mixed iterations from the standard start against the FP64
    oracle.  tau and kappa are measured against 1 + |c~^T x| + |b~^T y|, the
    size of the inner products tau_hat is formed from (as for the n = 2000
    grid's mixed iterations)."""
    p = small_box_qp()
    ref = ohsde.HSDE(p)
    u, nu = ref.initial()
    for _ in range(20):
        u, nu, _ = ref.step(u, nu)
    with hs.Handle(p, precision="mixed") as H:
        H.hsde_iterate(20)
        close(ref, H.hsde_get_state(0), to_state(ref, u, nu), 1e-4, "box QP mixed after 20",
              scalar_scale=inner_product_scale(ref, u))


def test_box_qp_solves_in_both_forms(hs):
    """Both forms reach SOLVED on the small box QP with objectives that agree
    within the stopping rule's accuracy, every large clique's projection
    converging (no eigensolve stopped at its step limit); the solution's
    clique blocks are PSD (Grone) and the dual blocks' Agler sum matches
    C - sum y_i A_i."""
    p = small_box_qp()
    objs = {}
    for prec in ("fp64", "mixed"):
        with hs.Handle(p, precision=prec) as H:
            st = H.solve(chunk=200)
            info = H.hsde_get_info(0)
            assert int(st[0]) == hs.SOLVED, (prec, info)
            assert info["jacobi_unconverged_iterations"] == 0, (prec, info)
            objs[prec] = info["pobj"]
    assert abs(objs["fp64"] - objs["mixed"]) <= 2e-3 * (1.0 + abs(objs["fp64"]))


def test_qr_path_batch_equals_single_bitwise(hs):
    """A QR-path instance batched with Jacobi-only instances iterates bitwise
    as it does alone."""
    big = synth.block_arrow(2, 125, 5, 4, np.random.default_rng(3))   # c = 130
    other = synth.maxcut_grid(6, 9, np.random.default_rng(4))
    with hs.Handle(big, precision="mixed") as H:
        H.hsde_iterate(15)
        alone = H.hsde_get_state(0)
    with hs.Handle([other, big], precision="mixed") as H:
        H.hsde_iterate(15)
        batched = H.hsde_get_state(1)
    assert np.array_equal(alone, batched)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_nan_in_a_qr_path_clique_gives_numerical_error(hs, prec):
    """A NaN planted in a large clique's s ends the instance with
    HSDE_NUMERICAL_ERROR after one iteration (the affine step already sees
    it), and it stays frozen."""
    p = synth.block_arrow(2, 125, 5, 4, np.random.default_rng(6))   # c = 130
    with hs.Handle(p, precision=prec) as H:
        H.hsde_iterate(3)
        sz = H.sizes[0]
        st = H.hsde_get_state(0)
        st[sz.N + 5] = np.nan
        H.hsde_set_state(0, st, 3)
        assert int(H.hsde_iterate(1)[0]) == hs.NUMERICAL_ERROR
        assert int(H.hsde_iterate(2)[0]) == hs.NUMERICAL_ERROR


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_clique_above_1024_rejected(hs, prec):
    p = synth.block_arrow(2, hs.MAX_CLIQUE[_prec(hs, prec)] + 1 - 5, 5, 2, np.random.default_rng(1))
    with pytest.raises(hs.HSDEError) as ei:
        hs.Handle(p, precision=prec)
    assert ei.value.code == hs.HSDE_ERANGE


def test_unrolled_differentiation_rejects_qr_path_cliques(hs):
    """The reverse mode records Jacobi eigenbases; cliques on the QR path
    give HSDE_ERANGE there, before any work."""
    p = synth.block_arrow(2, 120, 5, 4, np.random.default_rng(5))   # c = 125
    with hs.Handle(p, precision="mixed", alpha=1.0, scaling=0) as H:
        with pytest.raises(hs.HSDEError) as ei:
            H.hsde_unrolled_forward(5)
        assert ei.value.code == hs.HSDE_ERANGE


# ---------------------------------------------------------------------------
# the warp tridiagonal QR (one warp per clique, shared memory; mixed cliques
# of 33 to 64): options.eigensolver = 1 (the default 0 keeps the Jacobi)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("c", [33, 41, 55, 64])
def test_warp_qr_one_step_from_random_state(hs, c):
    p = synth.block_arrow(3, c - 5, 5, 6, np.random.default_rng(100 + c))
    ref = ohsde.HSDE(p)
    state = random_state(ref, np.random.default_rng(13), f32=True)
    with hs.Handle(p, precision="mixed", eigensolver=1, profile=1) as H:
        H.hsde_set_state(0, state, 0)
        H.hsde_iterate(1)
        got = H.hsde_get_state(0)
        sz = H.sizes[0]
        variants = H.hsde_get_profile()["phase_variant"]
        info = H.hsde_get_info(0)
    assert 3 in variants.values(), variants
    assert info["jacobi_unconverged"] == 0
    u0, nu0 = from_state(ref, state, sz)
    u1, nu1, _ = ref.step(u0, nu0)
    close(ref, got, to_state(ref, u1, nu1), 1e-4, f"warp QR, c = {c}")


def test_warp_qr_first_iterations_vs_oracle(hs):
    """The l = 100, d = 50 block-arrow (100 cliques of 55), 20 iterations from
    the standard start, warp QR forced, against the FP64 oracle."""
    p = synth.block_arrow_sweep(100, 50)
    ref = ohsde.HSDE(p)
    u, nu = ref.initial()
    for _ in range(20):
        u, nu, _ = ref.step(u, nu)
    with hs.Handle(p, precision="mixed", eigensolver=1) as H:
        H.hsde_iterate(20)
        close(ref, H.hsde_get_state(0), to_state(ref, u, nu), 1e-4, "warp QR after 20",
              scalar_scale=inner_product_scale(ref, u))


def test_warp_qr_and_jacobi_reach_the_same_verdict(hs):
    p = synth.block_arrow_sweep(100, 50)
    out = {}
    for es in (0, 1):
        with hs.Handle(p, precision="mixed", eigensolver=es) as H:
            st = H.solve(chunk=200)
            out[es] = (int(st[0]), H.hsde_get_info(0))
    assert out[0][0] == out[1][0] == hs.SOLVED
    o0, o1 = out[0][1]["pobj"], out[1][1]["pobj"]
    assert abs(o0 - o1) <= 2e-3 * (1.0 + abs(o0))
    it0, it1 = out[0][1]["iterations"], out[1][1]["iterations"]
    assert abs(it0 - it1) <= max(2, 0.1 * it0)


def test_warp_qr_only_when_asked_for(hs):
    """The default keeps the warm-started Jacobi on every bucket; with
    eigensolver = 1 the buckets of 33 to 64 run the warp QR and the others
    (and every FP64 bucket) the Jacobi."""
    p = synth.block_arrow_sweep(100, 50)
    q = synth.maxcut_grid(12, 30, np.random.default_rng(2))
    for prob, es, prec in ((p, 0, "mixed"), (p, 1, "mixed"), (q, 1, "mixed"), (p, 1, "fp64")):
        with hs.Handle(prob, precision=prec, eigensolver=es, profile=1) as H:
            H.hsde_iterate(2)
            var = H.hsde_get_profile()["phase_variant"]
        for name, v in var.items():
            cp = int(name[len("cone_c"):]) if name.startswith("cone_c") else 0
            want_qr = es == 1 and prec == "mixed" and 33 <= cp <= 64
            assert (v == 3) == want_qr, (prob.name, es, prec, name, v)
