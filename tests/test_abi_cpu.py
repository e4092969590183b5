"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/hsde.h declares, rejects invalid problems, and its host symbolic
analysis matches the oracle bit for bit."""
import os
import re

import numpy as np
import pytest

import synth
from oracle import symbolic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_1611_01828_gb300", "libhsde.so")


@pytest.fixture(scope="module")
def hs():
    if not os.path.exists(LIB):
        from paper_1611_01828_gb300 import _build
        _build.build()
    from paper_1611_01828_gb300 import hsde
    return hsde


def _declared():
    txt = open(os.path.join(ROOT, "include", "hsde.h")).read()
    return sorted(set(re.findall(r"HSDE_API\s+[\w\s\*]*?\b(hsde_\w+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(hs):
    names = _declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(hs.lib, n), n
    assert set(names) == set(hs._SIGS)


def test_default_options(hs):
    o = hs.default_options()
    assert o.eps_tol == 1e-4 and o.max_iter == 2000 and o.check_every == 1 and o.precision == hs.MIXED


def _cases():
    rng = np.random.default_rng(0)
    out = [synth.block_arrow_n50(), synth.block_arrow_n50(True), synth.maxcut_grid(7, 9, rng), synth.differentiation_maxcut_grid(),
           synth.block_arrow(5, 4, 3, 6, rng), synth.maxcut_grid_instance(), synth.box_qp_large_clique()]
    # random sparse patterns with fill
    for seed in range(4):
        n = 30 + 17 * seed
        r = rng.integers(0, n, 3 * n); c = rng.integers(0, n, 3 * n)
        lo, hi = np.maximum(r, c), np.minimum(r, c)
        key = np.unique(hi.astype(np.int64) * n + lo)
        rr = (key % n).astype(np.int32); cc = (key // n).astype(np.int32)
        out.append(synth.Problem(f"rand{seed}", n, 0, rr, cc, rng.standard_normal(len(rr)),
                                 np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32),
                                 np.zeros(0), np.zeros(0)))
    return out


@pytest.mark.parametrize("k", range(11))
def test_symbolic_bit_exact_against_oracle(hs, k):
    p = _cases()[k]
    got = hs.hsde_analyze(p)
    st = symbolic.analyze(p)
    assert np.array_equal(got["order"], st.order)
    assert np.array_equal(got["clique_ptr"], st.clique_ptr)
    assert np.array_equal(got["clique_idx"], st.clique_idx)
    assert np.array_equal(got["pat_colptr"], st.pat_colptr)
    assert np.array_equal(got["pat_row"], st.pat_row)
    assert np.array_equal(got["gather"], st.gather)
    assert np.array_equal(got["D"], st.D)
    assert got["n_d"] == st.n_d and got["P"] == st.P


def _mutate(p, **kw):
    q = synth.Problem(**{**p.__dict__})
    for k, v in kw.items():
        setattr(q, k, v)
    return q


def test_invalid_inputs_rejected(hs):
    p = synth.block_arrow_n50()
    bad = [
        _mutate(p, n=0),
        _mutate(p, C_row=np.where(np.arange(len(p.C_row)) == 3, 999, p.C_row).astype(np.int32)),
        _mutate(p, C_row=p.C_col.copy(), C_col=p.C_row.copy()),                       # upper triangle
        _mutate(p, C_val=np.where(np.arange(len(p.C_val)) == 0, np.nan, p.C_val)),
        _mutate(p, b=np.where(np.arange(p.m) == 0, np.inf, p.b)),
        _mutate(p, A_ptr=p.A_ptr[::-1].copy()),
    ]
    # duplicate entry inside C
    dup = _mutate(p, C_row=np.concatenate([p.C_row, p.C_row[:1]]), C_col=np.concatenate([p.C_col, p.C_col[:1]]),
                  C_val=np.concatenate([p.C_val, p.C_val[:1]]))
    bad.append(dup)
    for q in bad:
        with pytest.raises(hs.HSDEError) as ei:
            hs.hsde_analyze(q)
        assert ei.value.code == hs.HSDE_EINVAL


def test_default_options_of_the_practical_form(hs):
    # reading P7: the same defaults as the oracle
    from oracle import hsde as ohsde
    o = hs.default_options()
    assert o.alpha == ohsde.ALPHA and o.scaling == 1
    assert o.scale_norm == ohsde.SCALE_NORM and o.dual_weight == ohsde.DUAL_WEIGHT
    assert o.autotune == 1


@pytest.mark.parametrize("kw", [dict(alpha=0.0), dict(alpha=2.0), dict(scaling=2), dict(scale_norm=0.0),
                                dict(dual_weight=-1.0), dict(eps_tol=0.0), dict(max_iter=0), dict(autotune=5),
                                dict(autotune=-1), dict(eigensolver=2), dict(eigensolver=-1)])
def test_invalid_options_rejected_before_any_device_call(hs, kw):
    with pytest.raises(hs.HSDEError) as ei:
        hs.Handle(synth.block_arrow_n50(), **kw)
    assert ei.value.code == hs.HSDE_EINVAL


def test_clique_beyond_the_largest_eigensolver_is_rejected(hs):
    """A clique larger than the library's eigensolvers take gives HSDE_ERANGE
    at setup, before any device call (so this needs no GPU)."""
    big = 8 + hs.MAX_CLIQUE[hs.MIXED]      # the default precision
    p = synth.block_arrow(2, big - 5, 5, 4, np.random.default_rng(3))
    assert hs.hsde_analyze(p)["c_max"] == big
    with pytest.raises(hs.HSDEError) as ei:
        hs.Handle(p)
    assert ei.value.code == hs.HSDE_ERANGE
    assert str(big) in str(ei.value)


def test_large_block_arrow_structure_closed_form(hs):
    """The l = 2000, d = 50, h = 5 block-arrow (n = 100,005; the arrow rows are
    adjacent to every vertex): zero fill, the cliques are block_j U arrow in
    block order, N = l (d(d+1)/2 + d h) + h(h+1)/2, and D counts l cliques on
    the arrow corner and one elsewhere.  Also a guard on the analysis time:
    the arrow rows once made it quadratic in n."""
    import time
    l, d, h = 2000, 50, 5
    p = synth.block_arrow_sweep(l, d, h)
    t0 = time.perf_counter()
    st = hs.hsde_analyze(p)
    dt = time.perf_counter() - t0
    n = l * d + h
    assert st["p"] == l and st["c_max"] == d + h
    assert st["N"] == l * (d * (d + 1) // 2 + d * h) + h * (h + 1) // 2
    ptr, idx = st["clique_ptr"], st["clique_idx"]
    arrow = np.arange(n - h, n)
    for j in (0, 1, l // 2, l - 1):
        mem = idx[ptr[j]:ptr[j + 1]]
        assert np.array_equal(mem, np.concatenate([np.arange(j * d, (j + 1) * d), arrow]))
    col = np.repeat(np.arange(n), np.diff(st["pat_colptr"]))
    corner = (st["pat_row"] >= n - h) & (col >= n - h)
    assert np.all(st["D"][corner] == l) and np.all(st["D"][~corner] == 1)
    assert dt < 20.0, dt
