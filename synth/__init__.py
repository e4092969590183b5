"""Seeded synthetic SDP instances shaped like the paper's benchmark problems.

This module only *generates data*: sparse problem matrices C, A_1..A_m and the
vector b of the primal-dual pair (Section 3, Eqs. PrimalSDP / DualSDP).  It
holds none of the method's arithmetic (no chordal analysis, no ADMM, no
projection) so that both the FP64 oracle and the CUDA path can be fed from the
same inputs without sharing any code.

SDPLIB itself is not available, so the instances stand in for it, following
the shapes of Table 1 (problem size n, number of constraints m, clique count
and clique-size range):

* ``block_arrow``     -- l diagonal blocks of size d plus an arrow of width h.
                         Cliques are exactly ``block_j U arrow`` (size d+h).
                         Feasible by construction (X0 > 0 and Z0 > 0 given).
* ``maxcut_grid``     -- max-cut relaxation on an open R x K grid graph with
                         +-1 edge weights: C = weighted Laplacian, A_i = e_i e_i^T,
                         b = 1 (the maxG-type rows of Table 1).
* ``box_qp``          -- SDP relaxation of a box-constrained QP on a random
                         graph: X = diag(X1, S) with X1_ii + S_ii = 1 and
                         C = [[L_w, 0], [0, 0]] (the qpG-type rows of Table 1:
                         n = 2 n1, m = n1, singleton slack cliques plus the
                         graph's chordal cliques, up to ~300 vertices).
* ``make_primal_infeasible`` -- appends tr(X) = -1 (the infp-type row).
* ``make_dual_infeasible``   -- tilts C along a PSD direction in the null
                         space of A (the infd-type row).

Every matrix is returned as the LOWER triangle (row >= col) in COO form with
no duplicate entries, which is the convention of the C-ABI ``hsde_problem``.
Random numbers come from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem", "block_arrow", "maxcut_grid", "make_primal_infeasible",
    "make_dual_infeasible", "trace_one", "block_arrow_n50", "maxcut_grid_instance", "block_arrow_sweep",
    "serving_batch", "differentiation_maxcut_grid", "rng_for", "box_qp", "box_qp_large_clique",
]


@dataclass
class Problem:
    """One SDP instance: min <C,X> s.t. <A_i,X> = b_i, X psd (lower-triangle COO)."""

    name: str
    n: int
    m: int
    C_row: np.ndarray          # int32 [C_nnz]
    C_col: np.ndarray          # int32 [C_nnz]
    C_val: np.ndarray          # float64 [C_nnz]
    A_ptr: np.ndarray          # int64 [m+1]; entries of A_i are A_ptr[i]:A_ptr[i+1]
    A_row: np.ndarray          # int32
    A_col: np.ndarray          # int32
    A_val: np.ndarray          # float64
    b: np.ndarray              # float64 [m]
    kind: str = "feasible"     # "feasible" | "primal_infeasible" | "dual_infeasible"
    meta: dict = field(default_factory=dict)

    def data_bytes(self) -> int:
        arrs = [self.C_row, self.C_col, self.C_val, self.A_ptr, self.A_row,
                self.A_col, self.A_val, self.b]
        return int(sum(a.nbytes for a in arrs))


def rng_for(config: int, instance: int = 0) -> np.random.Generator:
    """Seed convention: PCG64(1000*config + instance)."""
    return np.random.Generator(np.random.PCG64(1000 * config + instance))


# ----------------------------------------------------------------------------
# helpers on lower-triangle COO data (pure data plumbing)
# ----------------------------------------------------------------------------

def _lower_key(r, c, n):
    return r.astype(np.int64) * n + c.astype(np.int64)


def _dedup_sum(r, c, v, n):
    """Sum duplicates of a lower COO list and sort by (col, row)."""
    key = c.astype(np.int64) * n + r.astype(np.int64)
    order = np.argsort(key, kind="stable")
    key, v = key[order], v[order]
    uk, inv = np.unique(key, return_inverse=True)
    vv = np.zeros(uk.shape[0])
    np.add.at(vv, inv, v)
    return (uk % n).astype(np.int32), (uk // n).astype(np.int32), vv


def _clique_lower_entries(members):
    """All (row, col) lower pairs inside one clique (members ascending)."""
    mem = np.asarray(members, dtype=np.int64)
    ii, jj = np.tril_indices(mem.shape[0])
    return mem[ii].astype(np.int32), mem[jj].astype(np.int32)


def _pack_constraints(rows, cols, vals, b, n):
    ptr = np.zeros(len(rows) + 1, dtype=np.int64)
    rr, cc, vv = [], [], []
    for i, (r, c, v) in enumerate(zip(rows, cols, vals)):
        r2, c2, v2 = _dedup_sum(np.asarray(r), np.asarray(c), np.asarray(v, dtype=np.float64), n)
        rr.append(r2); cc.append(c2); vv.append(v2)
        ptr[i + 1] = ptr[i] + r2.shape[0]
    cat = (lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt))
    return ptr, cat(rr, np.int32), cat(cc, np.int32), cat(vv, np.float64), np.asarray(b, np.float64)


def _sym_inner(r1, c1, v1, r2, c2, v2, n):
    """Frobenius inner product <M1, M2> of two symmetric matrices given as lower COO."""
    k1 = _lower_key(r1, c1, n)
    k2 = _lower_key(r2, c2, n)
    common, i1, i2 = np.intersect1d(k1, k2, assume_unique=True, return_indices=True)
    w = np.where(r1[i1] == c1[i1], 1.0, 2.0)
    return float(np.sum(w * v1[i1] * v2[i2]))


def _psd_on_cliques(rng, n, cliques, kappa):
    """X = sum_k E_k^T G_k G_k^T E_k + sigma I with cond(X) <= kappa.

    sigma uses a Gershgorin upper bound of lambda_max (lambda_min >= 0 for the
    sum of Gram blocks), so the bound on the condition number always holds.
    Returned as lower COO."""
    rr, cc, vv = [], [], []
    for mem in cliques:
        k = len(mem)
        G = rng.standard_normal((k, k))
        Y = G @ G.T
        ii, jj = np.tril_indices(k)
        mem = np.asarray(mem)
        rr.append(mem[ii]); cc.append(mem[jj]); vv.append(Y[ii, jj])
    r, c, v = _dedup_sum(np.concatenate(rr), np.concatenate(cc), np.concatenate(vv), n)
    # Gershgorin: lambda_max <= max_i sum_j |Y_ij|
    rowsum = np.zeros(n)
    np.add.at(rowsum, r, np.abs(v))
    off = r != c
    np.add.at(rowsum, c[off], np.abs(v[off]))
    lam_ub = float(rowsum.max())
    sigma = lam_ub / (kappa - 1.0)
    diag = r == c
    v = v.copy()
    v[diag] += sigma
    return r, c, v


# ----------------------------------------------------------------------------
# families
# ----------------------------------------------------------------------------

def block_arrow_cliques(l, d, h):
    arrow = list(range(l * d, l * d + h))
    return [list(range(j * d, (j + 1) * d)) + arrow for j in range(l)]


def block_arrow(l, d, h, m, rng, *, dense_constraints=False, kappa=1e3,
                assign="pairs", name=None):
    """Block-arrow SDP, primal and dual strictly feasible by construction.

    Pattern: l diagonal d x d blocks, an arrow of width h (the last h indices)
    coupled to every block.  Constraints:
      * dense_constraints=True : every A_i is N(0,1) iid on every lower entry
                                 of the whole pattern (mirrored);
      * assign="pairs"         : constraint i lives on clique (i // 2) mod l;
      * assign="roundrobin"    : constraint i lives on clique i mod l.
    b = A(X0) for X0 > 0 on the pattern, C = sum_i y0_i A_i + Z0, Z0 > 0.
    """
    n = l * d + h
    cliques = block_arrow_cliques(l, d, h)
    pr, pc = [], []
    for mem in cliques:
        r, c = _clique_lower_entries(mem)
        pr.append(r); pc.append(c)
    if dense_constraints:
        pat_r, pat_c, _ = _dedup_sum(np.concatenate(pr), np.concatenate(pc),
                                     np.zeros(sum(len(x) for x in pr)), n)
        E = pat_r.shape[0]
        Ar = np.tile(pat_r, m); Ac = np.tile(pat_c, m)
    else:
        # every clique has the same number of lower entries E; sort each
        # clique's list by (col, row) once
        E = pr[0].shape[0]
        cr = np.stack(pr); cc = np.stack(pc)
        order = np.argsort(cc.astype(np.int64) * n + cr, axis=1, kind="stable")
        cr = np.take_along_axis(cr, order, 1); cc = np.take_along_axis(cc, order, 1)
        j = (np.arange(m) // 2) % l if assign == "pairs" else np.arange(m) % l
        Ar = cr[j].reshape(-1); Ac = cc[j].reshape(-1)
    Av = rng.standard_normal(m * E)
    X0 = _psd_on_cliques(rng, n, cliques, kappa)
    Z0 = _psd_on_cliques(rng, n, cliques, kappa)
    y0 = rng.standard_normal(m)
    A_ptr = np.arange(m + 1, dtype=np.int64) * E
    A_row = Ar.astype(np.int32); A_col = Ac.astype(np.int32); A_val = Av
    b = _apply_A(A_ptr, A_row, A_col, A_val, X0, n)
    # C = sum_i y0_i A_i + Z0
    Cr = np.concatenate([A_row, Z0[0]])
    Cc = np.concatenate([A_col, Z0[1]])
    Cv = np.concatenate([np.repeat(y0, E) * A_val, Z0[2]])
    C_row, C_col, C_val = _dedup_sum(Cr, Cc, Cv, n)
    return Problem(name or f"block_arrow_l{l}_d{d}_h{h}_m{m}", n, m, C_row, C_col, C_val,
                   A_ptr, A_row, A_col, A_val, b, "feasible",
                   dict(family="block_arrow", l=l, d=d, h=h, X0=X0, Z0=Z0, y0=y0))


def _apply_A(A_ptr, A_row, A_col, A_val, X, n):
    """b_i = <A_i, X> (Frobenius) for all constraints, X given as lower COO."""
    xr, xc, xv = X
    xkey = xc.astype(np.int64) * n + xr
    srt = np.argsort(xkey)
    xkey, xv = xkey[srt], xv[srt]
    akey = A_col.astype(np.int64) * n + A_row
    pos = np.searchsorted(xkey, akey)
    pos_c = np.minimum(pos, xkey.shape[0] - 1)
    hit = (pos < xkey.shape[0]) & (xkey[pos_c] == akey)
    vals = np.where(hit, xv[pos_c], 0.0)
    w = np.where(A_row == A_col, 1.0, 2.0)
    contrib = w * A_val * vals
    m = A_ptr.shape[0] - 1
    out = np.zeros(m)
    nz = np.diff(A_ptr) > 0
    if contrib.shape[0]:
        sums = np.add.reduceat(contrib, A_ptr[:-1][nz])
        out[nz] = sums
    return out


def maxcut_grid(R, K, rng, name=None):
    """Max-cut relaxation on the open R x K grid (vertex i*K + j).

    C = weighted Laplacian L_w with edge weights +-1 (uniform), A_i = e_i e_i^T,
    b = 1, minimised as stated (min <L_w, X>)."""
    n = R * K
    v = np.arange(n).reshape(R, K)
    # edges in the order (row-major vertex, right neighbour first, then down)
    right = np.stack([v[:, :-1] + 1, v[:, :-1]], -1)          # (R, K-1, 2)
    down = np.stack([v[:-1, :] + K, v[:-1, :]], -1)           # (R-1, K, 2)
    er_l, ec_l = [], []
    for i in range(R):
        blk = []
        for j in range(K):
            if j + 1 < K:
                blk.append(right[i, j])
            if i + 1 < R:
                blk.append(down[i, j])
        if blk:
            blk = np.asarray(blk)
            er_l.append(blk[:, 0]); ec_l.append(blk[:, 1])
    er = np.concatenate(er_l).astype(np.int32); ec = np.concatenate(ec_l).astype(np.int32)
    w = rng.choice(np.array([-1.0, 1.0]), size=er.shape[0])
    deg = np.zeros(n)
    np.add.at(deg, er, w); np.add.at(deg, ec, w)
    Cr = np.concatenate([np.arange(n, dtype=np.int32), er])
    Cc = np.concatenate([np.arange(n, dtype=np.int32), ec])
    Cv = np.concatenate([deg, -w])
    C_row, C_col, C_val = _dedup_sum(Cr, Cc, Cv, n)
    idx = np.arange(n, dtype=np.int32)
    A_ptr = np.arange(n + 1, dtype=np.int64)
    return Problem(name or f"maxcut_grid_{R}x{K}", n, n, C_row, C_col, C_val, A_ptr,
                   idx.copy(), idx.copy(), np.ones(n), np.ones(n), "feasible",
                   dict(family="maxcut_grid", R=R, K=K))


def box_qp(n1, E, rng, name=None):
    """SDP relaxation of min x^T L_w x over x in [-1, 1]^n1 on a uniform random
    graph with E edges (+-1 weights), the box written with slacks:
    X = [[X1, .], [., S]] of size n = 2 n1, constraints X1_ii + S_ii = 1
    (m = n1, b = 1), C = [[L_w, 0], [0, 0]].  X = I/2 is feasible and
    X1_ii <= 1 bounds the objective.  The slack diagonal gives n1 singleton
    cliques; the graph part gives the chordal cliques."""
    n = 2 * n1
    seen = set()
    er, ec = [], []
    while len(er) < E:
        a, b = (int(t) for t in rng.integers(0, n1, 2))
        if a == b:
            continue
        r, c = max(a, b), min(a, b)
        if (r, c) in seen:
            continue
        seen.add((r, c))
        er.append(r)
        ec.append(c)
    er = np.asarray(er, np.int32)
    ec = np.asarray(ec, np.int32)
    w = rng.choice(np.array([-1.0, 1.0]), size=E)
    deg = np.zeros(n1)
    np.add.at(deg, er, w)
    np.add.at(deg, ec, w)
    Cr = np.concatenate([np.arange(n1, dtype=np.int32), er])
    Cc = np.concatenate([np.arange(n1, dtype=np.int32), ec])
    Cv = np.concatenate([deg, -w])
    C_row, C_col, C_val = _dedup_sum(Cr, Cc, Cv, n)
    i = np.arange(n1, dtype=np.int32)
    A_ptr = np.arange(0, 2 * n1 + 1, 2, dtype=np.int64)
    A_row = np.stack([i, i + n1], 1).ravel().astype(np.int32)
    return Problem(name or f"box_qp_n{n}_E{E}", n, n1, C_row, C_col, C_val, A_ptr, A_row, A_row.copy(),
                   np.ones(2 * n1), np.ones(n1), "feasible", dict(family="box_qp", n1=n1, E=E))


def trace_one(C_row, C_col, C_val, n, name="trace_one"):
    """min <C,X> s.t. tr X = 1, X psd; optimum lambda_min(C)."""
    idx = np.arange(n, dtype=np.int32)
    return Problem(name, n, 1, np.asarray(C_row, np.int32), np.asarray(C_col, np.int32),
                   np.asarray(C_val, np.float64), np.array([0, n], np.int64), idx.copy(),
                   idx.copy(), np.ones(n), np.ones(1), "feasible", dict(family="trace_one"))


def make_primal_infeasible(p: Problem) -> Problem:
    """Append the constraint tr(X) = -1 (no psd X satisfies it)."""
    n = p.n
    idx = np.arange(n, dtype=np.int32)
    A_ptr = np.concatenate([p.A_ptr, [p.A_ptr[-1] + n]]).astype(np.int64)
    meta = dict(p.meta)
    return Problem(p.name + "_pinf", n, p.m + 1, p.C_row.copy(), p.C_col.copy(), p.C_val.copy(),
                   A_ptr, np.concatenate([p.A_row, idx]), np.concatenate([p.A_col, idx]),
                   np.concatenate([p.A_val, np.ones(n)]), np.concatenate([p.b, [-1.0]]),
                   "primal_infeasible", meta)


def make_dual_infeasible(p: Problem, rng) -> Problem:
    """Tilt a block-arrow instance so that it is primal feasible but unbounded.

    g is a random unit vector on clique 0 and Dd = E_0^T g g^T E_0 (psd).
    Every A_i is made orthogonal to Dd and C gets <C, Dd> = -1; b = A(X0) keeps
    X0 feasible, so X0 + t*Dd is feasible for all t >= 0 with cost -> -inf."""
    assert p.meta.get("family") == "block_arrow"
    l, d, h = p.meta["l"], p.meta["d"], p.meta["h"]
    n = p.n
    mem = np.asarray(block_arrow_cliques(l, d, h)[0])
    g = rng.standard_normal(mem.shape[0]); g /= np.linalg.norm(g)
    ii, jj = np.tril_indices(mem.shape[0])
    Dr, Dc, Dv = mem[ii].astype(np.int32), mem[jj].astype(np.int32), np.outer(g, g)[ii, jj]
    DD = _sym_inner(Dr, Dc, Dv, Dr, Dc, Dv, n)
    # <A_i, Dd> for every constraint at once
    coef = _apply_A(p.A_ptr, p.A_row, p.A_col, p.A_val, (Dr, Dc, Dv), n) / DD
    # A_i <- A_i - coef_i Dd  (support grows to include clique 0)
    m = p.m
    cnt = np.diff(p.A_ptr)
    inst = np.repeat(np.arange(m), cnt)
    allr = np.concatenate([p.A_row, np.tile(Dr, m)])
    allc = np.concatenate([p.A_col, np.tile(Dc, m)])
    alli = np.concatenate([inst, np.repeat(np.arange(m), Dr.shape[0])])
    allv = np.concatenate([p.A_val, -np.repeat(coef, Dr.shape[0]) * np.tile(Dv, m)])
    key = (alli.astype(np.int64) * n + allc) * n + allr
    uk, inv = np.unique(key, return_inverse=True)
    vv = np.zeros(uk.shape[0])
    np.add.at(vv, inv, allv)
    ui = uk // (n * n); rem = uk % (n * n)
    A_row = (rem % n).astype(np.int32); A_col = (rem // n).astype(np.int32)
    A_ptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(A_ptr, ui + 1, 1)
    A_ptr = np.cumsum(A_ptr)
    A_val = vv
    X0 = p.meta["X0"]
    b = _apply_A(A_ptr, A_row, A_col, A_val, X0, n)
    cD = _sym_inner(p.C_row, p.C_col, p.C_val, Dr, Dc, Dv, n)
    C_row, C_col, C_val = _dedup_sum(np.concatenate([p.C_row, Dr]), np.concatenate([p.C_col, Dc]),
                                     np.concatenate([p.C_val, -(cD + 1.0) / DD * Dv]), n)
    meta = dict(p.meta); meta["Dd"] = (Dr, Dc, Dv)
    return Problem(p.name + "_dinf", n, p.m, C_row, C_col, C_val, A_ptr, A_row, A_col, A_val, b,
                   "dual_infeasible", meta)


# ----------------------------------------------------------------------------
# the five workload configurations
# ----------------------------------------------------------------------------

def block_arrow_n50(infeasible=False):
    """n=50 block-arrow (8 blocks of 6, arrow 2), m=20 dense constraints, cond(X0)<=100."""
    p = block_arrow(8, 6, 2, 20, rng_for(0), dense_constraints=True, kappa=100.0,
                    name="block_arrow_n50_m20")
    return make_primal_infeasible(p) if infeasible else p


def maxcut_grid_instance(R=20, K=100, instance=0):
    """maxG32-shaped max-cut: open 20 x 100 grid (n=2000, m=2000)."""
    return maxcut_grid(R, K, rng_for(1, instance), name=f"maxcut_grid{R}x{K}")


def block_arrow_sweep(l, d, h=5, instance=0):
    """Block-arrow sweep: m = 2l, constraints 2j, 2j+1 dense on clique j, cond <= 1e3."""
    return block_arrow(l, d, h, 2 * l, rng_for(2, instance), kappa=1e3, assign="pairs",
                       name=f"block_arrow_l{l}_d{d}")


def serving_batch(B=256, n_lo=100, n_hi=1500, seed_instance=0, select=None):
    """Batch of B independent instances of uneven sizes.

    Half max-cut grids (m = n), half block-arrow with m ~ U[n/2, 2n] assigned
    round-robin to cliques.  10% made primal-infeasible, 10% dual-infeasible
    (block-arrow only, since diag(X)=1 bounds the max-cut feasible set).
    `select` (iterable of indices) builds only those instances; every
    instance is the same whichever subset is built."""
    rng = rng_for(3, seed_instance)
    n_pinf = B // 10
    n_dinf = B // 10
    kinds = ["feasible"] * B
    # choose infeasible slots deterministically: dual-infeasible among block-arrow ones (odd)
    odd = [i for i in range(B) if i % 2 == 1]
    sel = rng.permutation(len(odd))[:n_dinf]
    for s in sel:
        kinds[odd[s]] = "dual_infeasible"
    rest = [i for i in range(B) if kinds[i] == "feasible"]
    for s in rng.permutation(len(rest))[:n_pinf]:
        kinds[rest[s]] = "primal_infeasible"
    specs = []
    for i in range(B):
        n = int(rng.integers(n_lo, n_hi + 1))
        if i % 2 == 0:
            specs.append(("grid", n, None, None))
        else:
            d = [10, 25, 50][int(rng.integers(0, 3))]
            l = max(2, (n - 5) // d)
            nn = l * d + 5
            m = int(rng.integers(max(1, nn // 2), 2 * nn + 1))
            specs.append(("arrow", n, d, m))
    out = []
    for i in (range(B) if select is None else select):
        kind, n, d, m = specs[i]
        sub = np.random.Generator(np.random.PCG64(3000 + 7919 * (seed_instance + 1) + i))
        if kind == "grid":
            R = 10
            K = max(2, n // R)
            p = maxcut_grid(R, K, sub, name=f"batch_{i}_maxcut_{R}x{K}")
        else:
            l = max(2, (n - 5) // d)
            p = block_arrow(l, d, 5, m, sub, kappa=1e3, assign="roundrobin",
                            name=f"batch_{i}_block_arrow_l{l}_d{d}_m{m}")
        if kinds[i] == "primal_infeasible":
            p = make_primal_infeasible(p)
        elif kinds[i] == "dual_infeasible":
            p = make_dual_infeasible(p, sub)
        out.append(p)
    return out


def differentiation_maxcut_grid():
    """Differentiation workload: max-cut on the open 10 x 100 grid (n=1000)."""
    return maxcut_grid(10, 100, rng_for(4), name="maxcut_grid10x100_diff")


def box_qp_large_clique(instance=0):
    """qpG51-shaped large-clique workload (Table 1: n = 2000, m = 1000,
    p = 1675, cliques 1-304): the box-QP relaxation on a random graph with
    1000 vertices and 2700 edges, whose minimum-degree chordal extension has
    cliques up to ~300."""
    return box_qp(1000, 2700, rng_for(5, instance), name="box_qp_n2000_E2700")
