"""ctypes binding of libhsde (include/hsde.h): argument marshalling only.

Every computation runs inside the library; this module converts NumPy arrays
to pointers and checks return codes.  The functions carry the C names.  If
the library is missing, importing this module raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhsde.so")

HSDE_OK, HSDE_EINVAL, HSDE_ENOMEM, HSDE_ECUDA, HSDE_ESTATE, HSDE_ERANGE = 0, -1, -2, -3, -4, -5
RUNNING, SOLVED, PRIMAL_INFEASIBLE, DUAL_INFEASIBLE, MAX_ITER, NUMERICAL_ERROR = 0, 1, 2, 3, 4, 5
STATUS_NAMES = {0: "running", 1: "solved", 2: "primal_infeasible", 3: "dual_infeasible", 4: "max_iter",
                5: "numerical_error"}
FP64, MIXED = 0, 1
MAX_CLIQUE = {FP64: 1024, MIXED: 1024}   # largest clique of the eigensolvers (HSDE_ERANGE above)
JACOBI_MAX = {FP64: 80, MIXED: 112}     # above: the tridiagonal QR path ("cone_qr")

_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_f64p = C.POINTER(C.c_double)


class hsde_problem(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("C_nnz", C.c_int64),
                ("C_row", _i32p), ("C_col", _i32p), ("C_val", _f64p),
                ("A_ptr", _i64p), ("A_row", _i32p), ("A_col", _i32p), ("A_val", _f64p),
                ("b", _f64p), ("pattern_nnz", C.c_int64), ("pattern_row", _i32p), ("pattern_col", _i32p)]


class hsde_options(C.Structure):
    _fields_ = [("eps_tol", C.c_double), ("max_iter", C.c_int32), ("check_every", C.c_int32),
                ("precision", C.c_int32), ("device", C.c_int32), ("cuda_stream", C.c_void_p),
                ("jacobi_max_sweeps", C.c_int32), ("use_graph", C.c_int32), ("jacobi_tol", C.c_double),
                ("profile", C.c_int32), ("warm_start", C.c_int32), ("warm_refresh", C.c_int32),
                ("scaling", C.c_int32), ("structured_factor", C.c_int32), ("alpha", C.c_double), ("scale_norm", C.c_double),
                ("dual_weight", C.c_double), ("autotune", C.c_int32), ("eigensolver", C.c_int32)]


class hsde_sizes(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("p", C.c_int32), ("c_max", C.c_int32),
                ("N", C.c_int64), ("P", C.c_int64), ("n_d", C.c_int64), ("state_len", C.c_int64),
                ("S_dense", C.c_int32), ("_pad", C.c_int32)]


class hsde_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("pres", C.c_double),
                ("dres", C.c_double), ("gap", C.c_double), ("pobj", C.c_double), ("dobj", C.c_double),
                ("tau", C.c_double), ("kappa", C.c_double), ("pinf_ratio", C.c_double),
                ("dinf_ratio", C.c_double), ("setup_ms", C.c_double), ("iterate_ms", C.c_double),
                ("jacobi_unconverged", C.c_int32), ("jacobi_unconverged_iterations", C.c_int32)]


MAX_PHASES = 24


class hsde_profile(C.Structure):
    _fields_ = [("kernels_per_iteration", C.c_int32), ("nphases", C.c_int32),
                ("phase_ms", C.c_double * MAX_PHASES), ("phase_name", (C.c_char * 24) * MAX_PHASES),
                ("phase_units", C.c_int64 * MAX_PHASES), ("sweeps_mean", C.c_double),
                ("sweeps_max", C.c_int32), ("_pad", C.c_int32),
                ("phase_sweeps_max", C.c_int32 * MAX_PHASES), ("phase_variant", C.c_int32 * MAX_PHASES)]


# Every function declared in include/hsde.h: name -> (restype, argtypes)
_SIGS = {
    "hsde_default_options": (None, [C.POINTER(hsde_options)]),
    "hsde_last_error": (C.c_char_p, []),
    "hsde_analyze": (C.c_int, [C.POINTER(hsde_problem), C.POINTER(C.c_void_p)]),
    "hsde_symbolic_sizes": (C.c_int, [C.c_void_p, C.POINTER(hsde_sizes)]),
    "hsde_symbolic_get": (C.c_int, [C.c_void_p] + [_i32p] * 7),
    "hsde_symbolic_free": (None, [C.c_void_p]),
    "hsde_setup": (C.c_int, [C.POINTER(hsde_problem), C.POINTER(hsde_options), C.POINTER(C.c_void_p)]),
    "hsde_setup_batch": (C.c_int, [C.POINTER(hsde_problem), C.c_int32, C.POINTER(hsde_options),
                                   C.POINTER(C.c_void_p)]),
    "hsde_iterate": (C.c_int, [C.c_void_p, C.c_int32, _i32p]),
    "hsde_sync": (C.c_int, [C.c_void_p]),
    "hsde_num_instances": (C.c_int, [C.c_void_p]),
    "hsde_get_sizes": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(hsde_sizes)]),
    "hsde_get_structure": (C.c_int, [C.c_void_p, C.c_int32] + [_i32p] * 7),
    "hsde_get_info": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(hsde_info)]),
    "hsde_get_state": (C.c_int, [C.c_void_p, C.c_int32, _f64p]),
    "hsde_set_state": (C.c_int, [C.c_void_p, C.c_int32, _f64p, C.c_int32]),
    "hsde_get_solution": (C.c_int, [C.c_void_p, C.c_int32, _f64p, _f64p, _f64p, _f64p, _f64p]),
    "hsde_get_certificate": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, _f64p, _f64p, _f64p]),
    "hsde_get_profile": (C.c_int, [C.c_void_p, C.POINTER(hsde_profile)]),
    "hsde_destroy": (None, [C.c_void_p]),
    "hsde_spd_inverse": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "hsde_set_data": (C.c_int, [C.c_void_p, C.c_int32, _f64p, _f64p]),
    "hsde_unrolled_forward": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, _f64p, _f64p, _f64p, _f64p]),
    "hsde_unrolled_backward": (C.c_int, [C.c_void_p, _f64p, _f64p, C.c_double, C.c_double, _f64p, _f64p]),
    "hsde_spd_inverse_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhsde.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class HSDEError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where} failed ({code}): {lib.hsde_last_error().decode()}")


def _ck(code, where):
    if code != HSDE_OK:
        raise HSDEError(code, where)


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def _dptr(a, n=None):
    """(ctypes pointer, keep-alive) for an FP64 array argument that may be a
    NumPy array (host memory) or an int (a device address of n values)."""
    if a is None:
        return None, None
    if isinstance(a, int):
        return C.cast(C.c_void_p(a), C.POINTER(C.c_double)), None
    arr = np.ascontiguousarray(a, np.float64)
    if n is not None and arr.shape[0] != n:
        raise ValueError(f"expected {n} values, got {arr.shape[0]}")
    return _ptr(arr, C.c_double), arr


class _ProblemView:
    """Keeps the contiguous arrays alive while the C struct points at them."""

    def __init__(self, p):
        self.arrs = dict(
            C_row=np.ascontiguousarray(p.C_row, np.int32), C_col=np.ascontiguousarray(p.C_col, np.int32),
            C_val=np.ascontiguousarray(p.C_val, np.float64), A_ptr=np.ascontiguousarray(p.A_ptr, np.int64),
            A_row=np.ascontiguousarray(p.A_row, np.int32), A_col=np.ascontiguousarray(p.A_col, np.int32),
            A_val=np.ascontiguousarray(p.A_val, np.float64), b=np.ascontiguousarray(p.b, np.float64))
        pr = getattr(p, "pattern_row", None)
        self.arrs["pattern_row"] = np.ascontiguousarray(pr, np.int32) if pr is not None else np.zeros(0, np.int32)
        pc = getattr(p, "pattern_col", None)
        self.arrs["pattern_col"] = np.ascontiguousarray(pc, np.int32) if pc is not None else np.zeros(0, np.int32)
        a = self.arrs
        self.s = hsde_problem(int(p.n), int(p.m), a["C_row"].shape[0], _ptr(a["C_row"], C.c_int32),
                              _ptr(a["C_col"], C.c_int32), _ptr(a["C_val"], C.c_double),
                              _ptr(a["A_ptr"], C.c_int64), _ptr(a["A_row"], C.c_int32),
                              _ptr(a["A_col"], C.c_int32), _ptr(a["A_val"], C.c_double),
                              _ptr(a["b"], C.c_double), a["pattern_row"].shape[0],
                              _ptr(a["pattern_row"], C.c_int32), _ptr(a["pattern_col"], C.c_int32))


def default_options(**kw) -> hsde_options:
    o = hsde_options()
    lib.hsde_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": FP64, "mixed": MIXED}[v]
        setattr(o, k, v)
    return o


def _structure(getter, obj, idx, sz):
    n, p, N, P = sz.n, sz.p, sz.N, sz.P
    out = dict(order=np.zeros(n, np.int32), clique_ptr=np.zeros(p + 1, np.int32),
               pat_colptr=np.zeros(n + 1, np.int32), pat_row=np.zeros(N, np.int32),
               gather=np.zeros(P, np.int32), D=np.zeros(N, np.int32))
    # clique_idx size = sum of clique sizes: get clique_ptr first
    args = [obj] + ([idx] if idx is not None else [])
    _ck(getter(*args, None, _ptr(out["clique_ptr"], C.c_int32), None, None, None, None, None), "get_structure")
    out["clique_idx"] = np.zeros(int(out["clique_ptr"][-1]), np.int32)
    _ck(getter(*args, *[_ptr(out[k], C.c_int32) for k in
                        ("order", "clique_ptr", "clique_idx", "pat_colptr", "pat_row", "gather", "D")]),
        "get_structure")
    return out


def hsde_analyze(problem) -> dict:
    """Host-only symbolic analysis; returns the structure arrays."""
    pv = _ProblemView(problem)
    h = C.c_void_p()
    _ck(lib.hsde_analyze(C.byref(pv.s), C.byref(h)), "hsde_analyze")
    try:
        sz = hsde_sizes()
        _ck(lib.hsde_symbolic_sizes(h, C.byref(sz)), "hsde_symbolic_sizes")
        out = _structure(lib.hsde_symbolic_get, h, None, sz)
        out.update(n=sz.n, p=sz.p, N=sz.N, P=sz.P, n_d=sz.n_d, c_max=sz.c_max)
        return out
    finally:
        lib.hsde_symbolic_free(h)


class Handle:
    """Owns an hsde_handle; methods map one-to-one to the C calls."""

    def __init__(self, problems, options: hsde_options | None = None, **kw):
        if not isinstance(problems, (list, tuple)):
            problems = [problems]
        self.views = [_ProblemView(p) for p in problems]
        arr = (hsde_problem * len(problems))(*[v.s for v in self.views])
        self.opt = options if options is not None else default_options(**kw)
        self.h = C.c_void_p()
        _ck(lib.hsde_setup_batch(arr, len(problems), C.byref(self.opt), C.byref(self.h)), "hsde_setup_batch")
        self.B = len(problems)
        self.sizes = []
        for i in range(self.B):
            sz = hsde_sizes()
            _ck(lib.hsde_get_sizes(self.h, i, C.byref(sz)), "hsde_get_sizes")
            self.sizes.append(sz)

    def close(self):
        if self.h:
            lib.hsde_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- calls ----
    def hsde_iterate(self, k: int, want_status: bool = True):
        st = np.zeros(self.B, np.int32) if want_status else None
        _ck(lib.hsde_iterate(self.h, int(k), _ptr(st, C.c_int32) if st is not None else None), "hsde_iterate")
        return st

    def hsde_sync(self):
        _ck(lib.hsde_sync(self.h), "hsde_sync")

    def hsde_get_info(self, i: int = 0) -> dict:
        inf = hsde_info()
        _ck(lib.hsde_get_info(self.h, i, C.byref(inf)), "hsde_get_info")
        return {k: getattr(inf, k) for k, _ in hsde_info._fields_}

    def hsde_get_structure(self, i: int = 0) -> dict:
        return _structure(lib.hsde_get_structure, self.h, i, self.sizes[i])

    def hsde_get_state(self, i: int = 0) -> np.ndarray:
        out = np.zeros(self.sizes[i].state_len)
        _ck(lib.hsde_get_state(self.h, i, _ptr(out, C.c_double)), "hsde_get_state")
        return out

    def hsde_set_state(self, i: int, state: np.ndarray, iterations: int = 0):
        st = np.ascontiguousarray(state, np.float64)
        assert st.shape[0] == self.sizes[i].state_len
        _ck(lib.hsde_set_state(self.h, i, _ptr(st, C.c_double), int(iterations)), "hsde_set_state")

    def hsde_get_solution(self, i: int = 0):
        sz = self.sizes[i]
        X, y, Z = np.zeros(sz.N), np.zeros(sz.m), np.zeros(sz.N)
        po, do = C.c_double(), C.c_double()
        _ck(lib.hsde_get_solution(self.h, i, _ptr(X, C.c_double), _ptr(y, C.c_double), _ptr(Z, C.c_double),
                                  C.byref(po), C.byref(do)), "hsde_get_solution")
        return X, y, Z, po.value, do.value

    def hsde_get_certificate(self, i: int, kind: int):
        sz = self.sizes[i]
        y, Z, X = np.zeros(sz.m), np.zeros(sz.N), np.zeros(sz.N)
        _ck(lib.hsde_get_certificate(self.h, i, int(kind), _ptr(y, C.c_double), _ptr(Z, C.c_double),
                                     _ptr(X, C.c_double)), "hsde_get_certificate")
        return (y, Z) if kind == PRIMAL_INFEASIBLE else X

    def hsde_get_profile(self) -> dict:
        pr = hsde_profile()
        _ck(lib.hsde_get_profile(self.h, C.byref(pr)), "hsde_get_profile")
        phases = {pr.phase_name[i].value.decode(): (pr.phase_ms[i], int(pr.phase_units[i]))
                  for i in range(pr.nphases)}
        phase_sweeps = {pr.phase_name[i].value.decode(): int(pr.phase_sweeps_max[i])
                        for i in range(pr.nphases) if pr.phase_name[i].value.startswith(b"cone_")}
        phase_variant = {pr.phase_name[i].value.decode(): int(pr.phase_variant[i])
                         for i in range(pr.nphases) if pr.phase_name[i].value.startswith(b"cone_")}
        return dict(kernels_per_iteration=pr.kernels_per_iteration, phases=phases,
                    sweeps_mean=pr.sweeps_mean, sweeps_max=pr.sweeps_max, phase_sweeps_max=phase_sweeps,
                    phase_variant=phase_variant)

    def hsde_set_data(self, i: int, c, b):
        """c, b: NumPy arrays, or ints holding device addresses (both the same kind)."""
        (pc, kc), (pb, kb) = _dptr(c), _dptr(b)
        _ck(lib.hsde_set_data(self.h, i, pc, pb), "hsde_set_data")

    def hsde_unrolled_forward(self, K: int, ckpt: int = 20, x=None, y=None):
        """Returns (x, y, tau, kappa).  x, y: ints holding device addresses to
        write into (then None is returned for them), or None for new NumPy arrays."""
        sz = self.sizes[0]
        xh = np.zeros(sz.N) if x is None else None
        yh = np.zeros(sz.m) if y is None else None
        px = _ptr(xh, C.c_double) if x is None else _dptr(x)[0]
        py = _ptr(yh, C.c_double) if y is None else _dptr(y)[0]
        tau, kappa = C.c_double(), C.c_double()
        _ck(lib.hsde_unrolled_forward(self.h, int(K), int(ckpt), px, py, C.byref(tau), C.byref(kappa)),
            "hsde_unrolled_forward")
        return xh, yh, tau.value, kappa.value

    def hsde_unrolled_backward(self, xbar, ybar, taubar: float, kappabar: float, gC=None, gb=None):
        """Returns (gC, gb).  xbar, ybar: NumPy arrays or device addresses (ints);
        gC, gb: device addresses to write into (None is returned for them) or None."""
        sz = self.sizes[0]
        (pxb, kx), (pyb, ky) = _dptr(xbar, sz.N), _dptr(ybar, sz.m)
        gCh = np.zeros(sz.N) if gC is None else None
        gbh = np.zeros(sz.m) if gb is None else None
        pg = _ptr(gCh, C.c_double) if gC is None else _dptr(gC)[0]
        pgb = _ptr(gbh, C.c_double) if gb is None else _dptr(gb)[0]
        _ck(lib.hsde_unrolled_backward(self.h, pxb, pyb, float(taubar), float(kappabar), pg, pgb),
            "hsde_unrolled_backward")
        return gCh, gbh

    # ---- convenience: run to a verdict in chunks ----
    def solve(self, chunk: int = 20):
        while True:
            st = self.hsde_iterate(chunk)
            if np.all(st != RUNNING):
                return st


def hsde_spd_inverse(S_dev_ptr: int, m: int, stream: int = 0):
    """In-place inverse of an SPD m x m row-major FP64 matrix at a device address."""
    _ck(lib.hsde_spd_inverse(C.c_void_p(S_dev_ptr), int(m), C.c_void_p(stream)), "hsde_spd_inverse")


def split_state(state: np.ndarray, sz: hsde_sizes):
    """Split a state vector into (x, s, y, v, tau, z, kappa)."""
    N, P, m = sz.N, sz.P, sz.m
    o = 0
    x = state[o:o + N]; o += N
    s = state[o:o + P]; o += P
    y = state[o:o + m]; o += m
    v = state[o:o + P]; o += P
    tau = state[o]; o += 1
    z = state[o:o + P]; o += P
    kappa = state[o]
    return x, s, y, v, float(tau), z, float(kappa)
