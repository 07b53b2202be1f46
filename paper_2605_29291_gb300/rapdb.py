"""Python binding of the rAPDB C ABI (include/rapdb.h): argument marshalling only.

Every step of the solver runs in the CUDA library ``librapdb.so``; PyTorch
provides device memory and the stream.  There is no CPU fallback: importing
this module fails when the library is missing or cannot be loaded.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, fields

HERE = os.path.dirname(os.path.abspath(__file__))
# RAPDB_LIBRARY selects another build of the library (the checked build in
# the tests); the default is the in-tree librapdb.so
LIB_PATH = os.environ.get("RAPDB_LIBRARY") or os.path.join(HERE, "librapdb.so")

OK, ERR_INVALID, ERR_CUDA, ERR_NOMEM, ERR_BACKTRACK, ERR_MAXITER, ERR_TIMEOUT, ERR_NUMERIC = range(8)
STATUS_NAMES = ["OK", "INVALID", "CUDA", "NOMEM", "BACKTRACK", "MAXITER", "TIMEOUT", "NUMERIC"]
YX, XY = 0, 1
F32, BF16, FP8 = 0, 1, 2
Q0_DENSE, Q0_DIAG, Q0_ZERO = 0, 1, 2
RESTART_NONE, RESTART_FIXED, RESTART_GAP = 0, 1, 2
DUAL_NONNEG, DUAL_SIMPLEX = 0, 1


class CParams(C.Structure):
    _fields_ = [
        ("variant", C.c_int32), ("c_nm", C.c_int32), ("backtracking", C.c_int32), ("restart", C.c_int32),
        ("mu", C.c_double), ("c_alpha", C.c_double), ("c_beta", C.c_double), ("delta", C.c_double),
        ("eta", C.c_double), ("tau_bar", C.c_double), ("gamma0", C.c_double),
        ("restart_period", C.c_int32), ("restart_from_average", C.c_int32),
        ("xi", C.c_double), ("q", C.c_double),
        ("gap_first", C.c_int32), ("gap_every", C.c_int32),
        ("storage", C.c_int32), ("refine", C.c_int32), ("stall_ratio", C.c_double),
        ("max_iter", C.c_int32), ("max_trials", C.c_int32), ("kkt_every", C.c_int32), ("use_graph", C.c_int32),
        ("tol", C.c_double), ("time_limit_s", C.c_double),
        ("rows_per_block", C.c_int32), ("gap_inner_max", C.c_int32), ("pass_variant", C.c_int32),
        ("dual_set", C.c_int32), ("dual_radius", C.c_double), ("restart_warm_tau", C.c_int32),
        ("pack_sym", C.c_int32),
    ]


class CExtras(C.Structure):
    _fields_ = [("p_eq", C.c_int64), ("A_eq", C.c_void_p), ("b_eq", C.c_void_p), ("x_hyp_a", C.c_void_p),
                ("x_hyp_beta", C.c_double)]


class CInfo(C.Structure):
    _fields_ = [
        ("iters", C.c_int32), ("trials", C.c_int32), ("restarts", C.c_int32), ("precision_switches", C.c_int32),
        ("passes", C.c_int32), ("status", C.c_int32),
        ("rel_kkt", C.c_double), ("r_stat", C.c_double), ("r_feas", C.c_double),
        ("obj", C.c_double), ("seconds", C.c_double), ("launches", C.c_int64),
        ("switch_iter", C.c_int32), ("reserved_", C.c_int32),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"the rAPDB library is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    P, I, vp = C.POINTER(CParams), C.POINTER(CInfo), C.c_void_p
    ctxpp = C.POINTER(vp)
    sig = {
        "rapdb_default_params": (None, [P, C.c_int32]),
        "rapdb_create": (C.c_int, [ctxpp, C.c_int64, C.c_int64, C.c_int32, vp, vp, vp, vp, vp, vp, P, vp]),
        "rapdb_create_eq": (C.c_int, [ctxpp, C.c_int64, C.c_int64, C.c_int32, vp, vp, vp, vp, vp, vp, C.c_int64,
                                      vp, vp, P, vp]),
        "rapdb_create_ex": (C.c_int, [ctxpp, C.c_int64, C.c_int64, C.c_int32, vp, vp, vp, vp, vp, vp,
                                      C.POINTER(CExtras), P, vp]),
        "rapdb_solve": (C.c_int, [vp, vp, vp, I]),
        "rapdb_kkt_residual": (C.c_int, [vp, vp, vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                         C.POINTER(C.c_double)]),
        "rapdb_coupling_pass": (C.c_int, [vp, vp, vp, vp, vp, vp, vp]),
        "rapdb_packed_pass": (C.c_int, [vp, vp, vp, vp, vp, vp, vp]),
        "rapdb_set_log": (C.c_int, [vp, C.c_int32, vp, vp, vp, vp, vp, vp, vp, vp]),
        "rapdb_create_batched": (C.c_int, [ctxpp, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                           C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                           C.POINTER(vp), P, vp]),
        "rapdb_solve_batched": (C.c_int, [vp, C.POINTER(vp), C.POINTER(vp), I]),
        "rapdb_get_state": (C.c_int, [vp, vp, C.POINTER(C.c_size_t)]),
        "rapdb_set_state": (C.c_int, [vp, vp, C.c_size_t]),
        "rapdb_resume": (C.c_int, [vp, vp, vp, I]),
        "rapdb_get_tile": (C.c_int, [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int32)]),
        "rapdb_get_instance_tile": (C.c_int, [vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "rapdb_time_pass": (C.c_int, [vp, C.c_int32, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
        "rapdb_get_solution_f64": (C.c_int, [vp, vp, vp]),
        "rapdb_coupling_pass_noalloc": (C.c_int, [C.c_int64, C.c_int64, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "rapdb_wait_selftest": (C.c_int, [C.c_int32, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                          C.POINTER(C.c_float)]),
        "rapdb_last_error": (C.c_char_p, [vp]),
        "rapdb_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class RapdbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"rapdb status {STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


@dataclass
class Params:
    """Mirror of rapdb_params; defaults are the library's (the paper's settings)."""
    variant: int = YX
    c_nm: int = 1
    backtracking: int = 1
    restart: int = RESTART_FIXED
    mu: float = 0.0
    c_alpha: float = 0.4
    c_beta: float = 0.0
    delta: float = 0.5
    eta: float = 0.7
    tau_bar: float = 1.0
    gamma0: float = 1.0
    restart_period: int = 200
    restart_from_average: int = 0
    xi: float = 0.04
    q: float = 0.5
    gap_first: int = 50
    gap_every: int = 500
    storage: int = F32
    refine: int = 1
    stall_ratio: float = 0.5
    max_iter: int = 50000
    max_trials: int = 60
    kkt_every: int = 1
    use_graph: int = 1
    tol: float = 1e-6
    time_limit_s: float = 0.0
    rows_per_block: int = 0
    gap_inner_max: int = 200
    pass_variant: int = 0
    dual_set: int = 0
    dual_radius: float = 1.0
    restart_warm_tau: int = 0
    pack_sym: int = 0

    @classmethod
    def default(cls, variant: int = YX, **kw) -> "Params":
        cp = CParams()
        lib.rapdb_default_params(C.byref(cp), variant)
        p = cls(**{f.name: getattr(cp, f.name) for f in fields(cls)})
        for k, v in kw.items():
            if not hasattr(p, k):
                raise AttributeError(k)
            setattr(p, k, v)
        return p

    def to_c(self) -> CParams:
        cp = CParams()
        for f in fields(self):
            setattr(cp, f.name, getattr(self, f.name))
        return cp


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _stream_handle(device):
    import torch
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _info_dict(ci: CInfo) -> dict:
    return {f[0]: getattr(ci, f[0]) for f in CInfo._fields_ if not f[0].endswith("_")}


def _check(st, ctx=None):
    if st != OK:
        msg = lib.rapdb_last_error(ctx)
        raise RapdbError(st, msg.decode() if msg else "")


class Solver:
    """One QCQP on one GPU.  ``data`` holds torch CUDA float32 tensors with the
    layout of rapdb_create (see workloads.QCQPData).  The tensors passed in
    must stay alive while the solver exists (float32 Q may be borrowed)."""

    def __init__(self, data, params: Params | None = None):
        import torch
        self.params = params or Params.default()
        A_eq, b_eq = getattr(data, "A_eq", None), getattr(data, "b_eq", None)
        hyp_a = getattr(data, "hyp_a", None)
        self.p_eq = 0 if A_eq is None else int(A_eq.shape[0])
        # m counts the equalities too: the dual vector has m entries, the
        # equality multipliers last
        self.n, self.m = int(data.n), int(data.m) + self.p_eq
        self._keep = [data.Q, data.c, data.d, data.lb, data.ub, data.q0diag, A_eq, b_eq, hyp_a]
        for t in self._keep:
            if t is not None:
                assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
        self.device = data.Q.device
        self.ctx = C.c_void_p()
        cp = self.params.to_c()
        ex = CExtras(self.p_eq, _ptr(A_eq), _ptr(b_eq), _ptr(hyp_a), float(getattr(data, "hyp_beta", 0.0)))
        st = lib.rapdb_create_ex(C.byref(self.ctx), self.n, int(data.m), int(data.q0_kind), _ptr(data.Q),
                                 _ptr(data.q0diag), _ptr(data.c), _ptr(data.d), _ptr(data.lb), _ptr(data.ub),
                                 C.byref(ex), C.byref(cp), _stream_handle(self.device))
        _check(st, None)
        self._log = None

    def close(self):
        if self.ctx:
            lib.rapdb_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, x, y, check: bool = True) -> dict:
        """Run rAPDB from (x, y) (CUDA float32, overwritten with the result)."""
        ci = CInfo()
        st = lib.rapdb_solve(self.ctx, _ptr(x), _ptr(y), C.byref(ci))
        if check and st not in (OK, ERR_MAXITER, ERR_BACKTRACK, ERR_TIMEOUT, ERR_NUMERIC):
            _check(st, self.ctx)
        return _info_dict(ci)

    def resume(self, x, y) -> dict:
        ci = CInfo()
        st = lib.rapdb_resume(self.ctx, _ptr(x), _ptr(y), C.byref(ci))
        if st not in (OK, ERR_MAXITER, ERR_BACKTRACK, ERR_TIMEOUT, ERR_NUMERIC):
            _check(st, self.ctx)
        return _info_dict(ci)

    def kkt_residual(self, x, y):
        rel, rs, rf = C.c_double(), C.c_double(), C.c_double()
        _check(lib.rapdb_kkt_residual(self.ctx, _ptr(x), _ptr(y), C.byref(rel), C.byref(rs), C.byref(rf)),
               self.ctx)
        return rel.value, rs.value, rf.value

    def coupling_pass(self, x, v, uold=None):
        """U[i] = Q_i x, W[i] = Q_i v and the (m+1, 5) float64 dots."""
        import torch
        U = torch.empty((self.m + 1, self.n), dtype=torch.float32, device=self.device)
        W = torch.empty_like(U)
        dots = torch.empty((self.m + 1, 5), dtype=torch.float64, device=self.device)
        _check(lib.rapdb_coupling_pass(self.ctx, _ptr(x), _ptr(v), _ptr(uold), _ptr(U), _ptr(W), _ptr(dots)),
               self.ctx)
        return U, W, dots

    def packed_pass(self, x, v, uold):
        """The packed incremental pass of a pack_sym context for the M stored
        matrices: W[s] = Q_i v, U[s] = uold[s] + W[s] and the (M, 5) float64
        dots (x'U, v'W, v'uold, c'x, c'v)."""
        import torch
        M = int(uold.shape[0])
        U = torch.empty((M, self.n), dtype=torch.float32, device=self.device)
        W = torch.empty_like(U)
        dots = torch.empty((M, 5), dtype=torch.float64, device=self.device)
        _check(lib.rapdb_packed_pass(self.ctx, _ptr(x), _ptr(v), _ptr(uold), _ptr(U), _ptr(W), _ptr(dots)),
               self.ctx)
        return U, W, dots

    def set_log(self, capacity: int, iterates: bool = True):
        """Record tau_k, trials, KKT residuals, smoothed gaps, f(x^{k+1}) and
        the mean constraint violation of the first `capacity` iterations, and
        (optionally) the iterates."""
        import torch
        dev = self.device
        if capacity <= 0:
            _check(lib.rapdb_set_log(self.ctx, 0, None, None, None, None, None, None, None, None), self.ctx)
            self._log = None
            return
        tau = torch.full((capacity,), float("nan"), dtype=torch.float64, device=dev)
        tr = torch.zeros((capacity,), dtype=torch.int32, device=dev)
        xl = torch.full((capacity, self.n), float("nan"), dtype=torch.float32, device=dev) if iterates else None
        yl = (torch.full((capacity, max(self.m, 1)), float("nan"), dtype=torch.float32, device=dev)
              if iterates else None)
        kk = torch.full((capacity,), float("nan"), dtype=torch.float64, device=dev)
        gp = torch.full((capacity,), float("nan"), dtype=torch.float64, device=dev)
        ob = torch.full((capacity,), float("nan"), dtype=torch.float64, device=dev)
        inf = torch.full((capacity,), float("nan"), dtype=torch.float64, device=dev)
        _check(lib.rapdb_set_log(self.ctx, capacity, _ptr(tau), _ptr(tr), _ptr(xl), _ptr(yl), _ptr(kk), _ptr(gp),
                                 _ptr(ob), _ptr(inf)), self.ctx)
        self._log = dict(tau=tau, trials=tr, x=xl, y=yl, kkt=kk, gap=gp, obj=ob, infeas=inf)

    @property
    def log(self):
        return self._log

    def get_state(self) -> bytes:
        n = C.c_size_t()
        _check(lib.rapdb_get_state(self.ctx, None, C.byref(n)), self.ctx)
        buf = C.create_string_buffer(n.value)
        _check(lib.rapdb_get_state(self.ctx, buf, C.byref(n)), self.ctx)
        return buf.raw

    def set_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        _check(lib.rapdb_set_state(self.ctx, buf, len(blob)), self.ctx)

    def solution_f64(self):
        """The solver's float64 iterate (x, y) of the last solve."""
        import torch
        x = torch.empty(self.n, dtype=torch.float64, device=self.device)
        y = torch.empty(max(self.m, 1), dtype=torch.float64, device=self.device)
        _check(lib.rapdb_get_solution_f64(self.ctx, _ptr(x), _ptr(y)), self.ctx)
        return x, y[:self.m]

    def time_pass(self, reps: int = 20, level: int = -1):
        """(average ms per coupling-pass launch, algorithmic bytes per pass) at a
        precision level (-1: where the last solve ended, 0 stored Q, 1 float32 Q,
        2 compensated float32 products, 3 their incremental form, 4 the
        incremental form through the packed tiles of a pack_sym context)."""
        ms, b = C.c_double(), C.c_int64()
        _check(lib.rapdb_time_pass(self.ctx, reps, level, C.byref(ms), C.byref(b)), self.ctx)
        return ms.value, b.value

    def tile(self) -> dict:
        rb, ctas, rpw, unr = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        lib.rapdb_get_tile(self.ctx, C.byref(rb), C.byref(ctas), C.byref(rpw), C.byref(unr))
        return {"rows_per_block": rb.value, "ctas": ctas.value, "rows_per_warp": rpw.value,
                "chunks_in_flight": unr.value}


def coupling_pass_noalloc(Q, c, x, v, uold=None, U=None, W=None, dots=None):
    """The context-free coupling pass that allocates no device memory in the
    library (see rapdb_coupling_pass_noalloc in include/rapdb.h).  Q is the
    (m+1, n, n) float32 stack; the outputs may be passed in preallocated."""
    import torch
    M, n = int(Q.shape[0]), int(Q.shape[1])
    if U is None:
        U = torch.empty((M, n), dtype=torch.float32, device=Q.device)
    if W is None:
        W = torch.empty((M, n), dtype=torch.float32, device=Q.device)
    if dots is None:
        dots = torch.empty((M, 5), dtype=torch.float64, device=Q.device)
    st = lib.rapdb_coupling_pass_noalloc(n, M - 1, _ptr(Q), _ptr(c), _ptr(x), _ptr(v), _ptr(uold), _ptr(U),
                                         _ptr(W), _ptr(dots), _stream_handle(Q.device))
    if st != OK:
        raise RapdbError(st, "rapdb_coupling_pass_noalloc rejected the call (sizes, alignment or scratch limit)")
    return U, W, dots


def wait_selftest(complete: bool, limit_us: int = 50000) -> dict:
    """Run the bounded-wait self-test on the current device (see
    rapdb_wait_selftest in include/rapdb.h): returns whether the wait gave
    up, how long it waited (ms) and the sum of the copied floats."""
    g, ms, sm = C.c_int32(0), C.c_double(0.0), C.c_float(0.0)
    st = lib.rapdb_wait_selftest(1 if complete else 0, int(limit_us), C.byref(g), C.byref(ms), C.byref(sm))
    if st != OK:
        raise RapdbError(st, "rapdb_wait_selftest failed")
    return {"gave_up": bool(g.value), "waited_ms": ms.value, "copied_sum": sm.value}


class BatchedSolver:
    """Many independent QCQPs (dense Q_0, float32) solved in one device loop."""

    def __init__(self, datas, params: Params | None = None):
        self.params = params or Params.default()
        self.B = len(datas)
        self._keep = [[d.Q, d.c, d.d, d.lb, d.ub] for d in datas]
        self.ns = [int(d.n) for d in datas]
        self.ms = [int(d.m) for d in datas]
        self.device = datas[0].Q.device
        arr = lambda ts: (C.c_void_p * self.B)(*[t.data_ptr() for t in ts])
        n = (C.c_int64 * self.B)(*self.ns)
        m = (C.c_int64 * self.B)(*self.ms)
        self.ctx = C.c_void_p()
        cp = self.params.to_c()
        st = lib.rapdb_create_batched(C.byref(self.ctx), self.B, n, m, arr([d.Q for d in datas]),
                                      arr([d.c for d in datas]), arr([d.d for d in datas]),
                                      arr([d.lb for d in datas]), arr([d.ub for d in datas]), C.byref(cp),
                                      _stream_handle(self.device))
        _check(st, None)

    def close(self):
        if self.ctx:
            lib.rapdb_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tile(self, b: int) -> dict:
        """Instance b's rows per block and the batch's tile variant."""
        rb, vi = C.c_int32(0), C.c_int32(0)
        _check(lib.rapdb_get_instance_tile(self.ctx, int(b), C.byref(rb), C.byref(vi)), self.ctx)
        return {"rows_per_block": rb.value, "variant": vi.value}

    def solve(self, xs, ys) -> list:
        infos = (CInfo * self.B)()
        xa = (C.c_void_p * self.B)(*[t.data_ptr() for t in xs])
        ya = (C.c_void_p * self.B)(*[t.data_ptr() for t in ys])
        st = lib.rapdb_solve_batched(self.ctx, xa, ya, infos)
        if st not in (OK, ERR_MAXITER, ERR_BACKTRACK, ERR_TIMEOUT, ERR_NUMERIC):
            _check(st, self.ctx)
        return [_info_dict(infos[b]) for b in range(self.B)]
