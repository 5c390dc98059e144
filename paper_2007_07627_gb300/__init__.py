"""Python binding of libfricp, a GB300 (sm_103a) implementation of the per-iteration
hot path of "Fast and Robust Iterative Closest Point" (Zhang, Yao, Deng 2020).

Argument marshalling only: every step of the registration runs in the CUDA
kernels of libfricp.so behind the C ABI of include/fricp.h. Functions carry the
C names without the `fricp_` prefix. Inputs may be numpy float32 arrays (host)
or torch CUDA tensors (device); torch supplies device memory and streams.

There is no CPU fallback: if libfricp.so is missing or cannot be loaded, every
call raises.
"""
from __future__ import annotations

import ctypes
import pathlib

import numpy as np

__all__ = [
    "P2P_AA", "P2P_WELSCH_AA", "P2PL_WELSCH_AA", "VARIANTS", "FricpError", "Params",
    "Result", "lib", "params_default", "Target", "target_create", "register",
    "closest_points", "eval_pass", "target_nu_min", "version", "counters",
]

P2P_AA, P2P_WELSCH_AA, P2PL_WELSCH_AA, P2PL_AA, SYM_WELSCH_AA = 0, 1, 2, 3, 4
VARIANTS = {"p2p": P2P_AA, "p2p_welsch": P2P_WELSCH_AA, "p2pl_welsch": P2PL_WELSCH_AA, "p2pl": P2PL_AA,
            "sym_welsch": SYM_WELSCH_AA}
PREC_FP64, PREC_FP32, PREC_FP16_STORAGE = 0, 1, 2
PRECISIONS = {"fp64": PREC_FP64, "fp32": PREC_FP32, "fp16": PREC_FP16_STORAGE}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EDEGENERATE", 6: "EUNSUPPORTED",
          7: "EBUSY", 8: "EOVERFLOW"}

_PKG = pathlib.Path(__file__).resolve().parent
_LIB_PATH = _PKG / "libfricp.so"


class FricpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("variant", ctypes.c_int32), ("anderson_m", ctypes.c_int32), ("max_iters", ctypes.c_int32),
        ("p2pl_iters_first", ctypes.c_int32), ("p2pl_iters_cap", ctypes.c_int32),
        ("max_line_search", ctypes.c_int32), ("eps", ctypes.c_double), ("nu_max", ctypes.c_double),
        ("nu_min", ctypes.c_double), ("nu_min_floor", ctypes.c_double), ("steps_per_sync", ctypes.c_int32),
        ("use_graph", ctypes.c_int32), ("time_passes", ctypes.c_int32), ("max_steps", ctypes.c_int32),
        ("timeout_s", ctypes.c_double), ("precision", ctypes.c_int32), ("search", ctypes.c_int32),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3), ("status", ctypes.c_int32),
        ("iterations", ctypes.c_int32), ("corr_passes", ctypes.c_int32), ("aa_accepted", ctypes.c_int32),
        ("reverts", ctypes.c_int32), ("line_search_trials", ctypes.c_int32), ("stages", ctypes.c_int32),
        ("device_steps", ctypes.c_int32), ("trace_len", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("nu_max", ctypes.c_double), ("nu_min", ctypes.c_double), ("final_energy", ctypes.c_double),
        ("scale", ctypes.c_double), ("center", ctypes.c_double * 3), ("pass_ms", ctypes.c_double),
        ("wall_ms", ctypes.c_double), ("search_ms", ctypes.c_double),
    ]


class StepRecord(ctypes.Structure):
    """fricp_step_record: one correspondence pass of a recorded registration."""
    _fields_ = [
        ("step", ctypes.c_int32), ("phase", ctypes.c_int32), ("revert", ctypes.c_int32),
        ("accepted", ctypes.c_int32), ("stage", ctypes.c_int32), ("done", ctypes.c_int32),
        ("nu", ctypes.c_double), ("E", ctypes.c_double), ("E_prev", ctypes.c_double),
        ("T", ctypes.c_double * 12), ("xi", ctypes.c_double * 6), ("result", ctypes.c_double * 12),
    ]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libfricp.so (built in-tree by build.build()); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not _LIB_PATH.exists():
        raise FricpError(3, f"{_LIB_PATH} not built: run paper_2007_07627_gb300.build.build()")
    L = ctypes.CDLL(str(_LIB_PATH))
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    L.fricp_params_default.argtypes = [i32, ctypes.POINTER(Params)]
    L.fricp_target_create.argtypes = [vp, vp, i64, i32, vp, ctypes.POINTER(vp)]
    L.fricp_target_destroy.argtypes = [vp]
    L.fricp_target_size.argtypes = [vp]
    L.fricp_target_size.restype = i64
    L.fricp_target_has_normals.argtypes = [vp]
    L.fricp_register.argtypes = [vp, vp, i64, i32, dp, ctypes.POINTER(Params), vp, ctypes.POINTER(Result), dp, i32]
    L.fricp_register_recorded.argtypes = [vp, vp, i64, i32, dp, ctypes.POINTER(Params), vp, ctypes.POINTER(Result),
                                          dp, i32, ctypes.POINTER(StepRecord), i32, ctypes.POINTER(i32)]
    L.fricp_register_symmetric.argtypes = [vp, vp, vp, i64, i32, dp, ctypes.POINTER(Params), vp,
                                           ctypes.POINTER(Result), dp, i32, ctypes.POINTER(StepRecord), i32,
                                           ctypes.POINTER(i32)]
    L.fricp_closest_points.argtypes = [vp, vp, i64, dp, vp, vp, vp]
    L.fricp_eval_pass.argtypes = [vp, vp, i64, i32, i32, dp, dbl, dbl, dp, vp, dp]
    L.fricp_target_nu_min.argtypes = [vp, i32, dbl, vp, dp]
    L.fricp_eval_pass_static.argtypes = [vp, vp, i64, i32, dp, dbl, dbl, dp, vp, dp]
    L.fricp_eval_pass_static.restype = ctypes.c_int
    L.fricp_counters.argtypes = [ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64), i32]
    L.fricp_counters.restype = None
    L.fricp_last_error.restype = ctypes.c_char_p
    L.fricp_last_error.argtypes = []
    L.fricp_version.restype = i32
    pp = ctypes.POINTER(vp)
    L.fricp_batch_register.argtypes = [i32, pp, pp, ctypes.POINTER(i64), i32, dp, ctypes.POINTER(Params), vp,
                                       ctypes.POINTER(Result), dp, i32]
    L.fricp_batch_last_shape.argtypes = [ctypes.POINTER(i32)] * 4
    L.fricp_batch_set_shape.argtypes = [i32, i32, i32]
    L.fricp_estimate_normals.argtypes = [vp, i64, i32, i32, dp, vp, vp]
    L.fricp_server_create.argtypes = [ctypes.c_size_t, i32, i32, i32, vp, ctypes.POINTER(vp)]
    L.fricp_server_submit.argtypes = [vp, vp, vp, i64, i32, dp, ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_uint64)]
    L.fricp_server_step.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.fricp_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(Result), ctypes.POINTER(i32)]
    L.fricp_server_destroy.argtypes = [vp]
    L.fricp_batch_last_shape.restype = None
    for name in ("fricp_params_default", "fricp_target_create", "fricp_target_destroy", "fricp_register",
                 "fricp_register_recorded", "fricp_register_symmetric",
                 "fricp_closest_points", "fricp_eval_pass", "fricp_target_nu_min", "fricp_batch_register",
                 "fricp_server_create", "fricp_server_submit", "fricp_server_step", "fricp_server_poll",
                 "fricp_server_destroy", "fricp_estimate_normals", "fricp_batch_set_shape"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise FricpError(status, lib().fricp_last_error().decode())


def version() -> int:
    return lib().fricp_version()


def counters(reset: bool = False) -> dict:
    """fricp_counters: kernel launches and host<->device bytes of this thread's calls."""
    k, h, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    lib().fricp_counters(ctypes.byref(k), ctypes.byref(h), ctypes.byref(d), int(reset))
    return {"kernel_launches": k.value, "h2d_bytes": h.value, "d2h_bytes": d.value}


def params_default(variant=P2P_WELSCH_AA, **overrides) -> Params:
    if isinstance(variant, str):
        variant = VARIANTS[variant]
    p = Params()
    _check(lib().fricp_params_default(int(variant), ctypes.byref(p)))
    for k, v in overrides.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        setattr(p, k, v)
    return p


def _points(x):
    """(pointer, n, on_device, keepalive) for a float32 [n,3] numpy array or torch CUDA tensor."""
    if x is None:
        return None, 0, 0, None
    if hasattr(x, "is_cuda"):
        import torch
        if x.dtype != torch.float32 or x.dim() != 2 or x.shape[1] != 3:
            raise ValueError("points must be float32 [n, 3]")
        if x.is_cuda:
            x = x.contiguous()
            return ctypes.c_void_p(x.data_ptr()), int(x.shape[0]), 1, x
        x = x.numpy()
    a = np.ascontiguousarray(x, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("points must be float32 [n, 3]")
    return a.ctypes.data_as(ctypes.c_void_p), int(a.shape[0]), 0, a


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _mat(T):
    if T is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(16))
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a


class Target:
    """A target set Q with its device index (fricp_target)."""

    def __init__(self, handle: int, n: int, has_normals: bool):
        self._h = ctypes.c_void_p(handle)
        self.n = n
        self.has_normals = has_normals

    @property
    def handle(self):
        return self._h

    def destroy(self):
        if self._h and self._h.value:
            lib().fricp_target_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def target_create(q, normals=None, stream=None) -> Target:
    qp, n, dev, qk = _points(q)
    npnt, nn, ndev, nk = _points(normals)
    if normals is not None and (nn != n or ndev != dev):
        raise ValueError("normals must match q in size and memory space")
    out = ctypes.c_void_p()
    _check(lib().fricp_target_create(qp, npnt, n, dev, _stream(stream), ctypes.byref(out)))
    return Target(out.value, n, normals is not None)


def _result(r: Result, trace=None) -> dict:
    d = {f: getattr(r, f) for f, _ in Result._fields_ if f not in ("R", "t", "center", "pad0")}
    d["R"] = np.array(r.R[:]).reshape(3, 3)
    d["t"] = np.array(r.t[:])
    d["center"] = np.array(r.center[:])
    d["status"] = STATUS.get(r.status, r.status)
    if trace is not None:
        d["trace"] = trace[: r.trace_len].copy()
    return d


def register(target: Target, p, T0=None, params: Params | None = None, stream=None,
             trace_capacity: int = 0, variant=None) -> dict:
    """fricp_register: Alg. 1 / Alg. 2 of the paper; returns R, t, counters and the energy trace."""
    if params is None:
        params = params_default(variant if variant is not None else P2P_WELSCH_AA)
    pp, m, dev, pk = _points(p)
    Tp, Tk = _mat(T0)
    trace = np.zeros(max(trace_capacity, 0), np.float64)
    tp = trace.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if trace_capacity > 0 else None
    r = Result()
    _check(lib().fricp_register(target.handle, pp, m, dev, Tp, ctypes.byref(params), _stream(stream),
                                ctypes.byref(r), tp, int(trace_capacity)))
    return _result(r, trace if trace_capacity > 0 else None)


def register_recorded(target: Target, p, T0=None, params: Params | None = None, stream=None,
                      trace_capacity: int = 0, steps_capacity: int = 4096, variant=None, source_normals=None):
    """fricp_register_recorded: as register(), plus one record per
    correspondence pass (a list of dicts: step, phase, revert, accepted, stage,
    done, nu, E, E_prev, T (4x4, normalised), xi (6), result (12 or 6)).
    With source_normals (float32 [m,3], p's memory space) it calls
    fricp_register_symmetric (params.variant must be "sym_welsch")."""
    if params is None:
        params = params_default(variant if variant is not None else P2P_WELSCH_AA)
    pp, m, dev, pk = _points(p)
    Tp, Tk = _mat(T0)
    trace = np.zeros(max(trace_capacity, 0), np.float64)
    tp = trace.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if trace_capacity > 0 else None
    r = Result()
    recs = (StepRecord * max(steps_capacity, 1))()
    n = ctypes.c_int32()
    if source_normals is None:
        _check(lib().fricp_register_recorded(target.handle, pp, m, dev, Tp, ctypes.byref(params), _stream(stream),
                                             ctypes.byref(r), tp, int(trace_capacity), recs, int(steps_capacity),
                                             ctypes.byref(n)))
    else:
        npp, nm, ndev, nk = _points(source_normals)
        if nm != m or ndev != dev:
            raise ValueError("source normals must match p in size and memory space")
        _check(lib().fricp_register_symmetric(target.handle, pp, npp, m, dev, Tp, ctypes.byref(params),
                                              _stream(stream), ctypes.byref(r), tp, int(trace_capacity), recs,
                                              int(steps_capacity), ctypes.byref(n)))
    steps = []
    for k in range(n.value):
        x = recs[k]
        T = np.eye(4)
        T[:3, :3] = np.array(x.T[:9]).reshape(3, 3)
        T[:3, 3] = np.array(x.T[9:12])
        steps.append(dict(step=x.step, phase=x.phase, revert=x.revert, accepted=x.accepted, stage=x.stage,
                          done=x.done, nu=x.nu, E=x.E, E_prev=x.E_prev, T=T, xi=np.array(x.xi[:]),
                          result=np.array(x.result[:])))
    return _result(r, trace if trace_capacity > 0 else None), steps


def register_symmetric(target: Target, p, source_normals, T0=None, params: Params | None = None, stream=None,
                       trace_capacity: int = 0) -> dict:
    """fricp_register_symmetric: the Welsch-robust symmetric objective (Sec. 7's
    proposed extension of Alg. 2) with the source's unit normals."""
    if params is None:
        params = params_default(SYM_WELSCH_AA)
    res, _ = register_recorded(target, p, T0=T0, params=params, stream=stream, trace_capacity=trace_capacity,
                               steps_capacity=0, source_normals=source_normals)
    return res


def batch_register(targets, sources, params=None, T0=None, stream=None, trace_capacity: int = 0) -> list:
    """fricp_batch_register: every (target, source) pair registered together; one
    Params per pair (or one for all). Sources are all host arrays or all CUDA
    tensors. Returns one result dict per pair."""
    n = len(targets)
    if len(sources) != n or n == 0:
        raise ValueError("targets and sources must be non-empty and of equal length")
    if params is None:
        params = [params_default()] * n
    elif isinstance(params, Params):
        params = [params] * n
    if len(params) != n:
        raise ValueError("one Params per pair")
    pts = [_points(s) for s in sources]
    devs = {d for _, _, d, _ in pts}
    if len(devs) != 1:
        raise ValueError("sources must all be host arrays or all CUDA tensors")
    tarr = (ctypes.c_void_p * n)(*[t.handle for t in targets])
    parr = (ctypes.c_void_p * n)(*[p[0] for p in pts])
    marr = (ctypes.c_int64 * n)(*[p[1] for p in pts])
    prm = (Params * n)(*params)
    res = (Result * n)()
    Ta = None
    Tp = None
    if T0 is not None:
        Ta = np.ascontiguousarray(np.asarray(T0, dtype=np.float64).reshape(n * 16))
        Tp = Ta.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    trace = np.zeros(n * max(trace_capacity, 0), np.float64)
    tp = trace.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if trace_capacity > 0 else None
    _check(lib().fricp_batch_register(n, tarr, parr, marr, devs.pop(), Tp, prm, _stream(stream), res, tp,
                                      int(trace_capacity)))
    out = []
    for i in range(n):
        tr = trace[i * trace_capacity:(i + 1) * trace_capacity] if trace_capacity > 0 else None
        out.append(_result(res[i], tr))
    return out


def batch_set_shape(chunk: int = 0, search_blocks_per_sm: int = 1, static_order=0) -> None:
    """fricp_batch_set_shape: fix the batched launch shape (chunk = 0: autotune again).
    static_order: 0 counter, 1 fixed stride (True), 2 query tiles."""
    _check(lib().fricp_batch_set_shape(chunk, search_blocks_per_sm, int(static_order)))


def batch_last_shape() -> dict:
    c, a, b, o = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    lib().fricp_batch_last_shape(ctypes.byref(c), ctypes.byref(a), ctypes.byref(b), ctypes.byref(o))
    return {"chunk": c.value, "search_blocks_per_sm": a.value, "accumulate_blocks_per_sm": b.value,
            "static_order": int(o.value)}


def estimate_normals(q, k: int = 30, viewpoint=None, stream=None):
    """fricp_estimate_normals: PCA normals over the k nearest neighbours (Sec. 6).
    Returns float32 [n, 3] in q's memory space (numpy array or CUDA tensor)."""
    qp, n, dev, qk = _points(q)
    if dev:
        import torch
        out = torch.empty((n, 3), dtype=torch.float32, device=qk.device)
        op = ctypes.c_void_p(out.data_ptr())
    else:
        out = np.empty((n, 3), np.float32)
        op = out.ctypes.data_as(ctypes.c_void_p)
    vp = None
    if viewpoint is not None:
        va = np.ascontiguousarray(np.asarray(viewpoint, dtype=np.float64).reshape(3))
        vp = va.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(lib().fricp_estimate_normals(qp, n, int(k), dev, vp, op, _stream(stream)))
    return out


class Server:
    """Serving loop with continuous batching (fricp_server_*)."""

    def __init__(self, hbm_budget: int = 0, max_slots: int = 256, steps_per_sync: int = 16, max_queue: int = 4096,
                 stream=None):
        out = ctypes.c_void_p()
        _check(lib().fricp_server_create(int(hbm_budget), int(max_slots), int(steps_per_sync), int(max_queue),
                                         _stream(stream), ctypes.byref(out)))
        self.handle = out.value

    def submit(self, target: Target, p, params: Params | None = None, T0=None) -> int:
        """Queue a registration; returns its ticket. Raises FricpError (EBUSY) when the queue is full."""
        if params is None:
            params = params_default()
        pp, m, dev, pk = _points(p)
        Tp, Tk = _mat(T0)
        ticket = ctypes.c_uint64()
        _check(lib().fricp_server_submit(self.handle, target.handle, pp, m, dev, Tp, ctypes.byref(params),
                                         ctypes.byref(ticket)))
        return ticket.value

    def step(self, nsteps: int = 16) -> tuple:
        """Advance every request in flight; returns (in_flight, queued)."""
        a, b = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().fricp_server_step(self.handle, int(nsteps), ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def poll(self, ticket: int):
        """The request's result dict once it has finished (returned once), else None."""
        r = Result()
        done = ctypes.c_int32()
        _check(lib().fricp_server_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(r), ctypes.byref(done)))
        return _result(r) if done.value else None

    def destroy(self):
        if self.handle:
            lib().fricp_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def closest_points(target: Target, p, T=None, stream=None):
    """fricp_closest_points on a torch CUDA float32 [m,3] tensor: (idx int64, d2 float64) tensors."""
    import torch
    if not (hasattr(p, "is_cuda") and p.is_cuda):
        raise ValueError("closest_points takes a CUDA tensor")
    p = p.contiguous()
    m = int(p.shape[0])
    idx = torch.empty(m, dtype=torch.int64, device=p.device)
    d2 = torch.empty(m, dtype=torch.float64, device=p.device)
    Tp, Tk = _mat(T)
    _check(lib().fricp_closest_points(target.handle, ctypes.c_void_p(p.data_ptr()), m, Tp,
                                      ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(d2.data_ptr()),
                                      _stream(stream)))
    return idx, d2


def eval_pass(target: Target, p, variant, T_normalized, nu=1.0, scale=1.0, center=None, stream=None):
    """fricp_eval_pass: energy, alignment / Gauss-Newton result and reduced sums of one pass (48 doubles)."""
    if isinstance(variant, str):
        variant = VARIANTS[variant]
    pp, m, dev, pk = _points(p)
    Tp, Tk = _mat(T_normalized)
    c = None
    if center is not None:
        ca = np.ascontiguousarray(np.asarray(center, dtype=np.float64))
        c = ca.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    out = np.zeros(48, np.float64)
    _check(lib().fricp_eval_pass(target.handle, pp, m, dev, int(variant), Tp, float(nu), float(scale), c,
                                 _stream(stream), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def target_nu_min(target: Target, variant, scale=1.0, stream=None) -> float:
    if isinstance(variant, str):
        variant = VARIANTS[variant]
    v = ctypes.c_double()
    _check(lib().fricp_target_nu_min(target.handle, int(variant), float(scale), _stream(stream), ctypes.byref(v)))
    return v.value
