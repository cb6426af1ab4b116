"""Python binding of the C ABI in ``include/ots.h`` (argument marshalling only).

Every function here has the name of the C entry point it wraps and does nothing but convert
numpy arrays and option values into the C structures and back; every step of the solver
runs in ``libots.so``.  The library must be built (``paper_2106_14485_gb300.build.build()``):
there is no fallback, and a missing library raises at load time.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libots.so")

OTS_OK, OTS_ERR_INVALID_ARG, OTS_ERR_INFEASIBLE, OTS_ERR_NOT_CONVERGED = 0, 1, 2, 3
OTS_ERR_TIMEOUT, OTS_ERR_OOM, OTS_ERR_CUDA, OTS_ERR_NUMERIC = 4, 5, 6, 7
OTS_PENDING = 8
OTS_ERR_DEVICE_WAIT = 9

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class ProblemDesc(ctypes.Structure):
    _fields_ = [
        ("n_nodes", ctypes.c_int32), ("n_edges", ctypes.c_int32),
        ("edge_src", _i32p), ("edge_dst", _i32p), ("edge_cost", _f64p), ("edge_capacity", _f64p),
        ("add_wait_loops", ctypes.c_int32),
        ("wait_cost", _f64p), ("wait_capacity", _f64p), ("commodity_cost", _f64p),
        ("T", ctypes.c_int32), ("L", ctypes.c_int32), ("eps", ctypes.c_double),
        ("n_sources", ctypes.c_int32), ("src_commodity", _i32p), ("src_state", _i32p), ("src_mass", _f64p),
        ("n_sinks", ctypes.c_int32), ("snk_commodity", _i32p), ("snk_state", _i32p), ("snk_mass", _f64p),
        ("device", ctypes.c_int32), ("stream", ctypes.c_void_p),
        ("alloc", ALLOC_FN), ("free_fn", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
        ("state_cost_t", _f64p),
        ("state_capacity_t", _f64p),
        ("psi_stride", ctypes.c_int32),
        ("commodity_t_in", _i32p), ("commodity_t_out", _i32p),
        ("commodity_capacity", _f64p),
        ("state_tail", _i32p), ("state_head", _i32p), ("state_hold", _i32p),
    ]


class ProblemStats(ctypes.Structure):
    _fields_ = [("n_states", ctypes.c_int32), ("n_nodes", ctypes.c_int32), ("T", ctypes.c_int32),
                ("L", ctypes.c_int32), ("padded_L", ctypes.c_int32), ("threads_per_node", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("kernels_per_pass", ctypes.c_int64),
                ("kernels_launched", ctypes.c_int64), ("passes_total", ctypes.c_int64),
                ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iters", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("timeout_ms", ctypes.c_double), ("warm_start", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("threads_per_node", ctypes.c_int32), ("eps_stages", ctypes.c_int32),
                ("eps_start", ctypes.c_double), ("eps_stage_tol", ctypes.c_double)]


class SolveReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("src_residual", ctypes.c_double),
                ("cap_violation", ctypes.c_double), ("dual_objective", ctypes.c_double),
                ("seconds", ctypes.c_double), ("status", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class LinearStats(ctypes.Structure):
    _fields_ = [("linear_passes", ctypes.c_int32), ("log_passes", ctypes.c_int32), ("rescalings", ctypes.c_int32),
                ("confirm_passes", ctypes.c_int32), ("kernel_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchDesc(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("stream", ctypes.c_void_p), ("pool_bytes", ctypes.c_int64),
                ("max_instances", ctypes.c_int32), ("max_items", ctypes.c_int32),
                ("ticks_per_launch", ctypes.c_int32),
                ("alloc", ALLOC_FN), ("free_fn", FREE_FN), ("alloc_ctx", ctypes.c_void_p)]


class BatchStats(ctypes.Structure):
    _fields_ = [("resident", ctypes.c_int32), ("running", ctypes.c_int32), ("pool_bytes", ctypes.c_int64),
                ("pool_used", ctypes.c_int64), ("launches", ctypes.c_int64), ("ticks", ctypes.c_int64),
                ("items", ctypes.c_int64), ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64)]


class ServerDesc(ctypes.Structure):
    _fields_ = [("batch", BatchDesc), ("builder_threads", ctypes.c_int32), ("max_queued", ctypes.c_int32),
                ("mode", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("queued", ctypes.c_int32), ("building", ctypes.c_int32), ("resident", ctypes.c_int32),
                ("large_running", ctypes.c_int32), ("pool_bytes", ctypes.c_int64), ("pool_used", ctypes.c_int64),
                ("batch_launches", ctypes.c_int64), ("batch_ticks", ctypes.c_int64)]


EXPORTED = ["ots_default_solve_opts", "ots_create_problem", "ots_check_problem", "ots_sinkhorn_solve", "ots_iterate", "ots_get_flows",
            "ots_get_commodity_flows", "ots_get_commodity_flows_noalloc", "ots_get_duals", "ots_set_duals", "ots_problem_info", "ots_last_pass_timing",
            "ots_set_wait_limit", "ots_linear_iterate", "ots_linear_solve", "ots_linear_solve_many", "ots_problem_stream", "ots_destroy_problem", "ots_status_string", "ots_last_error",
            "ots_default_batch_desc", "ots_batch_create", "ots_batch_add", "ots_batch_run", "ots_batch_status",
            "ots_batch_get_flows", "ots_batch_get_duals", "ots_batch_remove", "ots_batch_info", "ots_batch_mapping",
            "ots_batch_autotune", "ots_batch_destroy",
            "ots_default_server_desc", "ots_server_create", "ots_server_submit", "ots_server_poll", "ots_server_wait",
            "ots_server_get_flows", "ots_server_timing", "ots_server_release", "ots_server_info", "ots_server_destroy"]

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libots.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2106_14485_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.ots_default_solve_opts.argtypes = [ctypes.POINTER(SolveOpts)]
    lib.ots_create_problem.argtypes = [ctypes.POINTER(ProblemDesc), ctypes.POINTER(P)]
    lib.ots_check_problem.argtypes = [ctypes.POINTER(ProblemDesc)]
    lib.ots_sinkhorn_solve.argtypes = [P, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveReport)]
    lib.ots_iterate.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(SolveReport)]
    lib.ots_get_flows.argtypes = [P, ctypes.c_int32, ctypes.c_int32, _f64p]
    lib.ots_get_commodity_flows.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _f64p]
    lib.ots_get_commodity_flows_noalloc.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                    ctypes.c_int32, _f64p]
    lib.ots_get_duals.argtypes = [P, _f64p, _f64p, _f64p]
    lib.ots_set_duals.argtypes = [P, _f64p, _f64p, _f64p]
    lib.ots_set_wait_limit.argtypes = [P, ctypes.c_int32, ctypes.c_int32]
    lib.ots_linear_iterate.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(SolveReport),
                                       ctypes.POINTER(LinearStats)]
    lib.ots_linear_solve.argtypes = [P, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveReport),
                                     ctypes.POINTER(LinearStats)]
    lib.ots_linear_solve_many.argtypes = [ctypes.POINTER(P), ctypes.c_int32, ctypes.POINTER(SolveOpts),
                                          ctypes.POINTER(SolveReport), ctypes.POINTER(LinearStats)]
    lib.ots_problem_info.argtypes = [P, ctypes.POINTER(ProblemStats)]
    lib.ots_last_pass_timing.argtypes = [P, _f64p]
    lib.ots_problem_stream.argtypes = [P]
    lib.ots_problem_stream.restype = ctypes.c_void_p
    lib.ots_destroy_problem.argtypes = [P]
    lib.ots_destroy_problem.restype = None
    lib.ots_status_string.argtypes = [ctypes.c_int]
    lib.ots_status_string.restype = ctypes.c_char_p
    lib.ots_last_error.argtypes = []
    lib.ots_last_error.restype = ctypes.c_char_p
    lib.ots_default_batch_desc.argtypes = [ctypes.POINTER(BatchDesc)]
    lib.ots_batch_create.argtypes = [ctypes.POINTER(BatchDesc), ctypes.POINTER(P)]
    lib.ots_batch_add.argtypes = [P, ctypes.POINTER(ProblemDesc), ctypes.POINTER(SolveOpts), _i32p]
    lib.ots_batch_run.argtypes = [P, ctypes.c_int32, _i32p]
    lib.ots_batch_status.argtypes = [P, ctypes.c_int32, ctypes.POINTER(SolveReport)]
    lib.ots_batch_get_flows.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _f64p]
    lib.ots_batch_get_duals.argtypes = [P, ctypes.c_int32, _f64p, _f64p, _f64p]
    lib.ots_batch_remove.argtypes = [P, ctypes.c_int32]
    lib.ots_batch_info.argtypes = [P, ctypes.POINTER(BatchStats)]
    lib.ots_batch_mapping.argtypes = [P, ctypes.c_int32, _i32p, _i32p]
    lib.ots_batch_autotune.argtypes = [P, ctypes.c_char_p]
    lib.ots_batch_destroy.argtypes = [P]
    lib.ots_batch_destroy.restype = None
    lib.ots_default_server_desc.argtypes = [ctypes.POINTER(ServerDesc)]
    lib.ots_server_create.argtypes = [ctypes.POINTER(ServerDesc), ctypes.POINTER(P)]
    lib.ots_server_submit.argtypes = [P, ctypes.POINTER(ProblemDesc), ctypes.POINTER(SolveOpts),
                                      ctypes.POINTER(ctypes.c_int64)]
    lib.ots_server_poll.argtypes = [P, ctypes.c_int64, ctypes.POINTER(SolveReport)]
    lib.ots_server_wait.argtypes = [P, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(SolveReport)]
    lib.ots_server_get_flows.argtypes = [P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _f64p]
    lib.ots_server_timing.argtypes = [P, ctypes.c_int64, _f64p]
    lib.ots_server_release.argtypes = [P, ctypes.c_int64]
    lib.ots_server_info.argtypes = [P, ctypes.POINTER(ServerStats)]
    lib.ots_server_destroy.argtypes = [P]
    lib.ots_server_destroy.restype = None
    for name in ("ots_default_server_desc", "ots_server_create", "ots_server_submit", "ots_server_poll",
                 "ots_server_wait", "ots_server_get_flows", "ots_server_timing", "ots_server_release",
                 "ots_server_info"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("ots_default_batch_desc", "ots_batch_create", "ots_batch_add", "ots_batch_run", "ots_batch_status",
                 "ots_batch_get_flows", "ots_batch_get_duals", "ots_batch_remove", "ots_batch_info",
                 "ots_batch_mapping", "ots_batch_autotune"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("ots_default_solve_opts", "ots_create_problem", "ots_sinkhorn_solve", "ots_iterate",
                 "ots_get_flows", "ots_get_commodity_flows", "ots_get_commodity_flows_noalloc", "ots_get_duals", "ots_set_duals", "ots_problem_info",
                 "ots_last_pass_timing", "ots_set_wait_limit"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class OTSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ots_status_string(code)}: {msg}")
        self.code = code


def _check(code: int) -> int:
    if code != OTS_OK:
        raise OTSError(code, load_library().ots_last_error().decode())
    return code


def ots_status_string(code: int) -> str:
    return load_library().ots_status_string(int(code)).decode()


def _ptr(a, ct):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ct))


class Handle:
    """Owns an ``ots_problem*`` plus the host arrays and callbacks it was created from."""

    def __init__(self, ptr, keep, n_states, T, L, n_sources, n_sinks):
        self.ptr = ptr
        self._keep = keep
        self.n_states, self.T, self.L = n_states, T, L
        self.n_sources, self.n_sinks = n_sources, n_sinks

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                ots_destroy_problem(self)
            except Exception:
                pass


def _torch_allocator(device: int):
    import torch
    live = {}

    def alloc(nbytes, ctx):
        try:
            ptr = torch.cuda.caching_allocator_alloc(int(nbytes), device=device)
        except Exception:
            return None
        live[ptr] = nbytes
        return ptr

    def free(ptr, ctx):
        if ptr in live:
            del live[ptr]
            torch.cuda.caching_allocator_delete(ptr)

    return ALLOC_FN(alloc), FREE_FN(free)


def _problem_desc(inst, device: int = 0, stream: int | None = None):
    """ots_problem_desc of an object with the attributes of ``instances.Instance`` plus the
    host arrays it points into (keep them alive while the descriptor is used)."""
    c = lambda x, dt: np.ascontiguousarray(x, dtype=dt)
    arr = {
        "edge_src": c(inst.edge_src, np.int32), "edge_dst": c(inst.edge_dst, np.int32),
        "edge_cost": c(inst.edge_cost, np.float64), "edge_cap": c(inst.edge_cap, np.float64),
        "wait_cost": c(inst.wait_cost, np.float64), "wait_cap": c(inst.wait_cap, np.float64),
        "src_comm": c(inst.src_comm, np.int32), "src_state": c(inst.src_state, np.int32),
        "src_mass": c(inst.src_mass, np.float64), "snk_comm": c(inst.snk_comm, np.int32),
        "snk_state": c(inst.snk_state, np.int32), "snk_mass": c(inst.snk_mass, np.float64),
    }
    cc = getattr(inst, "commodity_cost", None)
    if cc is not None:
        arr["commodity_cost"] = c(cc, np.float64)
    ct = getattr(inst, "state_cost_t", None)
    if ct is not None:
        arr["state_cost_t"] = c(ct, np.float64)
    dt = getattr(inst, "state_capacity_t", None)
    if dt is not None:
        arr["state_capacity_t"] = c(dt, np.float64)
    ccap = getattr(inst, "commodity_capacity", None)
    if ccap is not None:
        arr["commodity_capacity"] = c(ccap, np.float64)
    for k in ("commodity_t_in", "commodity_t_out", "state_tail", "state_head", "state_hold"):
        w = getattr(inst, k, None)
        if w is not None:
            arr[k] = c(w, np.int32)
    d = ProblemDesc()
    d.n_nodes, d.n_edges = int(inst.n_nodes), int(len(arr["edge_src"]))
    d.edge_src, d.edge_dst = _ptr(arr["edge_src"], ctypes.c_int32), _ptr(arr["edge_dst"], ctypes.c_int32)
    d.edge_cost, d.edge_capacity = _ptr(arr["edge_cost"], ctypes.c_double), _ptr(arr["edge_cap"], ctypes.c_double)
    d.add_wait_loops = 1
    d.wait_cost, d.wait_capacity = _ptr(arr["wait_cost"], ctypes.c_double), _ptr(arr["wait_cap"], ctypes.c_double)
    d.commodity_cost = _ptr(arr.get("commodity_cost"), ctypes.c_double)
    d.state_cost_t = _ptr(arr.get("state_cost_t"), ctypes.c_double)
    d.state_capacity_t = _ptr(arr.get("state_capacity_t"), ctypes.c_double)
    d.commodity_t_in = _ptr(arr.get("commodity_t_in"), ctypes.c_int32)
    d.commodity_t_out = _ptr(arr.get("commodity_t_out"), ctypes.c_int32)
    d.commodity_capacity = _ptr(arr.get("commodity_capacity"), ctypes.c_double)
    d.state_tail = _ptr(arr.get("state_tail"), ctypes.c_int32)
    d.state_head = _ptr(arr.get("state_head"), ctypes.c_int32)
    d.state_hold = _ptr(arr.get("state_hold"), ctypes.c_int32)
    d.T, d.L, d.eps = int(inst.T), int(inst.L), float(inst.eps)
    d.n_sources = len(arr["src_comm"])
    d.src_commodity, d.src_state = _ptr(arr["src_comm"], ctypes.c_int32), _ptr(arr["src_state"], ctypes.c_int32)
    d.src_mass = _ptr(arr["src_mass"], ctypes.c_double)
    d.n_sinks = len(arr["snk_comm"])
    d.snk_commodity, d.snk_state = _ptr(arr["snk_comm"], ctypes.c_int32), _ptr(arr["snk_state"], ctypes.c_int32)
    d.snk_mass = _ptr(arr["snk_mass"], ctypes.c_double)
    d.device = int(device)
    d.stream = stream
    return d, arr


def ots_create_problem(inst, device: int = 0, stream: int | None = None, allocator: str = "torch",
                       psi_stride: int = 0) -> Handle:
    """Create a problem from an object with the attributes of ``instances.Instance``.

    allocator: "torch" (PyTorch caching allocator) or "cuda" (cudaMalloc inside the library);
    psi_stride: keep the backward messages every psi_stride-th t only (0 = all)."""
    lib = load_library()
    d, arr = _problem_desc(inst, device, stream)
    d.psi_stride = int(psi_stride)
    keep = [arr]
    if allocator == "torch":
        a, f = _torch_allocator(int(device))
        d.alloc, d.free_fn = a, f
        keep.append((a, f))
    elif allocator != "cuda":
        raise ValueError("allocator must be 'torch' or 'cuda'")
    out = ctypes.c_void_p()
    _check(lib.ots_create_problem(ctypes.byref(d), ctypes.byref(out)))
    S = int(inst.n_nodes) + d.n_edges
    return Handle(out, keep, S, d.T, d.L, d.n_sources, d.n_sinks)


def ots_check_problem(inst) -> None:
    """The host-side checks of ots_create_problem (no device needed); raises OTSError."""
    d, arr = _problem_desc(inst, 0, None)
    _check(load_library().ots_check_problem(ctypes.byref(d)))


def ots_default_solve_opts() -> SolveOpts:
    o = SolveOpts()
    _check(load_library().ots_default_solve_opts(ctypes.byref(o)))
    return o


def ots_sinkhorn_solve(h: Handle, tol: float = 1e-6, max_iters: int = 100000, check_every: int = 10,
                       timeout_ms: float = 0.0, warm_start: bool = False, use_graph: bool = True,
                       threads_per_node: int = 0, raise_on_error: bool = True, eps_start: float = 0.0,
                       eps_stages: int = 0, eps_stage_tol: float = 0.0) -> dict:
    o = ots_default_solve_opts()
    o.tol, o.max_iters, o.check_every, o.timeout_ms = tol, max_iters, check_every, timeout_ms
    o.warm_start, o.use_graph, o.threads_per_node = int(warm_start), int(use_graph), int(threads_per_node)
    o.eps_start, o.eps_stages, o.eps_stage_tol = float(eps_start), int(eps_stages), float(eps_stage_tol)
    r = SolveReport()
    code = load_library().ots_sinkhorn_solve(h.ptr, ctypes.byref(o), ctypes.byref(r))
    if raise_on_error and code not in (OTS_OK,):
        _check(code)
    return r.as_dict()


def ots_iterate(h: Handle, n: int, reset: bool = False) -> dict:
    r = SolveReport()
    _check(load_library().ots_iterate(h.ptr, int(n), int(reset), ctypes.byref(r)))
    return r.as_dict()


def _solve_opts(tol, max_iters, check_every, timeout_ms, warm_start, use_graph):
    o = ots_default_solve_opts()
    o.tol, o.max_iters, o.check_every, o.timeout_ms = tol, max_iters, check_every, timeout_ms
    o.warm_start, o.use_graph = int(warm_start), int(use_graph)
    return o


def ots_linear_iterate(h: Handle, n: int, reset: bool = False) -> dict:
    """n linear-domain passes (L = 1); the report of the last pass plus the pass counters."""
    r, st = SolveReport(), LinearStats()
    _check(load_library().ots_linear_iterate(h.ptr, int(n), int(reset), ctypes.byref(r), ctypes.byref(st)))
    return dict(r.as_dict(), linear=st.as_dict())


def ots_linear_solve(h: Handle, tol: float = 1e-6, max_iters: int = 100000, check_every: int = 10,
                     timeout_ms: float = 0.0, warm_start: bool = False, use_graph: bool = True,
                     raise_on_error: bool = True) -> dict:
    """Linear-domain passes to tol, confirmed by log-domain passes (L = 1)."""
    o = _solve_opts(tol, max_iters, check_every, timeout_ms, warm_start, use_graph)
    r, st = SolveReport(), LinearStats()
    code = load_library().ots_linear_solve(h.ptr, ctypes.byref(o), ctypes.byref(r), ctypes.byref(st))
    if raise_on_error:
        _check(code)
    return dict(r.as_dict(), linear=st.as_dict())


def ots_linear_solve_many(hs, tol: float = 1e-6, max_iters: int = 100000, check_every: int = 10,
                          timeout_ms: float = 0.0, warm_start: bool = False, use_graph: bool = True,
                          raise_on_error: bool = True):
    """The same for several L = 1 problems in one launch; returns (per-problem reports, counters)."""
    o = _solve_opts(tol, max_iters, check_every, timeout_ms, warm_start, use_graph)
    n = len(hs)
    arr = (ctypes.c_void_p * n)(*[h.ptr for h in hs])
    reps = (SolveReport * n)()
    st = LinearStats()
    code = load_library().ots_linear_solve_many(arr, n, ctypes.byref(o), reps, ctypes.byref(st))
    if raise_on_error and code != OTS_OK:
        _check(code)
    return [r.as_dict() for r in reps], st.as_dict()


def ots_get_flows(h: Handle, t_begin: int = 1, t_end: int | None = None) -> np.ndarray:
    t_end = h.T + 1 if t_end is None else t_end
    out = np.empty((t_end - t_begin, h.n_states), np.float64)
    _check(load_library().ots_get_flows(h.ptr, int(t_begin), int(t_end), _ptr(out, ctypes.c_double)))
    return out


def ots_get_commodity_flows(h: Handle, t_begin: int = 1, t_end: int | None = None, l_begin: int = 0,
                            l_end: int | None = None) -> np.ndarray:
    t_end = h.T + 1 if t_end is None else t_end
    l_end = h.L if l_end is None else l_end
    out = np.empty((t_end - t_begin, l_end - l_begin, h.n_states), np.float64)
    _check(load_library().ots_get_commodity_flows(h.ptr, int(t_begin), int(t_end), int(l_begin), int(l_end),
                                                  _ptr(out, ctypes.c_double)))
    return out


def ots_get_commodity_flows_noalloc(h: Handle, t_begin: int = 1, t_end: int | None = None, l_begin: int = 0,
                                    l_end: int | None = None) -> np.ndarray:
    """Same values as ots_get_commodity_flows; the library allocates no memory in this call
    (its scratch is a fixed static device array, see include/ots.h for the limits)."""
    t_end = h.T + 1 if t_end is None else t_end
    l_end = h.L if l_end is None else l_end
    out = np.empty((t_end - t_begin, l_end - l_begin, h.n_states), np.float64)
    _check(load_library().ots_get_commodity_flows_noalloc(h.ptr, int(t_begin), int(t_end), int(l_begin),
                                                          int(l_end), _ptr(out, ctypes.c_double)))
    return out


def ots_get_duals(h: Handle):
    lu = np.empty((h.T - 2, h.n_states), np.float64)
    u1 = np.empty(h.n_sources, np.float64)
    uT = np.empty(h.n_sinks, np.float64)
    _check(load_library().ots_get_duals(h.ptr, _ptr(lu, ctypes.c_double), _ptr(u1, ctypes.c_double),
                                        _ptr(uT, ctypes.c_double)))
    return lu, u1, uT


def ots_set_duals(h: Handle, log_u, log_U01, log_U0T) -> None:
    lu = np.ascontiguousarray(log_u, np.float64)
    u1 = np.ascontiguousarray(log_U01, np.float64)
    uT = np.ascontiguousarray(log_U0T, np.float64)
    _check(load_library().ots_set_duals(h.ptr, _ptr(lu, ctypes.c_double), _ptr(u1, ctypes.c_double),
                                        _ptr(uT, ctypes.c_double)))


def ots_set_wait_limit(h: Handle, tries: int = 0, withhold_stage: bool = False) -> None:
    _check(load_library().ots_set_wait_limit(h.ptr, int(tries), int(bool(withhold_stage))))


def ots_problem_info(h: Handle) -> dict:
    st = ProblemStats()
    _check(load_library().ots_problem_info(h.ptr, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in st._fields_}


def ots_last_pass_timing(h: Handle) -> dict:
    ms = np.zeros(4, np.float64)
    _check(load_library().ots_last_pass_timing(h.ptr, _ptr(ms, ctypes.c_double)))
    return {"source_ms": ms[0], "forward_ms": ms[1], "sink_ms": ms[2], "backward_ms": ms[3]}


def ots_problem_stream(h: Handle) -> int:
    return int(load_library().ots_problem_stream(h.ptr) or 0)


def ots_destroy_problem(h: Handle) -> None:
    if h.ptr:
        load_library().ots_destroy_problem(h.ptr)
        h.ptr = None


# ---------------------------------------------------------------------------------------
# batches
# ---------------------------------------------------------------------------------------
class Batch:
    """Owns an ``ots_batch*`` and the shapes of the instances added to it."""

    def __init__(self, ptr, keep):
        self.ptr = ptr
        self._keep = keep
        self.shapes = {}   # id -> (n_states, T, L, n_sources, n_sinks)

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                ots_batch_destroy(self)
            except Exception:
                pass


def ots_batch_create(device: int = 0, pool_bytes: int = 4 << 30, max_instances: int = 256, max_items: int = 0,
                     ticks_per_launch: int = 0, stream: int | None = None, allocator: str = "torch") -> Batch:
    lib = load_library()
    d = BatchDesc()
    _check(lib.ots_default_batch_desc(ctypes.byref(d)))
    d.device, d.stream, d.pool_bytes = int(device), stream, int(pool_bytes)
    d.max_instances, d.max_items, d.ticks_per_launch = int(max_instances), int(max_items), int(ticks_per_launch)
    keep = []
    if allocator == "torch":
        a, f = _torch_allocator(int(device))
        d.alloc, d.free_fn = a, f
        keep.append((a, f))
    elif allocator != "cuda":
        raise ValueError("allocator must be 'torch' or 'cuda'")
    out = ctypes.c_void_p()
    _check(lib.ots_batch_create(ctypes.byref(d), ctypes.byref(out)))
    return Batch(out, keep)


def ots_batch_add(b: Batch, inst, tol: float = 1e-6, max_iters: int = 100000, timeout_ms: float = 0.0,
                  raise_on_error: bool = True, eps_start: float = 0.0, eps_stage_tol: float = 0.0):
    """Add an instance; returns its id (or the status code when raise_on_error is False and the
    call failed, e.g. OTS_ERR_OOM when the batch is full)."""
    d, arr = _problem_desc(inst)
    o = ots_default_solve_opts()
    o.tol, o.max_iters, o.timeout_ms = tol, max_iters, timeout_ms
    o.eps_start, o.eps_stage_tol = float(eps_start), float(eps_stage_tol)
    i = ctypes.c_int32(-1)
    code = load_library().ots_batch_add(b.ptr, ctypes.byref(d), ctypes.byref(o), ctypes.byref(i))
    if code != OTS_OK:
        if raise_on_error:
            _check(code)
        return -code
    b.shapes[i.value] = (int(inst.n_nodes) + d.n_edges, d.T, d.L, d.n_sources, d.n_sinks)
    return i.value


def ots_batch_run(b: Batch, max_launches: int = 1 << 30) -> int:
    n = ctypes.c_int32(0)
    _check(load_library().ots_batch_run(b.ptr, int(max_launches), ctypes.byref(n)))
    return n.value


def ots_batch_status(b: Batch, i: int) -> dict:
    r = SolveReport()
    code = load_library().ots_batch_status(b.ptr, int(i), ctypes.byref(r))
    if code == OTS_ERR_INVALID_ARG:
        _check(code)
    out = r.as_dict()
    out["status"] = code
    return out


def ots_batch_get_flows(b: Batch, i: int, t_begin: int = 1, t_end: int | None = None) -> np.ndarray:
    S, T = b.shapes[i][0], b.shapes[i][1]
    t_end = T + 1 if t_end is None else t_end
    out = np.empty((t_end - t_begin, S), np.float64)
    _check(load_library().ots_batch_get_flows(b.ptr, int(i), int(t_begin), int(t_end), _ptr(out, ctypes.c_double)))
    return out


def ots_batch_get_duals(b: Batch, i: int):
    S, T, _, ns, nz = b.shapes[i]
    lu = np.empty((T - 2, S), np.float64)
    u1 = np.empty(ns, np.float64)
    uT = np.empty(nz, np.float64)
    _check(load_library().ots_batch_get_duals(b.ptr, int(i), _ptr(lu, ctypes.c_double), _ptr(u1, ctypes.c_double),
                                              _ptr(uT, ctypes.c_double)))
    return lu, u1, uT


def ots_batch_remove(b: Batch, i: int) -> None:
    _check(load_library().ots_batch_remove(b.ptr, int(i)))
    b.shapes.pop(i, None)


def ots_batch_info(b: Batch) -> dict:
    st = BatchStats()
    _check(load_library().ots_batch_info(b.ptr, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in st._fields_}


def ots_batch_mapping(b: Batch, L: int):
    g, c = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(load_library().ots_batch_mapping(b.ptr, int(L), ctypes.byref(g), ctypes.byref(c)))
    return g.value, c.value


def ots_batch_autotune(b: Batch, cache_path: str | None = None) -> None:
    _check(load_library().ots_batch_autotune(b.ptr, None if cache_path is None else cache_path.encode()))


def ots_batch_destroy(b: Batch) -> None:
    if b.ptr:
        load_library().ots_batch_destroy(b.ptr)
        b.ptr = None


# ---------------------------------------------------------------------------------------
# server
# ---------------------------------------------------------------------------------------
class Server:
    """Owns an ``ots_server*`` and the shapes of the requests submitted to it."""

    def __init__(self, ptr, keep):
        self.ptr = ptr
        self._keep = keep
        self.shapes = {}   # ticket -> (n_states, T)

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                ots_server_destroy(self)
            except Exception:
                pass


def ots_server_create(device: int = 0, pool_bytes: int = 4 << 30, max_instances: int = 256, ticks_per_launch: int = 8,
                      builder_threads: int = 2, max_queued: int = 0, mode: int = 0, allocator: str = "torch") -> Server:
    """mode 0: continuous batching; mode 1: one request at a time with the single-instance solver."""
    lib = load_library()
    d = ServerDesc()
    _check(lib.ots_default_server_desc(ctypes.byref(d)))
    d.batch.device, d.batch.pool_bytes, d.batch.max_instances = int(device), int(pool_bytes), int(max_instances)
    d.batch.ticks_per_launch = int(ticks_per_launch)
    d.builder_threads, d.max_queued, d.mode = int(builder_threads), int(max_queued), int(mode)
    keep = []
    if allocator == "torch":
        a, f = _torch_allocator(int(device))
        d.batch.alloc, d.batch.free_fn = a, f
        keep.append((a, f))
    elif allocator != "cuda":
        raise ValueError("allocator must be 'torch' or 'cuda'")
    out = ctypes.c_void_p()
    _check(lib.ots_server_create(ctypes.byref(d), ctypes.byref(out)))
    return Server(out, keep)


def ots_server_submit(s: Server, inst, tol: float = 1e-6, max_iters: int = 100000, timeout_ms: float = 0.0,
                      check_every: int = 1, eps_start: float = 0.0, eps_stages: int = 0) -> int:
    d, arr = _problem_desc(inst)
    o = ots_default_solve_opts()
    o.tol, o.max_iters, o.timeout_ms, o.check_every = tol, max_iters, timeout_ms, check_every
    o.eps_start, o.eps_stages = float(eps_start), int(eps_stages)
    t = ctypes.c_int64(0)
    _check(load_library().ots_server_submit(s.ptr, ctypes.byref(d), ctypes.byref(o), ctypes.byref(t)))
    s.shapes[t.value] = (int(inst.n_nodes) + d.n_edges, d.T)
    return t.value


def _report(code, r):
    out = r.as_dict()
    out["status"] = code
    return out


def ots_server_poll(s: Server, ticket: int) -> dict:
    r = SolveReport()
    code = load_library().ots_server_poll(s.ptr, int(ticket), ctypes.byref(r))
    return _report(code, r)


def ots_server_wait(s: Server, ticket: int, timeout_ms: float = 0.0) -> dict:
    r = SolveReport()
    code = load_library().ots_server_wait(s.ptr, int(ticket), float(timeout_ms), ctypes.byref(r))
    return _report(code, r)


def ots_server_get_flows(s: Server, ticket: int, t_begin: int = 1, t_end: int | None = None) -> np.ndarray:
    S, T = s.shapes[ticket]
    t_end = T + 1 if t_end is None else t_end
    out = np.empty((t_end - t_begin, S), np.float64)
    _check(load_library().ots_server_get_flows(s.ptr, int(ticket), int(t_begin), int(t_end),
                                               _ptr(out, ctypes.c_double)))
    return out


def ots_server_timing(s: Server, ticket: int) -> dict:
    ms = np.zeros(3, np.float64)
    _check(load_library().ots_server_timing(s.ptr, int(ticket), _ptr(ms, ctypes.c_double)))
    return {"wait_ms": ms[0], "run_ms": ms[1], "total_ms": ms[2]}


def ots_server_release(s: Server, ticket: int) -> None:
    _check(load_library().ots_server_release(s.ptr, int(ticket)))
    s.shapes.pop(ticket, None)


def ots_server_info(s: Server) -> dict:
    st = ServerStats()
    _check(load_library().ots_server_info(s.ptr, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in st._fields_}


def ots_server_destroy(s: Server) -> None:
    if s.ptr:
        load_library().ots_server_destroy(s.ptr)
        s.ptr = None
