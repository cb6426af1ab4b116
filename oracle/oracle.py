"""Python handle on the FP64 CPU oracle (``ots_oracle.c``).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use this module.  It imports nothing from the GPU package: instances are
passed in as plain objects carrying numpy arrays (the attributes of
``paper_2106_14485_gb300.instances.Instance``).

The oracle follows Algorithm 2 (Section 4.3) step by step in FP64 log domain on the
state-level line graph; see the header of ``ots_oracle.c`` for the notation and readings.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ots_oracle.c")
_SO = os.path.join(_HERE, "libots_oracle.so")

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")

ORC_OK, ORC_BAD_ARG, ORC_NOMEM, ORC_INFEASIBLE = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP, IEEE libm; no fast-math)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def _load(path: str | None = None):
    """The oracle library (built on first use), or, for the tests that plant mistakes in copies of
    the oracle, the library at path."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    if path is None:
        build()
    lib = ctypes.CDLL(path or _SO)
    lib.orc_create.restype = ctypes.c_void_p
    lib.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, _i32p, _i32p, ctypes.c_int, ctypes.c_int,
                               ctypes.c_double, _f64p, ctypes.c_int, _f64p,
                               ctypes.c_int, _i32p, _i32p, _f64p, ctypes.c_int, _i32p, _i32p, _f64p]
    lib.orc_destroy.argtypes = [ctypes.c_void_p]
    lib.orc_set_time_costs.argtypes = [ctypes.c_void_p, _f64p]
    lib.orc_set_time_costs.restype = ctypes.c_int
    lib.orc_set_time_capacities.argtypes = [ctypes.c_void_p, _f64p]
    lib.orc_set_time_capacities.restype = ctypes.c_int
    lib.orc_set_windows.argtypes = [ctypes.c_void_p, _i32p, _i32p]
    lib.orc_set_windows.restype = ctypes.c_int
    lib.orc_set_commodity_capacities.argtypes = [ctypes.c_void_p, _f64p]
    lib.orc_set_state_graph.argtypes = [ctypes.c_void_p, _i32p, _i32p, ctypes.c_void_p]
    lib.orc_set_state_graph.restype = ctypes.c_int
    lib.orc_set_commodity_capacities.restype = ctypes.c_int
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    lib.orc_get_threads.restype = ctypes.c_int
    lib.orc_num_states.argtypes = [ctypes.c_void_p]
    lib.orc_num_states.restype = ctypes.c_int
    lib.orc_nnz.argtypes = [ctypes.c_void_p]
    lib.orc_nnz.restype = ctypes.c_int64
    lib.orc_init_duals.argtypes = [ctypes.c_void_p]
    lib.orc_set_duals.argtypes = [ctypes.c_void_p, _f64p, _f64p, _f64p]
    lib.orc_get_duals.argtypes = [ctypes.c_void_p, _f64p, _f64p, _f64p]
    lib.orc_backward_sweep.argtypes = [ctypes.c_void_p]
    lib.orc_backward_sweep.restype = ctypes.c_int
    lib.orc_iteration.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    lib.orc_iteration.restype = ctypes.c_int
    lib.orc_dual_objective.argtypes = [ctypes.c_void_p]
    lib.orc_dual_objective.restype = ctypes.c_double
    lib.orc_solve.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.orc_solve.restype = ctypes.c_int
    lib.orc_messages.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.orc_messages.restype = ctypes.c_int
    lib.orc_projections.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _f64p]
    lib.orc_projections.restype = ctypes.c_int
    lib.orc_sample_backward_products.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    lib.orc_sample_backward_products.restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def state_cost_matrix(inst) -> np.ndarray:
    """C_L as used by the oracle: [S] (shared rows) or [L, S] (per-commodity)."""
    if getattr(inst, "commodity_cost", None) is not None:
        return np.ascontiguousarray(inst.commodity_cost, np.float64)
    return np.concatenate([inst.edge_cost, inst.wait_cost]).astype(np.float64)


class Oracle:
    """FP64 log-domain Algorithm 2 for one instance."""

    def __init__(self, inst, threads: int | None = None, lib_path: str | None = None):
        lib = _load(lib_path)
        if threads:
            lib.orc_set_threads(int(threads))
        self.inst = inst
        self.V = int(inst.n_nodes)
        self.E = int(inst.edge_src.shape[0])
        self.S = self.E + self.V
        self.L, self.T, self.eps = int(inst.L), int(inst.T), float(inst.eps)
        cost = state_cost_matrix(inst)
        per_comm = 1 if cost.ndim == 2 else 0
        cap = np.concatenate([inst.edge_cap, inst.wait_cap]).astype(np.float64)
        a = lambda x, dt: np.ascontiguousarray(x, dt)
        self._keep = [a(inst.edge_src, np.int32), a(inst.edge_dst, np.int32), a(cost.ravel(), np.float64),
                      cap, a(inst.src_comm, np.int32), a(inst.src_state, np.int32), a(inst.src_mass, np.float64),
                      a(inst.snk_comm, np.int32), a(inst.snk_state, np.int32), a(inst.snk_mass, np.float64)]
        k = self._keep
        self.h = lib.orc_create(self.V, self.E, k[0], k[1], self.L, self.T, self.eps, k[2], per_comm, k[3],
                                len(k[4]), k[4], k[5], k[6], len(k[7]), k[7], k[8], k[9])
        if not self.h:
            raise ValueError("oracle rejected the instance")
        self._lib = lib
        st = getattr(inst, "state_tail", None)
        if st is not None:                    # explicit state graph: storage states (Section 3.3)
            tl = np.ascontiguousarray(st, np.int32)
            hd = np.ascontiguousarray(inst.state_head, np.int32)
            hl = getattr(inst, "state_hold", None)
            hl = None if hl is None else np.ascontiguousarray(hl, np.int32)
            if tl.shape != (self.S,) or hd.shape != (self.S,) or (hl is not None and hl.shape != (self.S,)):
                raise ValueError("state_tail / state_head / state_hold must have n_states entries")
            self._keep += [tl, hd, hl]
            if lib.orc_set_state_graph(self.h, tl, hd, None if hl is None else hl.ctypes.data):
                raise ValueError("oracle: state heads and tails must be -1 or a node")
        ct = getattr(inst, "state_cost_t", None)
        if ct is not None:                    # time-varying network: one C_L per interval t
            ct = np.ascontiguousarray(ct, np.float64)
            if ct.shape != (self.T - 2, self.S):
                raise ValueError("state_cost_t must be (T-2) x n_states")
            if lib.orc_set_time_costs(self.h, ct.reshape(-1)):
                raise MemoryError("oracle: time-varying costs")
        dt = getattr(inst, "state_capacity_t", None)
        if dt is not None:
            dt = np.ascontiguousarray(dt, np.float64)
            if dt.shape != (self.T - 2, self.S):
                raise ValueError("state_capacity_t must be (T-2) x n_states")
            if lib.orc_set_time_capacities(self.h, dt.reshape(-1)):
                raise ValueError("oracle: per-interval capacities must be >= 0 (inf for none)")
        ta = getattr(inst, "commodity_t_in", None)
        tb = getattr(inst, "commodity_t_out", None)
        if ta is not None or tb is not None:
            ta = np.ascontiguousarray(np.ones(self.L) if ta is None else ta, np.int32)
            tb = np.ascontiguousarray(np.full(self.L, self.T) if tb is None else tb, np.int32)
            if lib.orc_set_windows(self.h, ta, tb):
                raise ValueError("oracle: commodity windows need 1 <= t_in < t_out <= T")
        cd = getattr(inst, "commodity_capacity", None)
        if cd is not None:
            cd = np.ascontiguousarray(cd, np.float64)
            if cd.shape != (self.L, self.S):
                raise ValueError("commodity_capacity must be L x n_states")
            if lib.orc_set_commodity_capacities(self.h, cd.reshape(-1)):
                raise ValueError("oracle: commodity capacities must be >= 0 (inf for none)")
        lib.orc_init_duals(self.h)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._lib.orc_destroy(h)
            self.h = None

    @property
    def nnz(self) -> int:
        return int(self._lib.orc_nnz(self.h))

    def init_duals(self):
        self._lib.orc_init_duals(self.h)

    def set_duals(self, logu, logU01, logU0T):
        self._lib.orc_set_duals(self.h, np.ascontiguousarray(logu, np.float64).reshape(-1),
                                np.ascontiguousarray(logU01, np.float64).reshape(-1),
                                np.ascontiguousarray(logU0T, np.float64).reshape(-1))

    def get_duals(self):
        logu = np.empty((self.T - 2, self.S))
        U01 = np.empty((self.L, self.S))
        U0T = np.empty((self.L, self.S))
        self._lib.orc_get_duals(self.h, logu.reshape(-1), U01.reshape(-1), U0T.reshape(-1))
        return logu, U01, U0T

    def backward_sweep(self):
        rc = self._lib.orc_backward_sweep(self.h)
        if rc:
            raise RuntimeError(f"oracle backward sweep failed ({rc})")

    def iteration(self, trace: bool = False):
        r, c = ctypes.c_double(), ctypes.c_double()
        tr = np.zeros(self.T) if trace else None
        rc = self._lib.orc_iteration(self.h, ctypes.byref(r), ctypes.byref(c),
                                     tr.ctypes.data if trace else None)
        if rc:
            raise RuntimeError(f"oracle iteration failed ({rc})")
        return r.value, c.value, tr

    def dual_objective(self) -> float:
        return float(self._lib.orc_dual_objective(self.h))

    def solve(self, max_iters: int = 10000, tol: float = 1e-6) -> dict:
        it, r, c = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        t0 = time.perf_counter()
        rc = self._lib.orc_solve(self.h, int(max_iters), float(tol), ctypes.byref(it), ctypes.byref(r), ctypes.byref(c))
        return {"status": rc, "iters": it.value, "src_resid": r.value, "cap_viol": c.value,
                "seconds": time.perf_counter() - t0}

    def messages(self, l0: int = 0, l1: int | None = None):
        """(hatPsi rows t=2..T, Psi rows t=1..T-1), each [T-1, l1-l0, S], log domain."""
        l1 = self.L if l1 is None else l1
        nl = l1 - l0
        h = np.empty((self.T - 1, nl, self.S))
        b = np.empty((self.T - 1, nl, self.S))
        rc = self._lib.orc_messages(self.h, l0, l1, h.ctypes.data, b.ctypes.data)
        if rc:
            raise RuntimeError(f"oracle messages failed ({rc})")
        return h, b

    def projections(self, l0: int = 0, l1: int | None = None) -> np.ndarray:
        """P_{0,t} for t = 1..T, shape [T, l1-l0, S]."""
        l1 = self.L if l1 is None else l1
        out = np.empty((self.T, l1 - l0, self.S))
        rc = self._lib.orc_projections(self.h, l0, l1, out.reshape(-1))
        if rc:
            raise RuntimeError(f"oracle projections failed ({rc})")
        return out

    def flows(self, chunk: int = 64) -> np.ndarray:
        """Aggregate flows P_t = sum_l P_{0,t}, shape [T, S] (Corollary 7)."""
        tot = np.zeros((self.T, self.S))
        for l0 in range(0, self.L, chunk):
            tot += self.projections(l0, min(self.L, l0 + chunk)).sum(axis=1)
        return tot

    def sample_backward_products(self, k: int, l1: int) -> None:
        rc = self._lib.orc_sample_backward_products(self.h, int(k), int(l1))
        if rc:
            raise RuntimeError(f"oracle sample failed ({rc})")
