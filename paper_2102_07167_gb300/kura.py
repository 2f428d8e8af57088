"""Thin ctypes binding of libkura (include/kura.h).

Every function named ``kura_*`` here has the name, arguments and meaning of
the C entry point of the same name; it only marshals arguments (torch tensors
or numpy arrays to pointers, Python numbers to C scalars) and raises
``KuraError`` for a non-zero status.  All computation happens in the
library's CUDA kernels; if ``libkura.so`` is missing, loading raises instead
of falling back to anything else.  ``Kuramoto`` bundles a handle with these
calls for convenience.

The method: Kuramoto model on graphs with localised order parameters
(arXiv 2102.07167, eq:KuramotoGraph and eq:KuramotoGraphApproach, Sec. 3),
integrated by classical RK4.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libkura.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "kura.h")

KURA_OK, KURA_EINVAL, KURA_ENOMEM, KURA_ECUDA, KURA_ESTATE, KURA_ETIMEOUT, KURA_ENUMERIC = range(7)
PREC_FP64, PREC_MIXED = 0, 1
SCALING_UNIFORM, SCALING_DEGREE = 0, 1

_lock = threading.Lock()
_lib = None


class KuraError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libkura status {status}: {msg}")
        self.status = status


class KuraOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("scaling", C.c_int32), ("tau", C.c_double),
                ("keep_host_csr", C.c_int32), ("tensor_cores", C.c_int32), ("bitmap_zmin", C.c_double),
                ("row_lanes", C.c_int32), ("persistent_small", C.c_int32), ("fused_trig", C.c_int32),
                ("reserved", C.c_int32)]


class KuraBlockStats(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("self_loops", C.c_int64),
                ("n_comm", C.c_int32), ("q_bits", C.c_int32), ("tau", C.c_double),
                ("dense_blocks", C.c_int64), ("sparse_blocks", C.c_int64), ("nonempty_blocks", C.c_int64),
                ("missing_entries", C.c_int64), ("sparse_entries", C.c_int64), ("max_row_entries", C.c_int64),
                ("tiles", C.c_int64), ("max_window", C.c_int64),
                ("stream_bytes", C.c_int64), ("node_bytes_row", C.c_int64), ("node_bytes_trig", C.c_int64),
                ("direct_edges", C.c_int64), ("tc_tiles", C.c_int64), ("tc_rows", C.c_int64),
                ("tc_mask_bits", C.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class KuraTuneResult(C.Structure):
    _fields_ = [("tau", C.c_double), ("tensor_cores", C.c_int32), ("candidates", C.c_int32),
                ("tile_work", C.c_int64), ("rhs_ms", C.c_double), ("initial_rhs_ms", C.c_double),
                ("seconds", C.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class KuraBatchInfo(C.Structure):
    _fields_ = [("n_traj", C.c_int32), ("precision", C.c_int32), ("n_total", C.c_int64),
                ("missing_listed", C.c_int64), ("present", C.c_int64), ("tc_traj", C.c_int32),
                ("pad", C.c_int32), ("tc_tiles", C.c_int64), ("tc_mask_bits", C.c_int64)]


class KuraGraphDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("label", C.c_void_p),
                ("n_comm", C.c_int32), ("omega", C.c_void_p), ("K", C.c_double)]


def header_functions() -> list:
    """Names of the functions declared in include/kura.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(kura_[a-z_0-9]+)\s*\(", txt)))


def load() -> C.CDLL:
    """Loads libkura.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first "
                               "(there is no fallback path)")
        L = C.CDLL(LIB_PATH)
        P, I64, I32, D, S = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_int
        sig = {
            "kura_default_opts": (None, [C.POINTER(KuraOpts)]),
            "kura_version": (I32, []),
            "kura_status_string": (C.c_char_p, [S]),
            "kura_create": (S, [I64, P, P, P, I32, P, D, C.POINTER(KuraOpts), P, C.POINTER(P)]),
            "kura_classify_blocks": (S, [P, D, C.POINTER(KuraBlockStats)]),
            "kura_get_stats": (S, [P, C.POINTER(KuraBlockStats)]),
            "kura_rhs": (S, [P, P, P]),
            "kura_rk4_steps": (S, [P, P, D, I64]),
            "kura_order_params": (S, [P, P, C.POINTER(D), C.POINTER(D), P, P]),
            "kura_set_param": (S, [P, P, P]),
            "kura_adjoint": (S, [P, P, D, I64, I32, I32, P, C.POINTER(D), P, C.POINTER(D), P]),
            "kura_direct_rhs": (S, [P, P, P, I32]),
            "kura_direct_rk4_steps": (S, [P, P, D, I64, I32]),
            "kura_set_timing": (S, [P, I32]),
            "kura_autotune": (S, [P, P, D, C.POINTER(KuraTuneResult)]),
            "kura_ensemble_create": (S, [I64, P, P, P, I32, I32, P, P, C.POINTER(KuraOpts), P, C.POINTER(P)]),
            "kura_measure_gather_rate": (S, [I64, I64, I32, P, C.POINTER(D)]),
            "kura_potential": (S, [P, P, C.POINTER(D)]),
            "kura_integrate": (S, [P, P, D, I64, I32, I32]),
            "kura_create_valued": (S, [I64, P, P, P, P, I32, P, D, C.POINTER(KuraOpts), P, C.POINTER(P)]),
            "kura_plan_build_valued": (S, [I64, P, P, P, P, I32, C.POINTER(KuraOpts), C.POINTER(P)]),
            "kura_plan_dense_values": (S, [P, I32, P, I32, C.POINTER(I32)]),
            "kura_mean_deviation": (S, [P, P, P, D, C.POINTER(D)]),
            "kura_kernel_times": (S, [P, P, I32, C.POINTER(I32)]),
            "kura_set_stream": (S, [P, P]),
            "kura_sync": (S, [P]),
            "kura_last_error": (C.c_char_p, [P]),
            "kura_destroy": (None, [P]),
            "kura_order_params_static": (S, [I64, P, P, I32, P, P]),
            "kura_plan_build": (S, [I64, P, P, P, I32, C.POINTER(KuraOpts), C.POINTER(P)]),
            "kura_batch_create": (S, [I32, C.POINTER(KuraGraphDesc), C.POINTER(KuraOpts), P, C.POINTER(P)]),
            "kura_batch_stats": (S, [P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64)]),
            "kura_batch_info": (S, [P, C.POINTER(KuraBatchInfo)]),
            "kura_batch_traj_params": (S, [P, I32, C.POINTER(D), C.POINTER(I32), C.POINTER(I32)]),
            "kura_batch_costs": (S, [I32, C.POINTER(KuraGraphDesc), C.POINTER(KuraOpts), P]),
            "kura_partition_lpt": (S, [P, I32, I32, P, P]),
            "kura_measure_l2_bandwidth": (S, [I64, P, C.POINTER(D)]),
            "kura_measure_graph_launch_floor": (S, [I32, I32, P, C.POINTER(D)]),
            "kura_plan_stats": (S, [P, C.POINTER(KuraBlockStats)]),
            "kura_plan_perm": (S, [P, P, P]),
            "kura_plan_row": (S, [P, I64, P, C.POINTER(I64), P, C.POINTER(I64), I64]),
            "kura_plan_dense_blocks": (S, [P, I32, P, I32, C.POINTER(I32)]),
            "kura_plan_export": (S, [P, C.POINTER(P), C.POINTER(I64), C.POINTER(P), C.POINTER(I64), C.POINTER(P),
                                     C.POINTER(I64), C.POINTER(P), C.POINTER(P), C.POINTER(I64)]),
            "kura_plan_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


# ----------------------------------------------------------------------------- marshalling
def _ptr(x, dtype=np.float64, n: Optional[int] = None):
    """Pointer to a contiguous torch tensor (any device) or numpy array; None -> NULL."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):                     # torch tensor
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64,
                np.float32: torch.float32}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        if n is not None and x.numel() < n:
            raise ValueError(f"tensor has {x.numel()} elements, need {n}")
        return x.data_ptr()
    if not isinstance(x, np.ndarray) or x.dtype != dtype or not x.flags.c_contiguous:
        raise TypeError(f"array must be a C-contiguous numpy {np.dtype(dtype).name} array")
    if n is not None and x.size < n:
        raise ValueError(f"array has {x.size} elements, need {n}")
    return x.ctypes.data


def _check(rc: int, h=None):
    if rc != KURA_OK:
        L = load()
        msg = L.kura_last_error(h)
        raise KuraError(rc, (msg or b"").decode() or L.kura_status_string(rc).decode())


def _current_stream() -> int:
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return 0


# ----------------------------------------------------------------------------- C-ABI mirrors
def kura_default_opts() -> KuraOpts:
    o = KuraOpts()
    load().kura_default_opts(C.byref(o))
    return o


def kura_version() -> int:
    return int(load().kura_version())


def kura_create(n, row_ptr, col, label, n_comm, omega, K, opts: Optional[KuraOpts] = None, stream=None):
    h = C.c_void_p()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    label = np.ascontiguousarray(label, dtype=np.int32)
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    if row_ptr.size != n + 1 or label.size != n or omega.size != n:
        raise ValueError("row_ptr must have n+1 entries, label and omega n")
    if col.size < int(row_ptr[-1]):
        raise ValueError("col shorter than row_ptr[n]")
    s = _current_stream() if stream is None else int(stream)
    rc = load().kura_create(int(n), row_ptr.ctypes.data, col.ctypes.data if col.size else None,
                            label.ctypes.data, int(n_comm), omega.ctypes.data, float(K),
                            C.byref(opts) if opts is not None else None, s or None, C.byref(h))
    _check(rc, None)
    return h


def _graph_descs(graphs):
    """kura_graph_desc array of (row_ptr, col, label, n_comm, omega, K) tuples, the arrays it points into
    (keep them alive) and the node offsets."""
    keep, descs, offs = [], [], [0]
    for (row_ptr, col, label, n_comm, omega, K) in graphs:
        om = np.ascontiguousarray(omega, dtype=np.float64)
        n = om.size
        keep.append(om)
        if row_ptr is None:                      # complete graph: no adjacency passed
            descs.append(KuraGraphDesc(n, None, None, None, 1, om.ctypes.data, float(K)))
        else:
            rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
            cl = np.ascontiguousarray(col, dtype=np.int32)
            lb = np.ascontiguousarray(label, dtype=np.int32)
            keep += [rp, cl, lb]
            descs.append(KuraGraphDesc(n, rp.ctypes.data, cl.ctypes.data if cl.size else None, lb.ctypes.data,
                                       int(n_comm), om.ctypes.data, float(K)))
        offs.append(offs[-1] + n)
    return (KuraGraphDesc * len(descs))(*descs), keep, offs


def kura_batch_create(graphs, opts: Optional[KuraOpts] = None, stream=None):
    """graphs: sequence of (row_ptr, col, label, n_comm, omega, K).  Returns (handle, node offsets)."""
    arr, keep, offs = _graph_descs(graphs)
    h = C.c_void_p()
    if opts is None:
        opts = kura_default_opts()
        opts.precision = PREC_MIXED
    s = _current_stream() if stream is None else int(stream)
    _check(load().kura_batch_create(len(arr), arr, C.byref(opts), s or None, C.byref(h)), None)
    return h, np.array(offs, dtype=np.int64)


def kura_batch_costs(graphs, opts: Optional[KuraOpts] = None) -> np.ndarray:
    """Host only: the work-queue cost of each trajectory of a would-be batch (see kura_batch_create)."""
    arr, keep, _ = _graph_descs(graphs)
    cost = np.zeros(len(arr), dtype=np.float64)
    _check(load().kura_batch_costs(len(arr), arr, C.byref(opts) if opts is not None else None,
                                   cost.ctypes.data if cost.size else None), None)
    return cost


def kura_partition_lpt(cost, n_parts: int):
    """Host only: longest-processing-time partition of items with these costs over n_parts parts.
    Returns (part of each item, load of each part); the same costs give the same partition everywhere."""
    c = np.ascontiguousarray(cost, dtype=np.float64)
    part = np.zeros(c.size, dtype=np.int32)
    load_ = np.zeros(max(int(n_parts), 0), dtype=np.float64)
    _check(load().kura_partition_lpt(c.ctypes.data if c.size else None, int(c.size), int(n_parts),
                                     part.ctypes.data if part.size else None,
                                     load_.ctypes.data if load_.size else None), None)
    return part, load_


def kura_batch_stats(h):
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    _check(load().kura_batch_stats(h, C.byref(a), C.byref(b), C.byref(c)), h)
    return {"n_total": a.value, "missing_entries": b.value, "sparse_entries": c.value}


def kura_batch_info(h):
    info = KuraBatchInfo()
    _check(load().kura_batch_info(h, C.byref(info)), h)
    return {k: getattr(info, k) for k, _ in KuraBatchInfo._fields_ if k != "pad"}


def kura_classify_blocks(h, tau: float = -1.0) -> dict:
    st = KuraBlockStats()
    _check(load().kura_classify_blocks(h, float(tau), C.byref(st)), h)
    return st.as_dict()


def kura_get_stats(h) -> dict:
    st = KuraBlockStats()
    _check(load().kura_get_stats(h, C.byref(st)), h)
    return st.as_dict()


def kura_rhs(h, theta, dtheta, n):
    _check(load().kura_rhs(h, _ptr(theta, n=n), _ptr(dtheta, n=n)), h)


def kura_rk4_steps(h, theta, step, n_steps, n):
    _check(load().kura_rk4_steps(h, _ptr(theta, n=n), float(step), int(n_steps)), h)


def kura_order_params(h, theta, n, n_comm, per_community: bool = False):
    r, psi = C.c_double(), C.c_double()
    rc_ = np.zeros(n_comm) if per_community else None
    pc_ = np.zeros(n_comm) if per_community else None
    _check(load().kura_order_params(h, _ptr(theta, n=n), C.byref(r), C.byref(psi),
                                    _ptr(rc_) if per_community else None,
                                    _ptr(pc_) if per_community else None), h)
    return (r.value, psi.value, rc_, pc_) if per_community else (r.value, psi.value)


def kura_set_param(h, omega=None, K=None, n=None):
    k = C.c_double(float(K)) if K is not None else None
    _check(load().kura_set_param(h, _ptr(omega, n=n), C.byref(k) if k is not None else None), h)


def kura_adjoint(h, theta0, step, n_steps, ckpt_every, loss_kind, target, g_omega, g_theta0, n):
    """Returns (loss, g_K); fills g_omega[n] and g_theta0[n] (tensors or arrays, user order)."""
    loss, gK = C.c_double(), C.c_double()
    _check(load().kura_adjoint(h, _ptr(theta0, n=n), float(step), int(n_steps), int(ckpt_every), int(loss_kind),
                               _ptr(target, n=n) if target is not None else None, C.byref(loss),
                               _ptr(g_omega, n=n), C.byref(gK), _ptr(g_theta0, n=n)), h)
    return loss.value, gK.value


def kura_direct_rhs(h, theta, dtheta, precision, n):
    _check(load().kura_direct_rhs(h, _ptr(theta, n=n), _ptr(dtheta, n=n), int(precision)), h)


def kura_direct_rk4_steps(h, theta, step, n_steps, precision, n):
    _check(load().kura_direct_rk4_steps(h, _ptr(theta, n=n), float(step), int(n_steps), int(precision)), h)


def kura_set_timing(h, on: bool):
    _check(load().kura_set_timing(h, 1 if on else 0), h)


def kura_kernel_times(h, cap: int = 4096) -> np.ndarray:
    buf = np.zeros(cap, dtype=np.float32)
    cnt = C.c_int32()
    _check(load().kura_kernel_times(h, buf.ctypes.data, cap, C.byref(cnt)), h)
    return buf[:min(cnt.value, cap)].copy()


STATIC_MAX_COMM = 4096


def kura_order_params_static(n, theta, label, n_comm, out, stream=None):
    """Order parameters into out[2 + 2 n_comm] (device) with the library's static scratch; allocates
    nothing.  theta, label (or None), out: device tensors."""
    s = _current_stream() if stream is None else int(stream)
    rc = load().kura_order_params_static(int(n), _ptr(theta, n=n),
                                         _ptr(label, np.int32, n) if label is not None else None,
                                         int(n_comm), _ptr(out, n=2 + 2 * n_comm), s or None)
    _check(rc, None)


def kura_set_stream(h, stream):
    _check(load().kura_set_stream(h, int(stream) or None), h)


def kura_sync(h):
    _check(load().kura_sync(h), h)


def kura_last_error(h=None) -> str:
    return (load().kura_last_error(h) or b"").decode()


def kura_autotune(h, theta, n, budget_s=30.0) -> dict:
    r = KuraTuneResult()
    _check(load().kura_autotune(h, _ptr(theta, n=n), float(budget_s), C.byref(r)), h)
    return r.as_dict()


def kura_measure_gather_rate(table_entries=1 << 20, gathers=1 << 28, entry_bytes=8, stream=None) -> float:
    """Random-gather rate of this device (gathers/s) from an L2-resident table: the peak of the row kernel's
    sparse-block gathers."""
    r = C.c_double()
    _check(load().kura_measure_gather_rate(int(table_entries), int(gathers), int(entry_bytes), stream or None,
                                           C.byref(r)), None)
    return r.value


def kura_measure_l2_bandwidth(nbytes=48 << 20, stream=None) -> float:
    """Read bandwidth (GB/s) of 16-byte loads streaming over an L2-resident buffer of nbytes."""
    r = C.c_double()
    _check(load().kura_measure_l2_bandwidth(int(nbytes), stream or None, C.byref(r)), None)
    return r.value


def kura_measure_graph_launch_floor(kernels=8, replays=2000, stream=None) -> float:
    """Microseconds per kernel node when replaying a CUDA graph of empty dependent kernels."""
    r = C.c_double()
    _check(load().kura_measure_graph_launch_floor(int(kernels), int(replays), stream or None, C.byref(r)), None)
    return r.value


INT_RK4, INT_RK2, INT_IMPLICIT_MIDPOINT = 0, 1, 2


def kura_integrate(h, theta, step, n_steps, method, iters, n):
    _check(load().kura_integrate(h, _ptr(theta, n=n), float(step), int(n_steps), int(method), int(iters)), h)


def kura_potential(h, theta, n) -> float:
    v = C.c_double()
    _check(load().kura_potential(h, _ptr(theta, n=n), C.byref(v)), h)
    return v.value


def kura_mean_deviation(h, theta_t, theta_0, t, n) -> float:
    v = C.c_double()
    _check(load().kura_mean_deviation(h, _ptr(theta_t, n=n), _ptr(theta_0, n=n), float(t), C.byref(v)), h)
    return v.value


def kura_destroy(h):
    load().kura_destroy(h)


def kura_plan_build(n, row_ptr, col, label, n_comm, tau=0.5, precision=PREC_MIXED, bitmap_zmin=-1.0,
                    tensor_cores=1):
    p = C.c_void_p()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    label = np.ascontiguousarray(label, dtype=np.int32)
    o = kura_default_opts()
    o.tau, o.precision, o.bitmap_zmin = float(tau), int(precision), float(bitmap_zmin)
    o.tensor_cores = int(tensor_cores)
    rc = load().kura_plan_build(int(n), row_ptr.ctypes.data, col.ctypes.data if col.size else None,
                                label.ctypes.data, int(n_comm), C.byref(o), C.byref(p))
    _check(rc, None)
    return p


def kura_plan_build_valued(n, row_ptr, col, val, label, n_comm, tau=0.5, precision=PREC_MIXED):
    p = C.c_void_p()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.int32)
    label = np.ascontiguousarray(label, dtype=np.int32)
    o = kura_default_opts()
    o.tau, o.precision = float(tau), int(precision)
    rc = load().kura_plan_build_valued(int(n), row_ptr.ctypes.data, col.ctypes.data if col.size else None,
                                       val.ctypes.data if val.size else None, label.ctypes.data, int(n_comm),
                                       C.byref(o), C.byref(p))
    _check(rc, None)
    return p


def kura_plan_dense_values(p, I) -> np.ndarray:
    cnt = C.c_int32()
    _check(load().kura_plan_dense_values(p, int(I), None, 0, C.byref(cnt)), None)
    out = np.zeros(max(cnt.value, 1), np.int32)
    _check(load().kura_plan_dense_values(p, int(I), out.ctypes.data, int(cnt.value), C.byref(cnt)), None)
    return out[:cnt.value]


def kura_plan_stats(p) -> dict:
    st = KuraBlockStats()
    _check(load().kura_plan_stats(p, C.byref(st)))
    return st.as_dict()


def kura_plan_perm(p, n, n_comm):
    perm = np.empty(n, dtype=np.int32)
    off = np.empty(n_comm + 1, dtype=np.int64)
    _check(load().kura_plan_perm(p, perm.ctypes.data, off.ctypes.data))
    return perm, off


def kura_plan_row(p, row, cap):
    miss = np.empty(max(cap, 1), dtype=np.int32)
    pres = np.empty(max(cap, 1), dtype=np.int32)
    nm, np_ = C.c_int64(), C.c_int64()
    _check(load().kura_plan_row(p, int(row), miss.ctypes.data, C.byref(nm), pres.ctypes.data, C.byref(np_),
                                int(cap)))
    return miss[:nm.value].copy(), pres[:np_.value].copy()


def kura_plan_dense_blocks(p, I, cap=1 << 16):
    buf = np.empty(cap, dtype=np.int32)
    cnt = C.c_int32()
    _check(load().kura_plan_dense_blocks(p, int(I), buf.ctypes.data, int(cap), C.byref(cnt)))
    return buf[:cnt.value].copy()


GROUP_DTYPE = np.dtype([("off", np.int64), ("len", np.int32), ("sub0", np.int32), ("nsub", np.int32),
                        ("pad", np.int32)])
TILE_DTYPE = np.dtype([("r0", np.int32), ("r1", np.int32), ("comm", np.int32), ("wbeg", np.int32),
                       ("wlen", np.int32), ("g0", np.int32), ("g1", np.int32), ("sub0", np.int32),
                       ("bm_off", np.int64), ("nsw", np.int32), ("flags", np.int32)])
TILE_BITMAP = 1
TILE_TC = 8
TILE_VALUED = 16
TC_KBLOCK = 128
TC_MBLOCK = 128


def kura_plan_export(p, n):
    """Copies of the packed stream, groups, tiles, row_sub0 and row bitmaps of a plan."""
    gs, gl, gr, ng, ti, nt, rs, bm, bl = (C.c_void_p(), C.c_int64(), C.c_void_p(), C.c_int64(), C.c_void_p(),
                                          C.c_int64(), C.c_void_p(), C.c_void_p(), C.c_int64())
    _check(load().kura_plan_export(p, C.byref(gs), C.byref(gl), C.byref(gr), C.byref(ng), C.byref(ti),
                                   C.byref(nt), C.byref(rs), C.byref(bm), C.byref(bl)))

    def view(ptr, count, dtype):
        if count == 0:
            return np.zeros(0, dtype=dtype)
        buf = (C.c_char * (count * np.dtype(dtype).itemsize)).from_address(ptr.value)
        return np.frombuffer(buf, dtype=dtype).copy()
    return (view(gs, gl.value, np.int32), view(gr, ng.value, GROUP_DTYPE), view(ti, nt.value, TILE_DTYPE),
            view(rs, n + 1, np.int32), view(bm, bl.value, np.uint32))


def kura_plan_destroy(p):
    load().kura_plan_destroy(p)


# ----------------------------------------------------------------------------- convenience wrapper
def kura_create_valued(n, row_ptr, col, val, label, n_comm, omega, K, opts: Optional[KuraOpts] = None, stream=None):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.int32)
    label = np.ascontiguousarray(label, dtype=np.int32)
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    if val.shape != col.shape:
        raise ValueError("val must match col")
    h = C.c_void_p()
    rc = load().kura_create_valued(int(n), row_ptr.ctypes.data, col.ctypes.data if col.size else None,
                                   val.ctypes.data if val.size else None, label.ctypes.data, int(n_comm),
                                   omega.ctypes.data, float(K), C.byref(opts) if opts is not None else None,
                                   stream or None, C.byref(h))
    _check(rc, None)
    return h


class Kuramoto:
    """A libkura handle: the graph, omega and K resident on the GPU.  val (optional, int32 1..127 parallel to
    col) makes the adjacency finite-valued (kura_create_valued)."""

    def __init__(self, row_ptr, col, label, n_comm, omega, K, precision=PREC_FP64,
                 scaling=SCALING_UNIFORM, tau=0.5, keep_host_csr=True, stream=None, bitmap_zmin=None,
                 tensor_cores=None, val=None, persistent_small=None, fused_trig=None):
        self.n = int(np.asarray(row_ptr).shape[0] - 1)
        self.n_comm = int(n_comm)
        o = kura_default_opts()
        o.precision, o.scaling, o.tau, o.keep_host_csr = int(precision), int(scaling), float(tau), int(keep_host_csr)
        if bitmap_zmin is not None:
            o.bitmap_zmin = float(bitmap_zmin)
        if tensor_cores is not None:
            o.tensor_cores = int(tensor_cores)
        if persistent_small is not None:
            o.persistent_small = int(persistent_small)
        if fused_trig is not None:
            o.fused_trig = int(fused_trig)
        if val is not None:
            self.h = kura_create_valued(self.n, row_ptr, col, val, label, n_comm, omega, K, o, stream)
        else:
            self.h = kura_create(self.n, row_ptr, col, label, n_comm, omega, K, o, stream)
        # the handle's current parameters (copies), so that callers can put them back
        self.omega = np.array(omega, dtype=np.float64)
        self.K = float(K)

    def rhs(self, theta, out):
        kura_rhs(self.h, theta, out, self.n)

    def rk4_steps(self, theta, step, n_steps):
        kura_rk4_steps(self.h, theta, step, n_steps, self.n)

    def order_params(self, theta, per_community=False):
        return kura_order_params(self.h, theta, self.n, self.n_comm, per_community)

    def set_param(self, omega=None, K=None):
        kura_set_param(self.h, omega, K, self.n)
        if omega is not None:
            self.omega = omega.clone() if hasattr(omega, "data_ptr") else np.array(omega, dtype=np.float64)
        if K is not None:
            self.K = float(K)

    def classify_blocks(self, tau=-1.0):
        return kura_classify_blocks(self.h, tau)

    def stats(self):
        return kura_get_stats(self.h)

    def integrate(self, theta, step, n_steps, method=INT_RK4, iters=4):
        """n_steps of RK4, explicit midpoint (INT_RK2) or implicit midpoint (INT_IMPLICIT_MIDPOINT, `iters`
        fixed-point sweeps of the stage) on theta in place."""
        kura_integrate(self.h, theta, step, n_steps, method, iters, self.n)

    def potential(self, theta):
        """Graph potential V (kura_potential)."""
        return kura_potential(self.h, theta, self.n)

    def mean_deviation(self, theta_t, theta_0, t):
        """(1/n) sum (theta_t - theta_0 - t omega) (kura_mean_deviation)."""
        return kura_mean_deviation(self.h, theta_t, theta_0, t, self.n)

    def autotune(self, theta, budget_s=30.0):
        """Times the right-hand side at theta for candidate plans and keeps the fastest (see kura_autotune)."""
        return kura_autotune(self.h, theta, self.n, budget_s)

    def adjoint(self, theta0, step, n_steps, ckpt_every=64, loss_kind=0, target=None, g_omega=None, g_theta0=None):
        """Loss and gradients (loss, g_omega, g_K, g_theta0) of the RK4 trajectory from theta0."""
        import torch
        if g_omega is None:
            g_omega = torch.empty_like(theta0) if hasattr(theta0, "data_ptr") else np.empty(self.n)
        if g_theta0 is None:
            g_theta0 = torch.empty_like(theta0) if hasattr(theta0, "data_ptr") else np.empty(self.n)
        loss, gK = kura_adjoint(self.h, theta0, step, n_steps, ckpt_every, loss_kind, target, g_omega, g_theta0,
                                self.n)
        return loss, g_omega, gK, g_theta0

    def direct_rhs(self, theta, out, precision=PREC_FP64):
        kura_direct_rhs(self.h, theta, out, precision, self.n)

    def direct_rk4_steps(self, theta, step, n_steps, precision=PREC_FP64):
        kura_direct_rk4_steps(self.h, theta, step, n_steps, precision, self.n)

    def set_timing(self, on=True):
        kura_set_timing(self.h, on)

    def kernel_times(self, cap=4096):
        return kura_kernel_times(self.h, cap)

    def sync(self):
        kura_sync(self.h)

    def close(self):
        if getattr(self, "h", None):
            kura_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kura_ensemble_create(n, row_ptr, col, label, n_comm, omega, K, opts: Optional[KuraOpts] = None, stream=None):
    """omega: (n_traj, n) array, K: (n_traj,) array; n_traj a multiple of 16."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    label = np.ascontiguousarray(label, dtype=np.int32)
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    K = np.ascontiguousarray(K, dtype=np.float64)
    n_traj = int(K.shape[0])
    if omega.shape != (n_traj, int(n)):
        raise ValueError("omega must have shape (n_traj, n)")
    h = C.c_void_p()
    rc = load().kura_ensemble_create(int(n), row_ptr.ctypes.data, col.ctypes.data if col.size else None,
                                     label.ctypes.data, int(n_comm), n_traj, omega.ctypes.data, K.ctypes.data,
                                     C.byref(opts) if opts is not None else None, stream or None, C.byref(h))
    _check(rc, None)
    return h


class KuramotoEnsemble:
    """Trajectories sharing one graph (own omega and K each): phases are (n_traj, n) arrays or tensors."""

    def __init__(self, row_ptr, col, label, n_comm, omega, K, tau=0.5, tensor_cores=1, stream=None):
        self.n = int(np.asarray(row_ptr).shape[0] - 1)
        self.n_traj = int(np.asarray(K).shape[0])
        o = kura_default_opts()
        o.precision, o.tau, o.tensor_cores = PREC_MIXED, float(tau), int(tensor_cores)
        self.h = kura_ensemble_create(self.n, row_ptr, col, label, n_comm, omega, K, o, stream)

    def rhs(self, theta, out):
        kura_rhs(self.h, theta, out, self.n * self.n_traj)

    def rk4_steps(self, theta, step, n_steps):
        kura_rk4_steps(self.h, theta, step, n_steps, self.n * self.n_traj)

    def stats(self):
        return kura_get_stats(self.h)

    def sync(self):
        kura_sync(self.h)

    def close(self):
        if getattr(self, "h", None):
            kura_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class KuramotoBatch:
    """A batch handle: independent trajectories (own graph, omega, K) integrated by one persistent launch.
    Phases are passed concatenated in trajectory order; `offsets[t]:offsets[t+1]` is trajectory t."""

    def __init__(self, graphs, tau=0.5, stream=None, precision=PREC_MIXED, tensor_cores=0, row_lanes=32):
        o = kura_default_opts()
        o.precision, o.tau, o.tensor_cores = int(precision), float(tau), int(tensor_cores)
        o.row_lanes = int(row_lanes)
        self.h, self.offsets = kura_batch_create(graphs, o, stream)
        self.n = int(self.offsets[-1])

    def rk4_steps(self, theta, step, n_steps):
        kura_rk4_steps(self.h, theta, step, n_steps, self.n)

    def rhs(self, theta, out):
        """Right-hand sides of every trajectory at theta (concatenated) into out."""
        kura_rhs(self.h, theta, out, self.n)

    def stats(self):
        return kura_batch_stats(self.h)

    def info(self):
        return kura_batch_info(self.h)

    def traj_params(self, t):
        """(tau, tensor_cores, row_lanes) of trajectory t."""
        tau, tc, lanes = C.c_double(), C.c_int32(), C.c_int32()
        _check(load().kura_batch_traj_params(self.h, int(t), C.byref(tau), C.byref(tc), C.byref(lanes)), self.h)
        return tau.value, tc.value, lanes.value

    def autotune(self, theta, budget_s=60.0):
        """Per size class: the fastest of the dense-zero encodings, row tiles and tau (see kura_autotune)."""
        return kura_autotune(self.h, theta, self.n, budget_s)

    def set_timing(self, on=True):
        kura_set_timing(self.h, on)

    def kernel_times(self, cap=16):
        return kura_kernel_times(self.h, cap)

    def sync(self):
        kura_sync(self.h)

    def close(self):
        if getattr(self, "h", None):
            kura_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
