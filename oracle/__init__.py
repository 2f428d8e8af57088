"""FP64 CPU oracle for the Kuramoto model on graphs (arXiv 2102.07167).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product library.  It
shares no code with the CUDA path.  The arithmetic lives in ``kura_oracle.c``
(plain C, single thread); this module only compiles it with gcc on first use
and marshals numpy arrays through ctypes.

Paper passages followed (see the C file for the per-function citations):
eq:Kuramoto, eq:KuramotoReformulation, eq:EulerCost, eq:OrderParameter,
eq:Potential, eq:Means (Sec. 2); eq:KuramotoGraph,
eq:KuramotoGraphApproach, eq:ExtendedPotentialConservation (Sec. 3).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kura_oracle.c")
_LIB = os.path.join(_HERE, "_kura_oracle.so")
_lock = threading.Lock()
_lib = None

_d = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile kura_oracle.c into _kura_oracle.so (gcc -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        L = C.CDLL(_LIB)
        I64, I32, D = C.c_int64, C.c_int32, C.c_double
        L.orc_rhs_dense.argtypes = [I64, _u8, _d, _d, D, C.c_int, _d]
        L.orc_rhs_csr.argtypes = [I64, _i64, _i32, _d, _d, D, C.c_int, _d]
        L.orc_rhs_csr_rows.argtypes = [I64, _i64, _i32, _d, _d, D, C.c_int, _i64, I64, _d]
        L.orc_rhs_complete_op.argtypes = [I64, _d, _d, D, _d]
        L.orc_rhs_block.argtypes = [I64, _i64, _i32, _i32, I32, _d, _d, D, C.c_int, D, _d, _i64]
        L.orc_rk4_csr.argtypes = [I64, _i64, _i32, _d, D, C.c_int, _d, D, I64]
        L.orc_rk4_complete.argtypes = [I64, _d, D, _d, D, I64]
        L.orc_order_params.argtypes = [I64, _d, C.POINTER(D), C.POINTER(D), C.c_void_p, I32,
                                       C.c_void_p, C.c_void_p]
        L.orc_potential_csr.argtypes = [I64, _i64, _i32, _d, _d, D, C.c_int, C.POINTER(D)]
        L.orc_mean_deviation.argtypes = [I64, _d, _d, _d, D, C.POINTER(D)]
        L.orc_adjoint_rk4_csr.argtypes = [I64, _i64, _i32, _d, D, C.c_int, _d, D, I64, C.c_int, C.c_void_p,
                                          C.POINTER(D), _d, C.POINTER(D), _d]
        L.orc_rk2_csr.argtypes = [I64, _i64, _i32, _d, D, C.c_int, _d, D, I64, C.c_int, C.c_int]
        L.orc_rhs_valued_csr.argtypes = [I64, _i64, _i32, _i32, _d, _d, D, _d]
        L.orc_rhs_valued_dense.argtypes = [I64, _i32, _d, _d, D, _d]
        L.orc_rhs_block_valued.argtypes = [I64, _i64, _i32, _i32, I32, _i32, I32, _d, _d, D, D, _d, C.c_void_p]
        L.orc_trig_count.restype = C.c_int64
        for f in ("orc_rhs_dense", "orc_rhs_csr", "orc_rhs_csr_rows", "orc_rhs_complete_op",
                  "orc_rhs_block", "orc_rk4_csr", "orc_rk4_complete", "orc_order_params",
                  "orc_potential_csr", "orc_mean_deviation", "orc_adjoint_rk4_csr", "orc_rk2_csr",
                  "orc_rhs_valued_csr", "orc_rhs_valued_dense", "orc_rhs_block_valued"):
            getattr(L, f).restype = C.c_int
        _lib = L
        return L


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def trig_count() -> int:
    return int(_load().orc_trig_count())


def trig_count_reset() -> None:
    _load().orc_trig_count_reset()


def rhs_dense(A, omega, theta, K, scaling=0):
    """eq:KuramotoGraph by brute force over a dense 0/1 matrix."""
    A = np.ascontiguousarray(A, dtype=np.uint8)
    n = A.shape[0]
    out = np.empty(n)
    _check(_load().orc_rhs_dense(n, A, _f64(omega), _f64(theta), float(K), int(scaling), out), "rhs_dense")
    return out


def rhs_csr(row_ptr, col, omega, theta, K, scaling=0, rows=None):
    """eq:KuramotoGraph over CSR edges (all rows, or the listed rows)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = row_ptr.shape[0] - 1
    L = _load()
    if rows is None:
        out = np.empty(n)
        _check(L.orc_rhs_csr(n, row_ptr, col, _f64(omega), _f64(theta), float(K), int(scaling), out), "rhs_csr")
        return out
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty(rows.shape[0])
    _check(L.orc_rhs_csr_rows(n, row_ptr, col, _f64(omega), _f64(theta), float(K), int(scaling),
                              rows, rows.shape[0], out), "rhs_csr_rows")
    return out


def rhs_complete_op(omega, theta, K):
    """Classical model via the precomputed sums S_M, C_M (eq:KuramotoReformulation)."""
    theta = _f64(theta)
    out = np.empty(theta.shape[0])
    _check(_load().orc_rhs_complete_op(theta.shape[0], _f64(omega), theta, float(K), out), "rhs_complete_op")
    return out


def rhs_block(row_ptr, col, label, n_comm, omega, theta, K, scaling=0, tau=0.5):
    """Block rule of eq:KuramotoGraphApproach.  Returns (f, stats dict)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    n = row_ptr.shape[0] - 1
    out = np.empty(n)
    st = np.zeros(6, dtype=np.int64)
    _check(_load().orc_rhs_block(n, row_ptr, np.ascontiguousarray(col, dtype=np.int32),
                                 np.ascontiguousarray(label, dtype=np.int32), int(n_comm),
                                 _f64(omega), _f64(theta), float(K), int(scaling), float(tau), out, st),
           "rhs_block")
    keys = ("dense_blocks", "sparse_blocks", "zero_terms", "nonzero_terms", "blocks", "trig_evals")
    return out, dict(zip(keys, (int(v) for v in st)))


def rk4_csr(row_ptr, col, omega, K, theta0, h, n_steps, scaling=0):
    """Classical fixed-step RK4 with the CSR definition as right-hand side."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    th = _f64(theta0).copy()
    _check(_load().orc_rk4_csr(row_ptr.shape[0] - 1, row_ptr, np.ascontiguousarray(col, dtype=np.int32),
                               _f64(omega), float(K), int(scaling), th, float(h), int(n_steps)), "rk4_csr")
    return th


def rhs_valued_csr(row_ptr, col, val, omega, theta, K):
    """Finite-valued A (Sec. 1, Generalisations): omega + (K/n) sum_l A_ml sin(theta_l - theta_m)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    out = np.empty(row_ptr.shape[0] - 1)
    _check(_load().orc_rhs_valued_csr(row_ptr.shape[0] - 1, row_ptr, np.ascontiguousarray(col, dtype=np.int32),
                                      np.ascontiguousarray(val, dtype=np.int32), _f64(omega), _f64(theta),
                                      float(K), out), "rhs_valued_csr")
    return out


def rhs_valued_dense(A, omega, theta, K):
    """The same by brute force over a dense int32 matrix."""
    A = np.ascontiguousarray(A, dtype=np.int32)
    out = np.empty(A.shape[0])
    _check(_load().orc_rhs_valued_dense(A.shape[0], A, _f64(omega), _f64(theta), float(K), out), "rhs_valued_dense")
    return out


def rhs_block_valued(row_ptr, col, val, max_val, label, n_comm, omega, theta, K, tau=0.5):
    """Prevalent-value block rule for finite-valued A.  Returns (f, block values [n_comm, n_comm])."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    n = row_ptr.shape[0] - 1
    out = np.empty(n)
    bv = np.zeros((n_comm, n_comm), np.int32)
    _check(_load().orc_rhs_block_valued(n, row_ptr, np.ascontiguousarray(col, dtype=np.int32),
                                        np.ascontiguousarray(val, dtype=np.int32), int(max_val),
                                        np.ascontiguousarray(label, dtype=np.int32), int(n_comm), _f64(omega),
                                        _f64(theta), float(K), float(tau), out, bv.ctypes.data), "rhs_block_valued")
    return out, bv


def rk2_csr(row_ptr, col, omega, K, theta0, h, n_steps, method=0, iters=4, scaling=0):
    """Second-order integrators: method 0 explicit midpoint, 1 implicit midpoint (`iters` fixed-point
    sweeps of the stage from the explicit predictor)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    th = _f64(theta0).copy()
    _check(_load().orc_rk2_csr(row_ptr.shape[0] - 1, row_ptr, np.ascontiguousarray(col, dtype=np.int32),
                               _f64(omega), float(K), int(scaling), th, float(h), int(n_steps), int(method),
                               int(iters)), "rk2_csr")
    return th


def rk4_complete(omega, K, theta0, h, n_steps):
    """Classical all-to-all model, RK4, order-parameter right-hand side."""
    th = _f64(theta0).copy()
    _check(_load().orc_rk4_complete(th.shape[0], _f64(omega), float(K), th, float(h), int(n_steps)),
           "rk4_complete")
    return th


def order_params(theta, label=None, n_comm=0):
    """eq:OrderParameter.  Returns (r, psi) or (r, psi, r_comm, psi_comm)."""
    theta = _f64(theta)
    r, psi = C.c_double(), C.c_double()
    L = _load()
    if label is None:
        _check(L.orc_order_params(theta.shape[0], theta, C.byref(r), C.byref(psi), None, 0, None, None),
               "order_params")
        return r.value, psi.value
    lab = np.ascontiguousarray(label, dtype=np.int32)
    rc_ = np.empty(n_comm)
    pc_ = np.empty(n_comm)
    _check(L.orc_order_params(theta.shape[0], theta, C.byref(r), C.byref(psi),
                              lab.ctypes.data, int(n_comm), rc_.ctypes.data, pc_.ctypes.data),
           "order_params")
    return r.value, psi.value, rc_, pc_


def potential_csr(row_ptr, col, omega, theta, K, scaling=0):
    """Graph potential, eq:ExtendedPotentialConservation."""
    V = C.c_double()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    _check(_load().orc_potential_csr(row_ptr.shape[0] - 1, row_ptr, np.ascontiguousarray(col, dtype=np.int32),
                                     _f64(omega), _f64(theta), float(K), int(scaling), C.byref(V)),
           "potential_csr")
    return V.value


def mean_deviation(theta_t, theta_0, omega, t):
    """eq:Means."""
    v = C.c_double()
    theta_t = _f64(theta_t)
    _check(_load().orc_mean_deviation(theta_t.shape[0], theta_t, _f64(theta_0), _f64(omega), float(t),
                                      C.byref(v)), "mean_deviation")
    return v.value


def adjoint_rk4_csr(row_ptr, col, omega, K, theta0, h, n_steps, loss_kind=0, target=None, scaling=0):
    """Discrete adjoint of RK4 for L = 1 - r(theta(T)) (loss_kind 0) or 1/2 ||theta(T) - target||^2 (1).
    Returns (L, dL/domega, dL/dK, dL/dtheta0)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    n = row_ptr.shape[0] - 1
    loss, gK = C.c_double(), C.c_double()
    g_om, g_th = np.empty(n), np.empty(n)
    tgt = None if target is None else _f64(target)
    _check(_load().orc_adjoint_rk4_csr(n, row_ptr, np.ascontiguousarray(col, dtype=np.int32), _f64(omega),
                                       float(K), int(scaling), _f64(theta0), float(h), int(n_steps),
                                       int(loss_kind), None if tgt is None else tgt.ctypes.data,
                                       C.byref(loss), g_om, C.byref(gK), g_th), "adjoint_rk4_csr")
    return loss.value, g_om, gK.value, g_th


def loss_rk4_csr(row_ptr, col, omega, K, theta0, h, n_steps, loss_kind=0, target=None, scaling=0):
    """Forward loss only (for finite differences)."""
    th = rk4_csr(row_ptr, col, omega, K, theta0, h, n_steps, scaling)
    if loss_kind == 0:
        return 1.0 - order_params(th)[0]
    return 0.5 * float(np.sum((th - np.asarray(target)) ** 2))
