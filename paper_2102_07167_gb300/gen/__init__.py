"""Seeded synthetic inputs (graphs, frequencies, phases) for the workloads.

This module draws inputs only; it holds none of the model's arithmetic, and
both the CUDA library's tests and the CPU oracle take their inputs from it.
The draws are implemented in ``synth.c`` (compiled with gcc + OpenMP on first
use); every value is a pure function of (seed, stream, index), independent of
the thread count.

Workload recipes (sizes and distributions of the paper's experiments, Sec. 2
"Numerical integration" and Sec. 3 block-matrix experiments, at the scales
of the benchmark configurations):

* ``complete(n)``: all-to-all graph without self-loops (classical model).
* ``sbm(...)``: stochastic block model, symmetric 0/1, no self-loops,
  community sizes ``min_size`` + Dirichlet(alpha) split (optionally clipped at
  ``max_size``), per-community intra probability, one inter probability,
  randomly relabelled so that the community structure is hidden in the user
  numbering; the planted labels are returned for re-blocking.
* ``paper_e2_inputs(M, omega0)``: the deterministic frequencies and phases
  of the paper's classical experiments, omega_m = 1 + omega0 (2m - M - 1)/(M - 1),
  theta_m(0) = 2 pi m / M, m = 1..M.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "_synth.so")
_lock = threading.Lock()
_lib = None

_d = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            U64, I64, I32, D = C.c_uint64, C.c_int64, C.c_int32, C.c_double
            L.syn_dirichlet_sizes.argtypes = [U64, I64, I32, I32, I64, I64, _i64]
            L.syn_dirichlet_sizes.restype = C.c_int
            L.syn_permutation.argtypes = [U64, I64, _i32]
            L.syn_pin_uniform.argtypes = [U64, I32, D, D, _d]
            L.syn_sbm_csr.argtypes = [U64, I64, I32, _i64, _d, D, _i32, _i64, C.c_void_p]
            L.syn_sbm_csr.restype = C.c_int64
            L.syn_uniform.argtypes = [U64, U64, I64, D, D, _d]
            L.syn_normal.argtypes = [U64, U64, I64, D, D, _d]
            L.syn_cauchy.argtypes = [U64, U64, I64, D, D, D, _d]
            _lib = L
        return _lib


# ---------------------------------------------------------------- per-node draws
def uniform(seed: int, tag: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    out = np.empty(n)
    _load().syn_uniform(seed, tag, n, lo, hi, out)
    return out


def normal(seed: int, tag: int, n: int, mu: float = 0.0, sigma: float = 1.0) -> np.ndarray:
    out = np.empty(n)
    _load().syn_normal(seed, tag, n, mu, sigma, out)
    return out


def cauchy(seed: int, tag: int, n: int, loc: float = 0.0, scale: float = 1.0, clip: float = 0.0) -> np.ndarray:
    out = np.empty(n)
    _load().syn_cauchy(seed, tag, n, loc, scale, clip, out)
    return out


def permutation(seed: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.int32)
    _load().syn_permutation(seed, n, out)
    return out


def dirichlet_sizes(seed: int, n: int, n_comm: int, alpha: int = 2, min_size: int = 0,
                    max_size: int = 0) -> np.ndarray:
    out = np.empty(n_comm, dtype=np.int64)
    rc = _load().syn_dirichlet_sizes(seed, n, n_comm, alpha, min_size, max_size, out)
    if rc != 0:
        raise ValueError("community size bounds cannot be met")
    return out


def pin_uniform(seed: int, n_comm: int, lo: float, hi: float) -> np.ndarray:
    out = np.empty(n_comm)
    _load().syn_pin_uniform(seed, n_comm, lo, hi, out)
    return out


# ---------------------------------------------------------------- graphs
@dataclass
class Graph:
    n: int
    row_ptr: np.ndarray          # int64[n+1]
    col: np.ndarray              # int32[nnz], sorted per row, user numbering
    label: np.ndarray            # int32[n], planted community of each user node
    n_comm: int
    sizes: np.ndarray = field(default=None)   # int64[n_comm]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def complete(n: int) -> Graph:
    """All-to-all graph without self-loops; one community."""
    row_ptr = np.arange(n + 1, dtype=np.int64) * (n - 1)
    cols = np.tile(np.arange(n, dtype=np.int32), (n, 1))
    mask = ~np.eye(n, dtype=bool)
    col = cols[mask].astype(np.int32)
    return Graph(n, row_ptr, col, np.zeros(n, dtype=np.int32), 1, np.array([n], dtype=np.int64))


def sbm(seed: int, sizes, p_in, p_out: float, relabel: bool = True) -> Graph:
    """Symmetric SBM with the given community sizes (see module docstring)."""
    sizes = np.ascontiguousarray(sizes, dtype=np.int64)
    n_comm = sizes.shape[0]
    n = int(sizes.sum())
    off = np.zeros(n_comm + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    p_in = np.ascontiguousarray(np.broadcast_to(np.asarray(p_in, dtype=np.float64), (n_comm,)))
    sigma = permutation(seed + 7919, n) if relabel else np.arange(n, dtype=np.int32)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    L = _load()
    nnz = L.syn_sbm_csr(seed, n, n_comm, off, p_in, float(p_out), sigma, row_ptr, None)
    if nnz < 0:
        raise RuntimeError("SBM generation failed")
    col = np.empty(max(nnz, 1), dtype=np.int32)
    if L.syn_sbm_csr(seed, n, n_comm, off, p_in, float(p_out), sigma, row_ptr, col.ctypes.data) != nnz:
        raise RuntimeError("SBM generation failed")
    col = col[:nnz]
    planted = np.repeat(np.arange(n_comm, dtype=np.int32), sizes)
    label = np.empty(n, dtype=np.int32)
    label[sigma] = planted
    return Graph(n, row_ptr, col, label, n_comm, sizes)


def from_dense(A: np.ndarray, label=None, n_comm: int = 1) -> Graph:
    """CSR of a dense 0/1 matrix (rows sorted); diagonal kept as given."""
    A = np.asarray(A)
    n = A.shape[0]
    rows, cols = np.nonzero(A)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    lab = np.zeros(n, dtype=np.int32) if label is None else np.asarray(label, dtype=np.int32)
    return Graph(n, row_ptr.astype(np.int64), cols.astype(np.int32), lab,
                 int(n_comm if label is None else max(n_comm, int(lab.max()) + 1)), None)


def paper_e2_inputs(M: int, omega0: float):
    """omega_m = 1 + omega0 (2m - M - 1)/(M - 1), theta_m(0) = 2 pi m / M (m = 1..M)."""
    m = np.arange(1, M + 1, dtype=np.float64)
    omega = 1.0 + omega0 * (2.0 * m - M - 1.0) / (M - 1.0)
    theta0 = 2.0 * np.pi * m / M
    return omega, theta0


# ---------------------------------------------------------------- workloads
@dataclass
class Workload:
    name: str
    graph: Graph
    omega: np.ndarray
    theta0: np.ndarray
    K: float
    h: float
    n_steps: int


def workload_complete(n: int = 512, seed: int = 0) -> Workload:
    """Classical all-to-all model: omega ~ N(0,1), theta0 ~ U[0, 2pi), K = 2, h = 0.01, 200 steps."""
    g = complete(n)
    return Workload(f"complete-{n}", g, normal(seed, 0, n), uniform(seed, 1, n, 0.0, 2 * np.pi), 2.0, 0.01, 200)


def workload_sbm_small(n: int = 65536, n_comm: int = 64, min_size: int = 128, seed: int = 0) -> Workload:
    """SBM, Dirichlet(2) sizes (min 128), p_in 0.95, p_out 0.001; omega ~ N(0,1), theta0 ~ U[0,2pi),
    K = 4, h = 0.005, 1000 steps."""
    sizes = dirichlet_sizes(seed, n, n_comm, 2, min_size, 0)
    g = sbm(seed, sizes, 0.95, 0.001)
    return Workload(f"sbm-{n}", g, normal(seed, 0, n), uniform(seed, 1, n, 0.0, 2 * np.pi), 4.0, 0.005, 1000)


def workload_sbm_large(n: int = 1 << 20, n_comm: int = 1024, min_size: int = 256, max_size: int = 4096,
                       p_out: float = 1e-4, seed: int = 0) -> Workload:
    """Large SBM: Dirichlet(2) sizes clipped to [256, 4096], p_in ~ U[0.5, 0.99] per community,
    p_out = 1e-4; omega ~ Cauchy(0, 0.5) clipped at +-10, theta0 ~ U[0, 2pi), K = 3, h = 0.01, 500 steps."""
    sizes = dirichlet_sizes(seed, n, n_comm, 2, min_size, max_size)
    p_in = pin_uniform(seed, n_comm, 0.5, 0.99)
    g = sbm(seed, sizes, p_in, p_out)
    return Workload(f"sbm-{n}", g, cauchy(seed, 0, n, 0.0, 0.5, 10.0), uniform(seed, 1, n, 0.0, 2 * np.pi),
                    3.0, 0.01, 500)


def workload_batch(n_traj: int = 2048, seed: int = 0, n_min: int = 256, n_max: int = 16384):
    """Ensemble of independent trajectories: sizes log-uniform in [n_min, n_max], even-indexed complete
    graphs (returned as None: the all-to-all graph needs no adjacency) and odd-indexed SBMs (8-32
    communities, p_in 0.9, p_out 0.005, Dirichlet(2) sizes with a floor of min(16, n / (2 C))); per
    trajectory omega ~ N(0,1), theta0 ~ U[0, 2pi), K ~ U[0.5, 5].  Returns a list of (graph or None, n,
    omega, theta0, K)."""
    u = uniform(seed, 11, n_traj)
    sizes_n = np.floor(np.exp(np.log(n_min) + u * (np.log(n_max) - np.log(n_min)))).astype(np.int64)
    Ks = uniform(seed, 12, n_traj, 0.5, 5.0)
    ncs = np.floor(8 + uniform(seed, 13, n_traj) * 25).astype(np.int64)        # 8..32
    out = []
    for t in range(n_traj):
        n = int(sizes_n[t])
        if t % 2 == 0:
            g = None
        else:
            c = int(min(ncs[t], max(1, n // 16)))
            mn = int(min(16, n // (2 * c)))
            g = sbm(seed + 1000 + t, dirichlet_sizes(seed + 1000 + t, n, c, 2, mn, 0), 0.9, 0.005)
        out.append((g, n, normal(seed + t, 21, n), uniform(seed + t, 22, n, 0.0, 2 * np.pi), float(Ks[t])))
    return out


def batch_graphs(ens):
    """(row_ptr, col, label, n_comm, omega, K) tuples of an ensemble for the batch API."""
    return [((None, None, None, 1, om, K) if g is None else (g.row_ptr, g.col, g.label, g.n_comm, om, K))
            for (g, n, om, th, K) in ens]
