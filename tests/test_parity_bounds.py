"""CPU pins of the parity bounds in tests/_parity.py (no GPU).

The scale-free bound e_i = |f_i - o_i| / ((K/calM_i)(1 + deg_i)) must
(a) be attainable by the precision design: an FP32 emulation of the mixed
    right-hand side (FP32 sin/cos of the phase reduced mod 2 pi, every listed
    entry summed in FP32, FP64 epilogue) stays below E_MIXED, and two FP64
    evaluation routes of the oracle stay far below E_FP64;
(b) have teeth where the stated mixed tolerance has none: a right-hand side
    whose coupling is off by 1e-4 of itself, or that drops one edge, passes
    the stated 2e-4 (1 + deg_i) max(1, |o_i|) bound and fails the scale-free
    one.
The graph is the 65536-node SBM (K = 4, N = 65536, rows of ~1000 entries);
e_i is independent of N, so the same margins hold at 2^20 nodes.
"""
import numpy as np
import pytest

import oracle
from _parity import E_FP64, E_MIXED, scale_free_error, stated_tolerance
from paper_2102_07167_gb300 import gen as G


@pytest.fixture(scope="module")
def case():
    w = G.workload_sbm_small()
    g = w.graph
    rows = np.unique(G.permutation(5, g.n)[:1500].astype(np.int64))
    ref = oracle.rhs_csr(g.row_ptr, g.col, w.omega, w.theta0, w.K, rows=rows)
    return w, rows, ref


def _mixed_emulation(w, rows):
    g = w.graph
    th = w.theta0
    red = (th - 2 * np.pi * np.rint(th / (2 * np.pi))).astype(np.float32)
    s32, c32 = np.sin(red), np.cos(red)
    f = np.empty(rows.shape[0])
    for k, i in enumerate(rows):
        nb = g.col[g.row_ptr[i]:g.row_ptr[i + 1]]
        acc_s = float(np.cumsum(s32[nb], dtype=np.float32)[-1]) if nb.size else 0.0
        acc_c = float(np.cumsum(c32[nb], dtype=np.float32)[-1]) if nb.size else 0.0
        f[k] = w.omega[i] + w.K / g.n * (np.cos(th[i]) * acc_s - np.sin(th[i]) * acc_c)
    return f


def test_mixed_emulation_meets_scale_free_bound(case):
    w, rows, ref = case
    f = _mixed_emulation(w, rows)
    deg = np.diff(w.graph.row_ptr)[rows]
    e = scale_free_error(f, ref, w.K, w.graph.n, deg)
    assert np.all(np.abs(f - ref) <= stated_tolerance(ref, deg, 1))
    assert e.max() <= E_MIXED / 5, e.max()          # at least 5x margin under the bound


def test_fp64_routes_meet_scale_free_bound():
    w = G.workload_sbm_small(n=3000, n_comm=6, min_size=128, seed=7)
    g = w.graph
    f_csr = oracle.rhs_csr(g.row_ptr, g.col, w.omega, w.theta0, w.K)
    f_blk, _ = oracle.rhs_block(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.theta0, w.K)
    e = scale_free_error(f_blk, f_csr, w.K, g.n, np.diff(g.row_ptr))
    assert e.max() <= E_FP64 / 100, e.max()


def test_perturbed_coupling_passes_stated_tolerance_but_not_scale_free(case):
    w, rows, ref = case
    deg = np.diff(w.graph.row_ptr)[rows]
    bad = ref + 1e-4 * (ref - w.omega[rows])
    assert np.all(np.abs(bad - ref) <= stated_tolerance(ref, deg, 1))
    assert scale_free_error(bad, ref, w.K, w.graph.n, deg).max() > E_MIXED


def test_dropped_edge_passes_stated_tolerance_but_not_scale_free(case):
    w, rows, ref = case
    g = w.graph
    th = w.theta0
    i = int(rows[len(rows) // 2])
    nb = g.col[g.row_ptr[i]:g.row_ptr[i + 1]]
    # the edge with the largest |sin(theta_j - theta_i)| of that row
    j = int(nb[np.argmax(np.abs(np.sin(th[nb] - th[i])))])
    k = int(np.searchsorted(rows, i))
    bad = ref.copy()
    bad[k] -= w.K / g.n * np.sin(th[j] - th[i])
    deg = np.diff(g.row_ptr)[rows]
    assert np.all(np.abs(bad - ref) <= stated_tolerance(ref, deg, 1))
    assert scale_free_error(bad, ref, w.K, g.n, deg).max() > E_MIXED
