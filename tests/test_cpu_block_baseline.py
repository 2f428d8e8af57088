"""The OpenMP CPU block method that bench.py reports as the all-cores CPU baseline computes the same
right-hand side and RK4 trajectory as the FP64 oracle (eq:KuramotoGraph by eq:KuramotoGraphApproach)."""
import numpy as np

import bench
import oracle
from _parity import check_rhs
from paper_2102_07167_gb300 import gen as G


def test_cpu_block_rhs_and_rk4_match_oracle():
    w = G.workload_sbm_small(n=6000, n_comm=8, min_size=128, seed=11)
    g = w.graph
    th = w.theta0 + 20.0 * G.uniform(3, 4, g.n, -1, 1)
    cb = bench.CpuBlock(g, w.omega, w.K)
    try:
        f = cb.rhs(th)
        ref = oracle.rhs_csr(g.row_ptr, g.col, w.omega, th, w.K)
        check_rhs(f, ref, np.diff(g.row_ptr), w.K, g.n, 0, "cpu block method")
        y = w.theta0.copy()
        cb.rk4(y, w.h, 5)
    finally:
        cb.close()
    ref_t = oracle.rk4_csr(g.row_ptr, g.col, w.omega, w.K, w.theta0, w.h, 5)
    assert np.abs(y - ref_t).max() <= 1e-10


def test_cpu_block_complete_graph():
    w = G.workload_complete(300)
    cb = bench.CpuBlock(w.graph, w.omega, w.K)
    try:
        f = cb.rhs(w.theta0)
    finally:
        cb.close()
    ref = oracle.rhs_complete_op(w.omega, w.theta0, w.K)
    check_rhs(f, ref, np.full(300, 299), w.K, 300, 0, "cpu block method, complete graph")
