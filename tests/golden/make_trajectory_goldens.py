"""Writes the FP64 trajectory goldens of the SBM workloads from the CPU oracle.

The expected phases come from ``oracle.rk4_csr`` only: classical fixed-step
RK4 (tableau 1/2, 1/2, 1; weights 1/6, 1/3, 1/3, 1/6) on eq:KuramotoGraph
(Sec. 3) with uniform scaling K/N, the right-hand side evaluated by the CSR
definition with one sine per edge and compensated sums.  The inputs come
from the seeded generators in ``paper_2102_07167_gb300.gen`` (which draw
inputs and hold none of the model's arithmetic).  Nothing here touches the
CUDA library.

The full trajectories take the single-threaded oracle minutes to hours, far
longer than a test may take, so each case stores theta(T) at a fixed random
sample of nodes, with a fingerprint of the inputs (SHA-256 of the CSR arrays,
sums of omega and theta0) that the GPU test checks before it compares.

Cases:
  sbm65536_1000   65536-node SBM (64 communities, Dirichlet(2) sizes with
                  minimum 128, p_in 0.95, p_out 0.001), K = 4, h = 0.005,
                  1000 steps (T = 5), seed 0
  sbm2p16_500     the 2^20-node recipe at N = 2^16 (64 communities, sizes
                  clipped to [256, 4096], p_in ~ U[0.5, 0.99], p_out 1e-4,
                  omega ~ Cauchy(0, 0.5) clipped at 10), K = 3, h = 0.01,
                  500 steps (T = 5), seed 0
  sbm2p20_10      the 2^20-node SBM itself (1024 communities), 10 steps of
                  h = 0.01, seed 0

  adjoint_sbm65536_4
                  the discrete RK4 adjoint (oracle.adjoint_rk4_csr: FP64, CSR
                  definition) of L = 1 - r(T) on the 65536-node SBM above
                  with h = 0.01 over 4 steps: L, dL/dK and dL/dtheta0,
                  dL/domega at the sampled nodes, and the gradient norms

Usage: python tests/golden/make_trajectory_goldens.py CASE [CASE ...]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_SAMPLE = 2048
SAMPLE_SEED = 20210215


def workload(case: str):
    from paper_2102_07167_gb300 import gen as G
    if case == "sbm65536_1000":
        return G.workload_sbm_small(), 0.005, 1000
    if case == "sbm2p16_500":
        return G.workload_sbm_large(n=1 << 16, n_comm=64), 0.01, 500
    if case == "sbm2p20_10":
        return G.workload_sbm_large(), 0.01, 10
    raise ValueError(f"unknown case {case}")


def fingerprint(w) -> dict:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(w.graph.row_ptr, dtype="<i8").tobytes())
    h.update(np.ascontiguousarray(w.graph.col, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(w.graph.label, dtype="<i4").tobytes())
    return {"n": int(w.graph.n), "nnz": int(w.graph.nnz), "n_comm": int(w.graph.n_comm),
            "graph_sha256": h.hexdigest(), "omega_sum": float(np.sum(w.omega)),
            "omega_abs_sum": float(np.sum(np.abs(w.omega))), "theta0_sum": float(np.sum(w.theta0))}


def sample_nodes(n: int) -> np.ndarray:
    return np.sort(np.random.default_rng(SAMPLE_SEED).choice(n, size=min(N_SAMPLE, n), replace=False))


def path(case: str) -> str:
    return os.path.join(HERE, f"traj_{case}_fp64.json")


ADJOINT_CASES = {"adjoint_sbm65536_4": (0.01, 4)}


def make_adjoint(case: str) -> None:
    import oracle
    from paper_2102_07167_gb300 import gen as G
    h, steps = ADJOINT_CASES[case]
    w = G.workload_sbm_small()
    fp = fingerprint(w)
    idx = sample_nodes(w.graph.n)
    t0 = time.time()
    L, g_om, g_K, g_th = oracle.adjoint_rk4_csr(w.graph.row_ptr, w.graph.col, w.omega, w.K, w.theta0, h, steps, 0)
    secs = time.time() - t0
    rec = {
        "case": case, "workload": w.name, "K": w.K, "h": h, "n_steps": steps, "loss": "1 - r(T)",
        "source": "oracle.adjoint_rk4_csr (discrete adjoint of classical RK4, FP64, CSR definition)",
        "oracle_seconds": round(secs, 1), **fp,
        "L": L, "g_K": g_K, "g_theta0_norm": float(np.linalg.norm(g_th)), "g_omega_norm": float(np.linalg.norm(g_om)),
        "idx": [int(i) for i in idx], "g_theta0": [float(v) for v in g_th[idx]],
        "g_omega": [float(v) for v in g_om[idx]],
    }
    out = os.path.join(HERE, f"{case}_fp64.json")
    with open(out + ".tmp", "w") as f:
        json.dump(rec, f, indent=0)
    os.replace(out + ".tmp", out)
    print(f"{case}: {steps} steps in {secs:.0f} s, L = {L:.9f}", flush=True)


def make(case: str) -> None:
    if case in ADJOINT_CASES:
        return make_adjoint(case)
    import oracle
    w, h, steps = workload(case)
    fp = fingerprint(w)
    idx = sample_nodes(w.graph.n)
    t0 = time.time()
    th = oracle.rk4_csr(w.graph.row_ptr, w.graph.col, w.omega, w.K, w.theta0, h, steps)
    secs = time.time() - t0
    r, psi = oracle.order_params(th)
    rec = {
        "case": case, "workload": w.name, "K": w.K, "h": h, "n_steps": steps, "precision": "fp64",
        "source": "oracle.rk4_csr (classical RK4 on eq:KuramotoGraph, CSR definition, uniform K/N)",
        "oracle_seconds": round(secs, 1), **fp,
        "r_T": r, "psi_T": psi,
        "idx": [int(i) for i in idx], "theta_T": [float(v) for v in th[idx]],
    }
    with open(path(case) + ".tmp", "w") as f:
        json.dump(rec, f, indent=0)
    os.replace(path(case) + ".tmp", path(case))
    print(f"{case}: {steps} steps in {secs:.0f} s, r(T) = {r:.6f}", flush=True)


if __name__ == "__main__":
    for c in sys.argv[1:]:
        make(c)
