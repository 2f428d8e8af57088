"""GPU RK4 trajectories of the SBM workloads against the FP64 oracle's, stored in tests/golden/.

The oracle needs minutes to hours for these horizons (tests/golden/make_trajectory_goldens.py wrote the
files with oracle.rk4_csr: classical RK4 on eq:KuramotoGraph by the CSR definition), so each golden holds
theta(T) at 2048 fixed random nodes and a fingerprint of the inputs.  The test rebuilds the inputs with
the same seeded generator, checks the fingerprint, integrates on the GPU through the C ABI and compares:

  FP64 handle:   |theta_i(T) - oracle_i(T)| <= 1e-8 (the stated trajectory tolerance)
  mixed handle:  <= 2 E_MIXED max_i (K/N)(1 + deg_i) T, the scale-free right-hand-side bound carried
                 over the horizon (the error of theta grows at most by the RHS error per unit time)

Cases: the 65536-node SBM over its full 1000 steps of h = 0.005; the 2^20-node recipe at N = 2^16
(64 communities) over its full 500 steps of h = 0.01; the 2^20-node SBM itself over 10 steps.
"""
import json
import os
import sys

import numpy as np
import pytest

from _parity import E_MIXED

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_trajectory_goldens as MG  # noqa: E402  (inputs and fingerprint only; never calls the oracle here)

if torch.cuda.is_available():
    from paper_2102_07167_gb300 import kura

CASES = ["sbm65536_1000", "sbm2p16_500", "sbm2p20_10"]


def _load(case):
    p = MG.path(case)
    if not os.path.exists(p):
        pytest.fail(f"golden file {os.path.basename(p)} is missing: run tests/golden/make_trajectory_goldens.py {case}")
    with open(p) as f:
        return json.load(f)


def _check_inputs(rec, w):
    fp = MG.fingerprint(w)
    for key in ("n", "nnz", "n_comm", "graph_sha256"):
        assert fp[key] == rec[key], f"input mismatch in {key}: the generator no longer draws the golden's graph"
    for key in ("omega_sum", "omega_abs_sum", "theta0_sum"):
        assert abs(fp[key] - rec[key]) <= 1e-12 * max(1.0, abs(rec[key])), key


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", CASES)
def test_rk4_trajectory_vs_oracle_golden(case, prec):
    rec = _load(case)
    w, h, steps = MG.workload(case)
    assert (h, steps) == (rec["h"], rec["n_steps"])
    _check_inputs(rec, w)
    g = w.graph
    idx = np.asarray(rec["idx"], dtype=np.int64)
    expect = np.asarray(rec["theta_T"])
    assert np.array_equal(idx, MG.sample_nodes(g.n))
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=prec) as k:
        th = torch.tensor(w.theta0, device="cuda:0")
        k.rk4_steps(th, h, steps)
        r, psi = k.order_params(th)
        got = th.cpu().numpy()
    err = np.abs(got[idx] - expect)
    if prec == 0:
        bound = 1e-8
    else:
        deg = np.diff(g.row_ptr)
        bound = 2.0 * E_MIXED * (w.K / g.n) * (1.0 + deg.max()) * h * steps
    assert err.max() <= bound, f"{case} prec {prec}: max |dtheta| {err.max():.3e} > {bound:.3e}"
    assert abs(r - rec["r_T"]) <= max(bound, 1e-12), (r, rec["r_T"])
