"""GPU parity of the tensor-core encoding of dense-block zeros (TILE_TC tiles: 0/1 mask x base-16 digits of
the fixed-point table on tcgen05).  Both encodings compute the same exact fixed-point sums, so in FP64 mode
the tensor-core path must agree with the index-list path bit for bit; both are also checked against the
FP64 oracle (eq:KuramotoGraph) at the parity tolerances of the other GPU tests."""
import numpy as np
import pytest

import oracle
from _parity import check_rhs
from paper_2102_07167_gb300 import gen as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2102_07167_gb300 import kura


def _ragged_graph(seed=5):
    """Symmetric block graph with ragged community sizes (1, 127, 129, 300, 513, 700, 1030: partial 128-row
    M-blocks, communities over several tiles, windows not aligned to 128 columns) and two dense off-diagonal
    block pairs (windows spanning several communities)."""
    rng = np.random.default_rng(seed)
    sizes = np.array([1, 127, 129, 300, 513, 700, 1030])
    p_in = [1.0, 0.9, 0.8, 0.6, 0.95, 0.7, 0.85]
    off = np.concatenate([[0], np.cumsum(sizes)])
    n = int(off[-1])
    P = np.full((len(sizes), len(sizes)), 0.01)
    np.fill_diagonal(P, p_in)
    P[3, 4] = P[4, 3] = 0.7
    P[5, 6] = P[6, 5] = 0.55
    lab = np.repeat(np.arange(len(sizes)), sizes)
    prob = P[lab][:, lab]
    A = (rng.random((n, n)) < prob).astype(np.uint8)
    A = np.triu(A, 1)
    A = A | A.T
    perm = rng.permutation(n)                     # labels not contiguous in user order
    A = A[perm][:, perm]
    return G.from_dense(A, lab[perm].astype(np.int32), len(sizes))


@pytest.fixture(scope="module")
def ragged():
    return _ragged_graph()


@pytest.fixture(scope="module")
def sbm_small():
    return G.workload_sbm_small(n=12000, n_comm=12, min_size=128, seed=3)


def _dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda:0")


def _rhs(k, theta):
    th = _dev(theta)
    out = torch.empty_like(th)
    k.rhs(th, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _traj(k, theta, h, steps):
    th = _dev(theta)
    k.rk4_steps(th, h, steps)
    torch.cuda.synchronize()
    return th.cpu().numpy()


@pytest.mark.parametrize("which", ["ragged", "sbm_small"])
def test_fp64_tensor_cores_bit_identical_to_index_lists(which, ragged, sbm_small):
    if which == "ragged":
        g = ragged
        rng = np.random.default_rng(1)
        omega, theta, K = rng.normal(size=g.n), rng.uniform(-40, 40, g.n), 2.5
    else:
        w = sbm_small
        g, omega, theta, K = w.graph, w.omega, w.theta0, w.K
    ks = {tcm: kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, omega, K, precision=kura.PREC_FP64,
                             tensor_cores=tcm) for tcm in (0, 2)}
    try:
        assert ks[0].stats()["tc_tiles"] == 0 and ks[2].stats()["tc_tiles"] > 0
        f0, f2 = _rhs(ks[0], theta), _rhs(ks[2], theta)
        assert np.array_equal(f0, f2)
        ref = oracle.rhs_csr(g.row_ptr, g.col, omega, theta, K)
        check_rhs(f2, ref, np.diff(g.row_ptr), K, g.n, 0, f"{which} tensor cores")
        t0, t2 = _traj(ks[0], theta, 0.01, 12), _traj(ks[2], theta, 0.01, 12)
        assert np.array_equal(t0, t2)
    finally:
        for k in ks.values():
            k.close()


@pytest.mark.parametrize("tcm", [1, 2])
def test_mixed_tensor_cores_vs_oracle(ragged, tcm):
    g = ragged
    rng = np.random.default_rng(2)
    omega, theta, K = rng.normal(size=g.n), rng.uniform(-40, 40, g.n), 2.5
    ref = oracle.rhs_csr(g.row_ptr, g.col, omega, theta, K)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, omega, K, precision=kura.PREC_MIXED,
                       tensor_cores=tcm) as k:
        f = _rhs(k, theta)
        st = k.stats()
    check_rhs(f, ref, np.diff(g.row_ptr), K, g.n, 1, f"ragged mixed tensor_cores={tcm}")
    if tcm == 2:
        assert st["tc_tiles"] > 0
    # the tensor-core sums are exact in fixed point: closer to the oracle than FP32 per-entry sums
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, omega, K, precision=kura.PREC_MIXED,
                       tensor_cores=0) as k0:
        f0 = _rhs(k0, theta)
    assert np.max(np.abs(f - ref)) <= np.max(np.abs(f0 - ref)) * 1.5 + 1e-12


def test_full_size_2p20_tensor_core_tiles_sampled_rows():
    """The 2^20-node SBM at its default encoding runs most communities on the tensor cores; sampled rows
    against the oracle (FP64: exact fixed-point sums)."""
    w = G.workload_sbm_large()
    g = w.graph
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=kura.PREC_FP64) as k:
        st = k.stats()
        assert st["tc_tiles"] > 0.5 * st["tiles"]
        f = _rhs(k, w.theta0)
    rows = np.random.default_rng(3).choice(g.n, 4000, replace=False)
    ref = oracle.rhs_csr(g.row_ptr, g.col, w.omega, w.theta0, w.K, rows=rows)
    deg = np.diff(g.row_ptr)[rows]
    check_rhs(f[rows], ref, deg, w.K, g.n, 0, "sbm-2^20 FP64 tensor-core tiles")


@pytest.mark.parametrize("loss_kind", [0, 1])
def test_adjoint_tensor_cores_vs_index_lists(ragged, loss_kind):
    """The adjoint's digits use their own scale (max |nu sin|, |nu cos|): gradients agree with the index-list
    path to FP32 rounding and with the oracle adjoint."""
    g = ragged
    rng = np.random.default_rng(4)
    omega, theta0, K = rng.normal(size=g.n), rng.uniform(0, 2 * np.pi, g.n), 1.5
    target = theta0 + 0.1 * rng.normal(size=g.n) if loss_kind == 1 else None
    h, steps, M = 0.01, 12, 5
    out = {}
    for tcm in (0, 2):
        with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, omega, K, precision=kura.PREC_MIXED,
                           tensor_cores=tcm) as k:
            tg = _dev(target) if target is not None else None
            L, gom, gK, gth = k.adjoint(_dev(theta0), h, steps, M, loss_kind, tg)
            torch.cuda.synchronize()
            out[tcm] = (L, gom.cpu().numpy(), gK, gth.cpu().numpy())
    L_ref, gom_ref, gK_ref, gth_ref = oracle.adjoint_rk4_csr(g.row_ptr, g.col, omega, K, theta0, h, steps,
                                                             loss_kind, target)

    def rel(a, b):
        return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))
    for tcm in (0, 2):
        L, gom, gK, gth = out[tcm]
        assert abs(L - L_ref) <= 1e-6 * max(1.0, abs(L_ref))
        assert rel(gom, gom_ref) < 2e-4 and rel(gth, gth_ref) < 2e-4, (tcm, rel(gom, gom_ref), rel(gth, gth_ref))
        assert abs(gK - gK_ref) <= 2e-4 * max(abs(gK_ref), 1e-12), (tcm, gK, gK_ref)
    assert rel(out[2][1], out[0][1]) < 2e-4 and rel(out[2][3], out[0][3]) < 2e-4


def test_autotune_keeps_the_right_hand_side(sbm_small):
    """The autotuner times candidate plans (encoding, tile work, tau) and keeps the fastest; the right-hand
    side stays within the FP64 parity tolerance of the oracle (every plan computes the same sums)."""
    w = sbm_small
    g = w.graph
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=kura.PREC_FP64) as k:
        res = k.autotune(_dev(w.theta0), budget_s=60.0)
        assert res["candidates"] >= 4 and res["rhs_ms"] <= res["initial_rhs_ms"] + 1e-9
        assert res["tau"] in (0.35, 0.5, 0.65) and res["tensor_cores"] in (0, 1)
        f = _rhs(k, w.theta0)
        st = k.stats()
        assert abs(st["tau"] - res["tau"]) < 1e-12
    ref = oracle.rhs_csr(g.row_ptr, g.col, w.omega, w.theta0, w.K)
    check_rhs(f, ref, np.diff(g.row_ptr), w.K, g.n, 0, "autotuned plan")


def test_gather_rate_probe():
    """The roofline probe measures a plausible random-gather rate (between 10^10 and 10^13 per second)."""
    r8 = kura.kura_measure_gather_rate(1 << 20, 1 << 24, 8)
    r16 = kura.kura_measure_gather_rate(1 << 20, 1 << 24, 16)
    assert 1e10 < r8 < 1e13 and 1e10 < r16 < 1e13


@pytest.mark.parametrize("prec", [0, 1])
def test_repeated_rhs_bitwise_identical_sbm_2p19(prec):
    """Every right-hand side is a fixed function of theta: 150 repeated evaluations on the 2^19-node SBM
    (rows with ~105 sparse entries next to tensor-core masks, the regime in which the row kernel's ring
    slots turn over fastest) are bitwise identical.  A slot handed back to TMA before the warp's reads of
    it had completed showed up here as one row of a few percent of FP64 evaluations differing."""
    w = G.workload_sbm_large(n=1 << 19, n_comm=512, p_out=2e-4)
    g = w.graph
    th = torch.tensor(w.theta0, device="cuda:0")
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=prec) as k:
        assert k.stats()["tc_tiles"] > 0
        out = torch.empty_like(th)
        k.rhs(th, out)
        k.sync()
        first = out.clone()
        bad = 0
        for _ in range(150):
            k.rhs(th, out)
            k.sync()
            bad += int((out != first).sum())
    assert bad == 0


def test_handles_with_different_plans_coexist(sbm_small):
    """The row kernel's shared-memory limit is shared by every handle: after one handle is re-planned to a
    smaller layout (the autotuner moving it to index lists), a second handle whose plan needs more shared
    memory (tensor-core stages) still runs, and so does its own autotuning."""
    w = sbm_small
    g = w.graph
    th = _dev(w.theta0)
    ref = oracle.rhs_csr(g.row_ptr, g.col, w.omega, w.theta0, w.K)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=kura.PREC_MIXED,
                       tensor_cores=2) as k1, \
            kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=kura.PREC_MIXED,
                          tensor_cores=2) as k2:
        k1.classify_blocks(0.5)
        k1.autotune(th, budget_s=10.0)
        f2 = _rhs(k2, w.theta0)
        k2.autotune(th, budget_s=10.0)
        f1 = _rhs(k1, w.theta0)
    deg = np.diff(g.row_ptr)
    check_rhs(f1, ref, deg, w.K, g.n, 1, "first handle")
    check_rhs(f2, ref, deg, w.K, g.n, 1, "second handle")


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("tcm", [0, 2])
@pytest.mark.parametrize("which", ["ragged", "sbm_small"])
def test_fused_trig_bit_identical_to_a_trig_launch_per_stage(which, tcm, prec, ragged, sbm_small):
    """kura_rk4_steps with the fused trig (each stage's row kernel makes the next stage's table, digits and
    block sums; one trig launch per run) gives the same bits as a trig/block-sum launch before every stage:
    index lists and tensor-core digits, partial 128-node digit blocks (ragged sizes), 11 steps (an 8-step
    graph and a 3-step one), and the FP64 result stays within 1e-8 of the oracle's trajectory."""
    if which == "ragged":
        g = ragged
        rng = np.random.default_rng(4)
        omega, theta, K = rng.normal(size=g.n), rng.uniform(0, 2 * np.pi, g.n), 2.5
    else:
        w = sbm_small
        g, omega, theta, K = w.graph, w.omega, w.theta0, w.K
    out = {}
    for fused in (1, 0):
        with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, omega, K, precision=prec, tensor_cores=tcm,
                           persistent_small=0, fused_trig=fused) as k:
            assert (k.stats()["tc_tiles"] > 0) == (tcm == 2)
            out[fused] = _traj(k, theta, 0.01, 11)
            # a later call starts from the state the last one left
            out[fused] = np.concatenate([out[fused], _traj(k, out[fused], 0.01, 2)])
    assert np.array_equal(out[1], out[0])
    if prec == 0:
        ref = oracle.rk4_csr(g.row_ptr, g.col, omega, K, theta, 0.01, 11)
        assert np.max(np.abs(out[1][:g.n] - ref)) < 1e-8
