"""GPU discrete RK4 adjoint (kura_adjoint, FP32 right-hand side, FP64 state) against the FP64 oracle adjoint
and against central finite differences of the forward map."""
import numpy as np
import pytest

import oracle
from _parity import check_rhs
from paper_2102_07167_gb300 import gen as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2102_07167_gb300 import kura


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.fixture(scope="module")
def small():
    w = G.workload_sbm_small(n=3000, n_comm=5, min_size=200, seed=7)
    return w


@pytest.mark.parametrize("loss_kind", [0, 1])
def test_adjoint_matches_oracle_adjoint(small, loss_kind):
    w = small
    g = w.graph
    h, steps, M = 0.01, 30, 8          # 4 segments: 8 + 8 + 8 + 6
    rng = np.random.default_rng(loss_kind)
    target = w.theta0 + 0.2 * rng.normal(size=g.n) if loss_kind == 1 else None
    L_ref, gom_ref, gK_ref, gth_ref = oracle.adjoint_rk4_csr(g.row_ptr, g.col, w.omega, w.K, w.theta0, h, steps,
                                                             loss_kind, target)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=kura.PREC_MIXED) as k:
        th0 = torch.tensor(w.theta0, device="cuda:0")
        tg = torch.tensor(target, device="cuda:0") if target is not None else None
        L, gom, gK, gth = k.adjoint(th0, h, steps, M, loss_kind, tg)
        torch.cuda.synchronize()
        gom, gth = gom.cpu().numpy(), gth.cpu().numpy()
        assert np.array_equal(th0.cpu().numpy(), w.theta0)          # theta0 is not modified
        # a second call gives the bitwise same result (deterministic reductions)
        L2, gom2, gK2, gth2 = k.adjoint(th0, h, steps, M, loss_kind, tg)
        assert L2 == L and gK2 == gK and np.array_equal(gom2.cpu().numpy(), gom)
    assert abs(L - L_ref) <= 1e-6 * max(1.0, abs(L_ref))
    assert _rel(gth, gth_ref) < 2e-4, _rel(gth, gth_ref)
    assert _rel(gom, gom_ref) < 2e-4, _rel(gom, gom_ref)
    assert abs(gK - gK_ref) <= 2e-4 * max(abs(gK_ref), 1e-12), (gK, gK_ref)


def test_adjoint_matches_finite_differences_of_forward(small):
    """Directional derivatives by central differences (eps = 1e-6) of the FP64 forward loss 1 - r(T)."""
    w = small
    g = w.graph
    h, steps = 0.01, 40
    rng = np.random.default_rng(5)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=kura.PREC_MIXED) as ka, \
            kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K) as kf:
        L, gom, gK, gth = ka.adjoint(torch.tensor(w.theta0, device="cuda:0"), h, steps, 16, 0)
        gth, gom = gth.cpu().numpy(), gom.cpu().numpy()

        def loss(theta0, omega, K):
            kf.set_param(omega=np.ascontiguousarray(omega), K=K)
            th = torch.tensor(theta0, device="cuda:0")
            kf.rk4_steps(th, h, steps)
            return 1.0 - kf.order_params(th)[0]

        eps = 1e-6
        for _ in range(3):
            d = rng.normal(size=g.n)
            fd = (loss(w.theta0 + eps * d, w.omega, w.K) - loss(w.theta0 - eps * d, w.omega, w.K)) / (2 * eps)
            assert abs(fd - gth @ d) <= 1e-3 * abs(fd) + 1e-7, (fd, gth @ d)
            fd = (loss(w.theta0, w.omega + eps * d, w.K) - loss(w.theta0, w.omega - eps * d, w.K)) / (2 * eps)
            assert abs(fd - gom @ d) <= 1e-3 * abs(fd) + 1e-7, (fd, gom @ d)
        fd = (loss(w.theta0, w.omega, w.K + eps) - loss(w.theta0, w.omega, w.K - eps)) / (2 * eps)
        assert abs(fd - gK) <= 1e-3 * abs(fd) + 1e-7, (fd, gK)


def test_adjoint_uncoupled_closed_form(small):
    w = small
    g = w.graph
    h, steps = 0.05, 12
    T = h * steps
    target = np.zeros(g.n)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, 0.0, precision=kura.PREC_MIXED) as k:
        L, gom, gK, gth = k.adjoint(np.ascontiguousarray(w.theta0), h, steps, 5, 1, target)
    resid = w.theta0 + T * w.omega
    np.testing.assert_allclose(gth, resid, atol=1e-12, rtol=0)
    np.testing.assert_allclose(gom, T * resid, atol=1e-11, rtol=0)


def test_adjoint_rejects_unsupported_handles(small):
    w = small
    g = w.graph
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K) as k:      # FP64 handle
        with pytest.raises(kura.KuraError) as e:
            k.adjoint(np.ascontiguousarray(w.theta0), 0.01, 2)
        assert e.value.status == kura.KURA_ESTATE


@pytest.mark.parametrize("loss_kind", [0, 1])
def test_adjoint_directed_graph_vs_oracle(loss_kind):
    """A directed A (each SBM edge kept in one direction only with probability 0.3, plus one-way dense
    off-diagonal blocks): the nu-weighted sums of J^T w run over the plan of A^T; against the FP64 oracle
    adjoint, which forms J^T from the CSR directly."""
    rng = np.random.default_rng(21)
    sizes = [300, 513, 129, 700]
    lab = np.repeat(np.arange(4), sizes)
    n = int(sum(sizes))
    P = np.full((4, 4), 0.01)
    np.fill_diagonal(P, [0.9, 0.7, 0.95, 0.8])
    P[0, 3] = 0.75                                              # a dense block whose transpose is sparse
    A = (rng.random((n, n)) < P[lab][:, lab]).astype(np.uint8)
    np.fill_diagonal(A, 0)
    drop = rng.random((n, n)) < 0.3
    A[drop] = 0                                                 # breaks the symmetry
    perm = rng.permutation(n)
    gd = G.from_dense(A[perm][:, perm], lab[perm].astype(np.int32), 4)
    omega, theta0, K = rng.normal(size=n), rng.uniform(0, 2 * np.pi, n), 3.0
    h, steps, M = 0.01, 20, 6
    target = theta0 + 0.1 * rng.normal(size=n) if loss_kind == 1 else None
    L_ref, gom_ref, gK_ref, gth_ref = oracle.adjoint_rk4_csr(gd.row_ptr, gd.col, omega, K, theta0, h, steps,
                                                             loss_kind, target)
    with kura.Kuramoto(gd.row_ptr, gd.col, gd.label, 4, omega, K, precision=kura.PREC_MIXED) as k:
        tg = torch.tensor(target, device="cuda:0") if target is not None else None
        L, gom, gK, gth = k.adjoint(torch.tensor(theta0, device="cuda:0"), h, steps, M, loss_kind, tg)
        gom, gth = gom.cpu().numpy(), gth.cpu().numpy()
    assert abs(L - L_ref) <= 1e-6 * max(1.0, abs(L_ref))
    assert _rel(gth, gth_ref) < 2e-4, _rel(gth, gth_ref)
    assert _rel(gom, gom_ref) < 2e-4, _rel(gom, gom_ref)
    assert abs(gK - gK_ref) <= 2e-4 * max(abs(gK_ref), 1e-12), (gK, gK_ref)


def test_autograd_function(small):
    from paper_2102_07167_gb300.autograd import KuraRK4Loss
    w = small
    g = w.graph
    dev = torch.device("cuda", 0)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=kura.PREC_MIXED) as k:
        th0 = torch.tensor(w.theta0, device=dev, requires_grad=True)
        om = torch.tensor(w.omega, device=dev, requires_grad=True)
        K = torch.tensor(w.K, dtype=torch.float64, device=dev, requires_grad=True)
        loss = KuraRK4Loss.apply(th0, om, K, k, 0.01, 20, 8, 0, None)
        (2.0 * loss).backward()
        L, gom, gK, gth = k.adjoint(torch.tensor(w.theta0, device=dev), 0.01, 20, 8, 0)
        assert abs(loss.item() - L) < 1e-15
        assert torch.allclose(th0.grad, 2.0 * gth, rtol=0, atol=0)
        assert torch.allclose(om.grad, 2.0 * gom, rtol=0, atol=0)
        assert abs(K.grad.item() - 2.0 * gK) < 1e-15
        # one gradient step on K lowers 1 - r (strengthening the coupling synchronises)
        with torch.no_grad():
            K2 = K - 50.0 * K.grad
        loss2 = KuraRK4Loss.apply(th0.detach(), om.detach(), K2, k, 0.01, 20, 8, 0, None)
        assert loss2.item() < loss.item()
        # the handle has its own omega and K back: its right-hand side is the oracle's with w.omega, w.K
        assert k.K == w.K
        th = torch.tensor(w.theta0, device=dev)
        f = torch.empty_like(th)
        k.rhs(th, f)
        k.sync()
        ref = oracle.rhs_csr(g.row_ptr, g.col, w.omega, w.theta0, w.K)
        check_rhs(f.cpu().numpy(), ref, np.diff(g.row_ptr), w.K, g.n, 1, "handle after KuraRK4Loss")


def test_adjoint_config5_graph_vs_oracle_adjoint_golden():
    """The 65536-node SBM of the adjoint workload (64 communities, p_in 0.95, p_out 0.001, K = 4), loss 1 - r(T),
    h = 0.01 over 4 steps with a checkpoint every 2: the mixed-precision adjoint against the FP64 oracle adjoint
    stored in tests/golden/ (the oracle needs about two minutes for it)."""
    import json
    import os
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    sys.path.insert(0, os.path.join(here, "golden"))
    import make_trajectory_goldens as MG
    path = os.path.join(here, "golden", "adjoint_sbm65536_4_fp64.json")
    rec = json.load(open(path))
    w = G.workload_sbm_small()
    g = w.graph
    fp = MG.fingerprint(w)
    assert fp["graph_sha256"] == rec["graph_sha256"] and fp["nnz"] == rec["nnz"]
    assert abs(fp["omega_sum"] - rec["omega_sum"]) <= 1e-12 * max(1.0, abs(rec["omega_sum"]))
    idx = np.asarray(rec["idx"], dtype=np.int64)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=kura.PREC_MIXED) as k:
        L, gom, gK, gth = k.adjoint(torch.tensor(w.theta0, device="cuda:0"), rec["h"], rec["n_steps"], 2, 0)
        gom, gth = gom.cpu().numpy(), gth.cpu().numpy()
    assert abs(L - rec["L"]) <= 1e-6 * abs(rec["L"])
    assert abs(gK - rec["g_K"]) <= 2e-4 * abs(rec["g_K"]), (gK, rec["g_K"])
    assert _rel(gth[idx], rec["g_theta0"]) < 2e-4, _rel(gth[idx], rec["g_theta0"])
    assert _rel(gom[idx], rec["g_omega"]) < 2e-4, _rel(gom[idx], rec["g_omega"])
    assert abs(np.linalg.norm(gth) - rec["g_theta0_norm"]) <= 2e-4 * rec["g_theta0_norm"]
    assert abs(np.linalg.norm(gom) - rec["g_omega_norm"]) <= 2e-4 * rec["g_omega_norm"]


def test_adjoint_config5_finite_differences_32_directions():
    """The adjoint workload itself: 65536-node SBM, loss 1 - r(T), T = 20 (h = 0.01, 2000 steps), a checkpoint
    every 64 steps, FP32 right-hand side and FP64 state.  Directional derivatives along 32 random directions of
    (theta0, omega, K), by central differences (eps = 1e-6) of the FP64 forward loss, against the adjoint's."""
    w = G.workload_sbm_small()
    g = w.graph
    h, steps, M, eps = 0.01, 2000, 64, 1e-6
    rng = np.random.default_rng(2000)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=kura.PREC_MIXED) as ka, \
            kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K) as kf:
        L, gom, gK, gth = ka.adjoint(torch.tensor(w.theta0, device="cuda:0"), h, steps, M, 0)
        gth, gom = gth.cpu().numpy(), gom.cpu().numpy()

        def loss(theta0, omega, K):
            kf.set_param(omega=np.ascontiguousarray(omega), K=K)
            th = torch.tensor(theta0, device="cuda:0")
            kf.rk4_steps(th, h, steps)
            return 1.0 - kf.order_params(th)[0]

        assert abs(loss(w.theta0, w.omega, w.K) - L) <= 1e-6
        fd, ad = [], []
        for _ in range(32):
            dth, dom, dK = rng.normal(size=g.n), rng.normal(size=g.n), float(rng.normal())
            lp = loss(w.theta0 + eps * dth, w.omega + eps * dom, w.K + eps * dK)
            lm = loss(w.theta0 - eps * dth, w.omega - eps * dom, w.K - eps * dK)
            fd.append((lp - lm) / (2 * eps))
            ad.append(gth @ dth + gom @ dom + gK * dK)
    fd, ad = np.array(fd), np.array(ad)
    assert np.linalg.norm(ad - fd) <= 2e-3 * np.linalg.norm(fd), (np.linalg.norm(ad - fd), np.linalg.norm(fd))


def test_adjoint_after_a_replan_with_more_tiles(small):
    """The per-tile dK accumulators follow the plan: after kura_classify_blocks re-plans the handle into more
    tiles, the next adjoint sizes them anew and gives the result of a handle planned that way from the
    start."""
    w = small
    g = w.graph
    h, steps, M = 0.01, 12, 4
    th0 = torch.tensor(w.theta0, device="cuda:0")
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=kura.PREC_MIXED,
                       tensor_cores=0) as k:
        k.adjoint(th0, h, steps, M, 0)
        tiles0 = k.stats()["tiles"]
        k.classify_blocks(0.01)                 # the dense blocks become sparse: many more listed entries
        assert k.stats()["tiles"] > tiles0
        L, gom, gK, gth = k.adjoint(th0, h, steps, M, 0)
        got = (L, gom.cpu().numpy(), gK, gth.cpu().numpy())
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=kura.PREC_MIXED,
                       tensor_cores=0, tau=0.01) as k2:
        L2, gom2, gK2, gth2 = k2.adjoint(th0, h, steps, M, 0)
    assert abs(got[0] - L2) <= 1e-12 and abs(got[2] - gK2) <= 1e-10 * abs(gK2)
    assert _rel(got[1], gom2.cpu().numpy()) < 1e-10 and _rel(got[3], gth2.cpu().numpy()) < 1e-10


@pytest.mark.parametrize("tcm", [0, 2])
def test_two_stream_backward_matches_one_stream(small, tcm):
    """With the fused trig the backward recomputes segment c - 1 on a second stream while segment c's adjoint
    stages run, alternating two sets of stage buffers, and the forward keeps its last segment; without it,
    every segment is recomputed and then adjoined on one stream.  The kernels and their data are the same,
    so the gradients agree bit for bit: 4 full segments (captured graphs, both buffer sets), index lists and
    tensor-core tiles, two calls in a row."""
    w = small
    g = w.graph
    h, steps, M = 0.01, 32, 8
    res = {}
    for fused in (1, 0):
        with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=kura.PREC_MIXED,
                           tensor_cores=tcm, fused_trig=fused) as k:
            th0 = torch.tensor(w.theta0, device="cuda:0")
            out = []
            for _ in range(2):
                L, gom, gK, gth = k.adjoint(th0, h, steps, M, 0)
                out.append((L, gom.cpu().numpy(), gK, gth.cpu().numpy()))
            res[fused] = out
    for call in range(2):
        (L1, gom1, gK1, gth1), (L0, gom0, gK0, gth0) = res[1][call], res[0][call]
        assert L1 == L0 and gK1 == gK0
        assert np.array_equal(gom1, gom0) and np.array_equal(gth1, gth0)
