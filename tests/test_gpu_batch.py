"""Batched ensembles (kura_batch_create + kura_rhs / kura_rk4_steps): every trajectory of one persistent launch
agrees with the FP64 oracle of the same trajectory, in both precisions and with the dense-block zeros on the
tensor cores (split BF16 mask product) or as index lists; the launch is deterministic.

Right-hand sides are checked with the bounds of tests/_parity.py (stated tolerance and scale-free error);
FP64 trajectories to 1e-8; mixed trajectories to the scale-free bound carried over the horizon."""
import numpy as np
import pytest

import oracle
from _parity import E_MIXED, check_rhs
from paper_2102_07167_gb300 import gen as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2102_07167_gb300 import kura


@pytest.fixture(scope="module")
def ensemble():
    return G.workload_batch(n_traj=24, seed=3, n_min=64, n_max=3000)


def _oracle_rhs(g, n, om, th, K, rows=None):
    if g is None:                                   # complete graph: the classical reformulation
        f = oracle.rhs_complete_op(om, th, K)
        return f if rows is None else f[rows]
    return oracle.rhs_csr(g.row_ptr, g.col, om, th, K, rows=rows)


def _deg(g, n, rows=None):
    d = np.full(n, n - 1) if g is None else np.diff(g.row_ptr)
    return d if rows is None else d[rows]


def _large_ensemble(seed=5):
    """n in {8192, 16384}: complete graphs and SBMs (8 and 16 communities, p_in 0.9, p_out 0.005)."""
    out = []
    for t, (n, c) in enumerate([(16384, 0), (16384, 16), (8192, 8), (8192, 0), (12000, 12)]):
        om = G.normal(seed + t, 21, n)
        th = G.uniform(seed + t, 22, n, 0.0, 2 * np.pi)
        K = float(G.uniform(seed, 12, 8, 0.5, 5.0)[t])
        if c == 0:
            out.append((None, n, om, th, K))
        else:
            g = G.sbm(seed + 100 + t, G.dirichlet_sizes(seed + 100 + t, n, c, 2, 16, 0), 0.9, 0.005)
            out.append((g, n, om, th, K))
    return out


@pytest.mark.parametrize("prec,tcm", [(1, 0), (1, 2), (0, 0)])
def test_batch_rhs_every_trajectory_vs_oracle(ensemble, prec, tcm):
    graphs = G.batch_graphs(ensemble)
    theta = np.concatenate([th + 30.0 * G.uniform(7, t, th.size, -1, 1) for t, (_, _, _, th, _) in enumerate(ensemble)])
    with kura.KuramotoBatch(graphs, precision=prec, tensor_cores=tcm) as b:
        info = b.info()
        assert info["precision"] == prec
        assert (info["tc_tiles"] > 0) == (tcm == 2)
        off = b.offsets
        f = np.empty_like(theta)
        b.rhs(theta, f)                                     # host pointers
        th_d = torch.tensor(theta, device="cuda:0")
        f_d = torch.empty_like(th_d)
        b.rhs(th_d, f_d)                                    # device pointers
        b.sync()
        assert np.array_equal(f, f_d.cpu().numpy())
    for t, (g, n, om, _, K) in enumerate(ensemble):
        th = theta[off[t]:off[t + 1]]
        ref = _oracle_rhs(g, n, om, th, K)
        check_rhs(f[off[t]:off[t + 1]], ref, _deg(g, n), K, n, prec, f"trajectory {t} (n {n}) prec {prec} tc {tcm}")


@pytest.mark.parametrize("prec,tcm", [(1, 0), (1, 2), (0, 0)])
def test_batch_rhs_large_trajectories_vs_oracle(prec, tcm):
    """Trajectories at the largest sizes (16384 nodes mixed; FP64 up to 8192), sampled rows vs the oracle."""
    ens = [e for e in _large_ensemble() if prec == 1 or e[1] <= 8192]
    graphs = G.batch_graphs(ens)
    theta = np.concatenate([th for (_, _, _, th, _) in ens])
    with kura.KuramotoBatch(graphs, precision=prec, tensor_cores=tcm) as b:
        if tcm == 2:
            assert b.info()["tc_traj"] == sum(1 for e in ens if e[0] is not None)
        off = b.offsets
        f = np.empty_like(theta)
        b.rhs(theta, f)
    for t, (g, n, om, th, K) in enumerate(ens):
        rows = np.unique(G.permutation(40 + t, n)[:800].astype(np.int64))
        ref = _oracle_rhs(g, n, om, th, K, rows)
        check_rhs(f[off[t]:off[t + 1]][rows], ref, _deg(g, n, rows), K, n, prec,
                  f"large trajectory {t} (n {n}) prec {prec} tc {tcm}")


@pytest.mark.parametrize("prec,tcm", [(1, 0), (1, 2), (0, 0)])
def test_batch_trajectories_vs_oracle(ensemble, prec, tcm):
    h, steps = 0.01, 25
    graphs = G.batch_graphs(ensemble)
    theta0 = np.concatenate([th for (_, _, _, th, _) in ensemble])
    with kura.KuramotoBatch(graphs, precision=prec, tensor_cores=tcm) as b:
        off = b.offsets
        th = torch.tensor(theta0, device="cuda:0")
        b.rk4_steps(th, h, steps)
        b.sync()
        got = th.cpu().numpy()
        th2 = torch.tensor(theta0, device="cuda:0")
        b.rk4_steps(th2, h, steps)
        b.sync()
        assert torch.equal(th, th2)                                  # deterministic
    for t, (g, n, om, th0, K) in enumerate(ensemble):
        ref = oracle.rk4_complete(om, K, th0, h, steps) if g is None else oracle.rk4_csr(g.row_ptr, g.col, om, K,
                                                                                            th0, h, steps)
        seg = got[off[t]:off[t + 1]]
        bound = 1e-8 if prec == 0 else 2.0 * E_MIXED * K / n * (1 + _deg(g, n).max()) * h * steps
        assert np.abs(seg - ref).max() <= bound, (t, np.abs(seg - ref).max(), bound)
        if prec == 1 and tcm == 0 and 0 < t < 6 and g is not None:
            with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, om, K, precision=kura.PREC_MIXED) as k:
                ts = torch.tensor(th0, device="cuda:0")
                k.rk4_steps(ts, h, steps)
                k.sync()
                assert np.abs(ts.cpu().numpy() - seg).max() < 1e-6


def test_batch_large_trajectory_rk4_vs_oracle():
    """A 16384-node SBM trajectory (16 communities) over 10 RK4 steps, tensor cores on, against the oracle."""
    g, n, om, th0, K = _large_ensemble()[1]
    h, steps = 0.01, 10
    with kura.KuramotoBatch([(g.row_ptr, g.col, g.label, g.n_comm, om, K)], tensor_cores=2) as b:
        assert b.info()["tc_tiles"] > 0
        th = torch.tensor(th0, device="cuda:0")
        b.rk4_steps(th, h, steps)
        b.sync()
        got = th.cpu().numpy()
    ref = oracle.rk4_csr(g.row_ptr, g.col, om, K, th0, h, steps)
    bound = 2.0 * E_MIXED * K / n * (1 + np.diff(g.row_ptr).max()) * h * steps
    assert np.abs(got - ref).max() <= bound


def test_persistent_single_cta_complete_512_fp64_full_horizon():
    """The classical all-to-all model (N = 512, K = 2, h = 0.01, 200 steps) as a batch of one: a single
    persistent CTA runs every step of the trajectory; FP64 against the oracle to 1e-8."""
    w = G.workload_complete(512)
    with kura.KuramotoBatch([(None, None, None, 1, w.omega, w.K)], precision=kura.PREC_FP64) as b:
        th = torch.tensor(w.theta0, device="cuda:0")
        b.rk4_steps(th, w.h, w.n_steps)
        b.sync()
        got = th.cpu().numpy()
    ref = oracle.rk4_complete(w.omega, w.K, w.theta0, w.h, w.n_steps)
    assert np.abs(got - ref).max() <= 1e-8


def test_batch_host_pointers_and_limits(ensemble):
    graphs = G.batch_graphs(ensemble[:4])
    theta0 = np.concatenate([th for (_, _, _, th, _) in ensemble[:4]])
    with kura.KuramotoBatch(graphs) as b:
        host = theta0.copy()
        b.rk4_steps(host, 0.01, 3)
        dev = torch.tensor(theta0, device="cuda:0")
        b.rk4_steps(dev, 0.01, 3)
        b.sync()
        assert np.array_equal(host, dev.cpu().numpy())
        st = b.stats()
        assert st["n_total"] == theta0.size
    with pytest.raises(kura.KuraError) as e:
        kura.KuramotoBatch([(None, None, None, 1, np.zeros(16385), 1.0)])
    assert e.value.status == kura.KURA_EINVAL
    with pytest.raises(kura.KuraError) as e:
        kura.KuramotoBatch([(None, None, None, 1, np.zeros(8193), 1.0)], precision=kura.PREC_FP64)
    assert e.value.status == kura.KURA_EINVAL


@pytest.mark.parametrize("tcm", [0, 2])
def test_batch_integration_bitwise_repeatable(tcm):
    """Three integrations of 256 batch trajectories (50 RK4 steps each, fresh handles) give bitwise equal
    states: block sums are exact fixed-point sums and every other sum has a fixed order."""
    ens = G.workload_batch(n_traj=256)
    theta0 = np.concatenate([t0 for (_, _, _, t0, _) in ens])
    res = []
    for _ in range(3):
        with kura.KuramotoBatch(G.batch_graphs(ens), tensor_cores=tcm) as b:
            th = torch.tensor(theta0, device="cuda:0")
            b.rk4_steps(th, 0.01, 50)
            torch.cuda.synchronize()
            res.append(th.cpu().numpy())
    assert all(np.array_equal(r, res[0]) for r in res)


@pytest.mark.parametrize("prec,lanes", [(1, 16), (1, 8), (0, 8)])
def test_batch_row_tiles_vs_oracle(ensemble, prec, lanes):
    """Row tiles of 16 and 8 lanes per row (2 and 4 rows per warp) give the same right-hand sides."""
    graphs = G.batch_graphs(ensemble)
    theta = np.concatenate([th for (_, _, _, th, _) in ensemble])
    with kura.KuramotoBatch(graphs, precision=prec, row_lanes=lanes) as b:
        assert b.traj_params(1)[2] == lanes
        off = b.offsets
        f = np.empty_like(theta)
        b.rhs(theta, f)
    for t, (g, n, om, th, K) in enumerate(ensemble):
        check_rhs(f[off[t]:off[t + 1]], _oracle_rhs(g, n, om, th, K), _deg(g, n), K, n, prec,
                  f"trajectory {t} lanes {lanes}")


@pytest.mark.parametrize("prec", [1, 0])
def test_batch_autotune_keeps_the_right_hand_side(ensemble, prec):
    """The batch autotuner times the dense-zero encodings (mixed precision), row tiles and tau per size class
    and rebuilds the batch; every choice computes the same right-hand sides up to rounding."""
    graphs = G.batch_graphs(ensemble)
    theta = np.concatenate([th for (_, _, _, th, _) in ensemble])
    with kura.KuramotoBatch(graphs, precision=prec) as b:
        res = b.autotune(theta, budget_s=60.0)
        assert res["candidates"] >= 4 and res["rhs_ms"] > 0 and res["initial_rhs_ms"] > 0
        params = [b.traj_params(t) for t in range(len(ensemble))]
        off = b.offsets
        f = np.empty_like(theta)
        b.rhs(theta, f)
    for t, (tau, tc, lanes) in enumerate(params):
        assert tau in (0.35, 0.5, 0.65) and tc in ((0, 2) if prec == 1 else (0,)) and lanes in (32, 16, 8)
    for t, (g, n, om, th, K) in enumerate(ensemble):
        check_rhs(f[off[t]:off[t + 1]], _oracle_rhs(g, n, om, th, K), _deg(g, n), K, n, prec,
                  f"tuned trajectory {t}")
