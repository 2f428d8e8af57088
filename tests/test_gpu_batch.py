"""Batched ensembles (kura_batch_create + kura_rk4_steps): every trajectory of one persistent launch agrees
with the FP64 oracle's RK4 of the same trajectory (mixed-precision tolerance) and with the single-graph
mixed path; the launch is deterministic."""
import numpy as np
import pytest

import oracle
from paper_2102_07167_gb300 import gen as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2102_07167_gb300 import kura


@pytest.fixture(scope="module")
def ensemble():
    return G.workload_batch(n_traj=24, seed=3, n_min=64, n_max=3000)


def test_batch_matches_oracle_and_single_graph(ensemble):
    h, steps = 0.01, 25
    graphs = G.batch_graphs(ensemble)
    theta0 = np.concatenate([th for (_, _, _, th, _) in ensemble])
    with kura.KuramotoBatch(graphs) as b:
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
        assert np.abs(seg - ref).max() < 2e-5, (t, np.abs(seg - ref).max())
        if 0 < t < 6 and g is not None:
            with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, om, K, precision=kura.PREC_MIXED) as k:
                ts = torch.tensor(th0, device="cuda:0")
                k.rk4_steps(ts, h, steps)
                k.sync()
                assert np.abs(ts.cpu().numpy() - seg).max() < 1e-6


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


def test_batch_integration_bitwise_repeatable():
    """Three integrations of 256 batch trajectories (50 RK4 steps each, fresh handles) give bitwise equal
    states: block sums are exact fixed-point sums and every other sum has a fixed order."""
    ens = G.workload_batch(n_traj=256)
    theta0 = np.concatenate([t0 for (_, _, _, t0, _) in ens])
    res = []
    for _ in range(3):
        with kura.KuramotoBatch(G.batch_graphs(ens)) as b:
            th = torch.tensor(theta0, device="cuda:0")
            b.rk4_steps(th, 0.01, 50)
            torch.cuda.synchronize()
            res.append(th.cpu().numpy())
    assert all(np.array_equal(r, res[0]) for r in res)
