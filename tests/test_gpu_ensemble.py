"""GPU parity of ensembles sharing one graph (kura_ensemble_create): every trajectory's right-hand side and RK4
trajectory against the FP64 oracle of eq:KuramotoGraph with that trajectory's omega and K.  The dense-block
product runs as a BF16 0/1 mask times split BF16 hi + lo (sin, cos) GEMM with FP32 accumulation, so the
tolerances are the mixed-precision ones of the other GPU tests."""
import numpy as np
import pytest

import oracle
from _parity import check_rhs
from paper_2102_07167_gb300 import gen as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2102_07167_gb300 import kura


def _block_graph(sizes, p_in, p_out, seed, dense_pairs=()):
    rng = np.random.default_rng(seed)
    sizes = np.asarray(sizes)
    n = int(sizes.sum())
    P = np.full((len(sizes), len(sizes)), p_out)
    np.fill_diagonal(P, p_in)
    for (I, J, p) in dense_pairs:
        P[I, J] = P[J, I] = p
    lab = np.repeat(np.arange(len(sizes)), sizes)
    A = (rng.random((n, n)) < P[lab][:, lab]).astype(np.uint8)
    A = np.triu(A, 1)
    A = A | A.T
    perm = rng.permutation(n)
    return G.from_dense(A[perm][:, perm], lab[perm].astype(np.int32), len(sizes))


@pytest.fixture(scope="module")
def ragged():
    # ragged sizes (partial 128-row tiles, communities over several tiles), a sparse diagonal block
    # (p_in 0.3: listed present entries inside the community) and dense off-diagonal pairs
    return _block_graph([1, 127, 129, 300, 513, 700, 1030, 200], [1.0, 0.9, 0.8, 0.6, 0.95, 0.7, 0.85, 0.3],
                        0.01, 5, dense_pairs=((3, 4, 0.7), (5, 6, 0.55)))


def _inputs(g, n_traj, seed):
    rng = np.random.default_rng(seed)
    omega = rng.normal(size=(n_traj, g.n))
    K = rng.uniform(0.5, 5.0, n_traj)
    theta = rng.uniform(-40, 40, (n_traj, g.n))
    return omega, K, theta


@pytest.mark.parametrize("tcm", [1, 0])
def test_ensemble_rhs_every_trajectory_vs_oracle(ragged, tcm):
    g = ragged
    omega, K, theta = _inputs(g, 32, 1)
    with kura.KuramotoEnsemble(g.row_ptr, g.col, g.label, g.n_comm, omega, K, tensor_cores=tcm) as e:
        st = e.stats()
        assert (st["tc_tiles"] > 0) == (tcm != 0)
        th = torch.tensor(theta, device="cuda:0")
        out = torch.empty_like(th)
        e.rhs(th, out)
        e.sync()
        f = out.cpu().numpy()
        # host pointers give the same result
        fh = np.empty_like(theta)
        e.rhs(np.ascontiguousarray(theta), fh)
        assert np.array_equal(fh, f)
    deg = np.diff(g.row_ptr)
    for b in range(32):
        ref = oracle.rhs_csr(g.row_ptr, g.col, omega[b], theta[b], K[b])
        check_rhs(f[b], ref, deg, K[b], g.n, 1, f"ragged ensemble trajectory {b}")


def test_ensemble_rk4_trajectories_vs_oracle(ragged):
    g = ragged
    omega, K, theta = _inputs(g, 16, 2)
    theta = np.mod(theta, 2 * np.pi)
    steps, h = 20, 0.01
    with kura.KuramotoEnsemble(g.row_ptr, g.col, g.label, g.n_comm, omega, K) as e:
        th = torch.tensor(theta, device="cuda:0")
        e.rk4_steps(th, h, steps)
        e.sync()
        out = th.cpu().numpy()
    for b in (0, 5, 15):
        ref = oracle.rk4_csr(g.row_ptr, g.col, omega[b], K[b], theta[b], h, steps)
        assert np.abs(out[b] - ref).max() < 1e-5, b


def test_ensemble_sbm_matches_oracle_and_single_handles():
    """On an SBM the ensemble's right-hand sides agree with the oracle and with single-trajectory
    mixed-precision handles to FP32-sum rounding."""
    w = G.workload_sbm_small(n=6000, n_comm=6, min_size=128, seed=9)
    g = w.graph
    omega, K, theta = _inputs(g, 16, 3)
    with kura.KuramotoEnsemble(g.row_ptr, g.col, g.label, g.n_comm, omega, K) as e:
        th = torch.tensor(theta, device="cuda:0")
        out = torch.empty_like(th)
        e.rhs(th, out)
        e.sync()
        f = out.cpu().numpy()
    deg = np.diff(g.row_ptr)
    for b in (0, 7, 15):
        with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, omega[b], K[b], precision=kura.PREC_MIXED) as k:
            t1 = torch.tensor(theta[b], device="cuda:0")
            o1 = torch.empty_like(t1)
            k.rhs(t1, o1)
            k.sync()
            f1 = o1.cpu().numpy()
        ref = oracle.rhs_csr(g.row_ptr, g.col, omega[b], theta[b], K[b])
        check_rhs(f[b], ref, deg, K[b], g.n, 1, f"sbm-6000 ensemble trajectory {b} vs oracle")
        check_rhs(f1, ref, deg, K[b], g.n, 1, f"sbm-6000 single handle {b} vs oracle")
        check_rhs(f[b], f1, deg, K[b], g.n, 1, f"sbm-6000 ensemble trajectory {b} vs single handle",
                  e_bound=2e-6)


def test_ensemble_64x65536_sampled_rows_vs_oracle():
    """The benchmarked ensemble shape: 64 trajectories on the 65536-node SBM (64 communities, p_in 0.95,
    p_out 0.001), every dense community on the tensor cores; sampled rows of four trajectories (one per
    group of 16) against the oracle."""
    w = G.workload_sbm_small()
    g = w.graph
    omega, K, theta = _inputs(g, 64, 6)
    with kura.KuramotoEnsemble(g.row_ptr, g.col, g.label, g.n_comm, omega, K) as e:
        assert e.stats()["tc_tiles"] > 0
        th = torch.tensor(theta, device="cuda:0")
        out = torch.empty_like(th)
        e.rhs(th, out)
        e.sync()
        f = out.cpu().numpy()
    rows = np.unique(G.permutation(15, g.n)[:1500].astype(np.int64))
    deg = np.diff(g.row_ptr)[rows]
    for b in (0, 21, 42, 63):
        ref = oracle.rhs_csr(g.row_ptr, g.col, omega[b], theta[b], K[b], rows=rows)
        check_rhs(f[b][rows], ref, deg, K[b], g.n, 1, f"64x65536 ensemble trajectory {b}")


def test_ensemble_rejects_bad_sizes(ragged):
    g = ragged
    omega, K, _ = _inputs(g, 8, 4)
    with pytest.raises(Exception):
        kura.KuramotoEnsemble(g.row_ptr, g.col, g.label, g.n_comm, omega, K)      # 8 is not a multiple of 16


def test_ensemble_rhs_bitwise_repeatable():
    """The ensemble's right-hand side is a fixed function of theta: 100 repeated evaluations for 64
    trajectories on the 65536-node SBM (mask and trajectory images streamed by TMA into two stages)
    are bitwise identical."""
    w = G.workload_sbm_small()
    g = w.graph
    omega, K, theta = _inputs(g, 64, 6)
    with kura.KuramotoEnsemble(g.row_ptr, g.col, g.label, g.n_comm, omega, K) as e:
        th = torch.tensor(theta, device="cuda:0")
        out = torch.empty_like(th)
        e.rhs(th, out)
        e.sync()
        first = out.clone()
        bad = 0
        for _ in range(100):
            e.rhs(th, out)
            e.sync()
            bad += int((out != first).any(dim=1).sum())
    assert bad == 0
