"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle,
element by element on the same seeded inputs.

Tolerances (the stated ones, and the scale-free bound):
  FP64 right-hand side:   |df_i| <= 1e-11 (1 + deg_i)
  mixed right-hand side:  |df_i| <= 2e-4 (1 + deg_i) max(1, |f_i|)
  and, for both, the scale-free error e_i = |df_i| / ((K/calM_i)(1 + deg_i))
  below 1e-10 (FP64) and 1e-6 (mixed), which binds at every N (tests/_parity.py)
  FP64 RK4 trajectories:  |dtheta_i| <= 1e-8
"""
import numpy as np
import pytest

import oracle
from _parity import check_rhs
from paper_2102_07167_gb300 import gen as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2102_07167_gb300 import kura


def _dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda:0")


def _rhs_gpu(sysk, theta):
    th = _dev(theta)
    out = torch.empty_like(th)
    sysk.rhs(th, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1])
def test_rhs_phases_across_the_reduction_ranges(prec):
    """Mixed mode reduces a phase mod 2 pi in 64-bit fixed point for 2^-10 <= |theta| < 2^21 and in FP64
    outside: phases of both signs from 1e-5 to 1e7 rad, the boundaries 2^-10 and 2^21 included, give the
    oracle's right-hand side within the stated bounds (FP64 mode as a control)."""
    w = G.workload_sbm_small(n=12000, n_comm=12, min_size=128, seed=3)
    g = w.graph
    rng = np.random.default_rng(21)
    theta = rng.choice([-1.0, 1.0], g.n) * 10.0 ** rng.uniform(-5, 7, g.n)
    edges = np.array([2.0**-10, np.nextafter(2.0**-10, 0), 2.0**21, np.nextafter(2.0**21, 0), 0.0, np.pi,
                      2 * np.pi, 1e6 * np.pi])
    theta[:edges.size] = edges
    theta[edges.size:2 * edges.size] = -edges
    ref = oracle.rhs_csr(g.row_ptr, g.col, w.omega, theta, w.K)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=prec) as k:
        f = _rhs_gpu(k, theta)
    check_rhs(f, ref, np.diff(g.row_ptr), w.K, g.n, prec, "phases across the reduction ranges")


@pytest.fixture(scope="module")
def sbm_small():
    return G.workload_sbm_small(n=12000, n_comm=12, min_size=128, seed=3)


@pytest.fixture(scope="module")
def sbm_mid():
    return G.workload_sbm_small()            # N = 65536, 64 communities, p_in 0.95, p_out 0.001


@pytest.fixture(scope="module")
def sbm_large():
    return G.workload_sbm_large()            # N = 2^20, 1024 communities


# ----------------------------------------------------------------------------- right-hand side
@pytest.mark.parametrize("prec", [0, 1])
def test_rhs_complete_graph(prec):
    w = G.workload_complete(512)
    g = w.graph
    ref = oracle.rhs_csr(g.row_ptr, g.col, w.omega, w.theta0, w.K)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, 1, w.omega, w.K, precision=prec) as k:
        st = k.stats()
        assert st["dense_blocks"] == 1 and st["missing_entries"] == 0 and st["sparse_entries"] == 0
        f = _rhs_gpu(k, w.theta0)
    check_rhs(f, ref, np.diff(g.row_ptr), w.K, g.n, prec, "complete-512")


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("tau", [0.0, 0.5, 1.0])
def test_rhs_sbm_small_all_tau(sbm_small, prec, tau):
    w = sbm_small
    g = w.graph
    th = w.theta0 + 40.0 * G.uniform(9, 3, g.n, -1, 1)       # unwrapped phases up to ~50 rad
    ref = oracle.rhs_csr(g.row_ptr, g.col, w.omega, th, w.K)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=prec, tau=tau) as k:
        f = _rhs_gpu(k, th)
    check_rhs(f, ref, np.diff(g.row_ptr), w.K, g.n, prec, f"sbm-12000 tau {tau}")


@pytest.mark.parametrize("prec", [0, 1])
def test_rhs_degree_scaling(sbm_small, prec):
    w = sbm_small
    g = w.graph
    ref = oracle.rhs_csr(g.row_ptr, g.col, w.omega, w.theta0, w.K, scaling=1)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, scaling=1, precision=prec) as k:
        f = _rhs_gpu(k, w.theta0)
    deg = np.diff(g.row_ptr)
    check_rhs(f, ref, deg, w.K, np.maximum(deg, 1), prec, "degree scaling")


@pytest.mark.parametrize("prec", [0, 1])
def test_rhs_full_size_65536_sampled_rows(sbm_mid, prec):
    w = sbm_mid
    g = w.graph
    rows = np.unique(G.permutation(5, g.n)[:3000].astype(np.int64))
    ref = oracle.rhs_csr(g.row_ptr, g.col, w.omega, w.theta0, w.K, rows=rows)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=prec) as k:
        f = _rhs_gpu(k, w.theta0)[rows]
    deg = np.diff(g.row_ptr)[rows]
    check_rhs(f, ref, deg, w.K, g.n, prec, "sbm-65536 sampled rows")


@pytest.mark.parametrize("prec", [0, 1])
def test_rhs_full_size_2p20_sampled_rows_and_invariant(sbm_large, prec):
    w = sbm_large
    g = w.graph
    rows = np.unique(G.permutation(6, g.n)[:600].astype(np.int64))
    ref = oracle.rhs_csr(g.row_ptr, g.col, w.omega, w.theta0, w.K, rows=rows)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=prec) as k:
        f_all = _rhs_gpu(k, w.theta0)
    f = f_all[rows]
    deg = np.diff(g.row_ptr)[rows]
    check_rhs(f, ref, deg, w.K, g.n, prec, "sbm-2^20 sampled rows")
    # symmetric A, uniform scaling: the coupling terms sum to zero at any size (Sec. 3).  In units of
    # the largest coupling of the whole graph, K/N sum_i deg_i: rounding level in FP64, and in mixed
    # mode the FP32 terms' errors (about 1e-7 each, random in sign) summed over 1.1e9 entries.
    coupling_sum = np.sum(f_all - w.omega) / (w.K / g.n)
    assert abs(coupling_sum) / g.nnz < (1e-15 if prec == 0 else 1e-9), coupling_sum


@pytest.mark.parametrize("prec", [0, 1])
def test_rhs_window_cap_exceeded_and_ragged(prec):
    """A community larger than the staged window (global-gather path), tiny and empty communities,
    an isolated node, self-loops (dropped) and ragged row lengths."""
    sizes = [5000, 3, 1, 777, 250]
    g = G.sbm(21, sizes, [0.9, 1.0, 0.5, 0.7, 0.2], 0.01)
    lab = g.label.copy()
    n_comm = 6                                  # community 5 is empty
    A_rp, A_col = g.row_ptr.copy(), g.col.copy()
    # add self-loops to a few rows
    rows = [0, 17, 4000]
    rp, cols = [0], []
    for u in range(g.n):
        c = list(A_col[A_rp[u]:A_rp[u + 1]])
        if u in rows:
            c = sorted(c + [u])
        cols += c
        rp.append(len(cols))
    rp, cols = np.array(rp, np.int64), np.array(cols, np.int32)
    omega, theta = G.normal(2, 0, g.n), G.uniform(2, 1, g.n, 0, 6.3)
    ref = oracle.rhs_csr(rp, cols, omega, theta, 2.5)
    with kura.Kuramoto(rp, cols, lab, n_comm, omega, 2.5, precision=prec) as k:
        st = k.stats()
        assert st["self_loops"] == 3
        f = _rhs_gpu(k, theta)
    check_rhs(f, ref, np.diff(rp), 2.5, g.n, prec, "ragged")


def test_single_node_and_edgeless_graph():
    with kura.Kuramoto(np.array([0, 0]), np.zeros(0, np.int32), np.zeros(1, np.int32), 1, np.array([0.7]), 3.0) as k:
        assert np.array_equal(_rhs_gpu(k, np.array([1.0])), [0.7])
    n = 100
    with kura.Kuramoto(np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(n, np.int32), 1,
                       np.arange(n, dtype=float), 1.0) as k:
        assert np.array_equal(_rhs_gpu(k, np.ones(n)), np.arange(n, dtype=float))


def test_host_pointers_match_device(sbm_small):
    w = sbm_small
    g = w.graph
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K) as k:
        f_dev = _rhs_gpu(k, w.theta0)
        f_host = np.empty(g.n)
        k.rhs(np.ascontiguousarray(w.theta0), f_host)
        assert np.array_equal(f_dev, f_host)
        th_h = w.theta0.copy()
        k.rk4_steps(th_h, w.h, 3)
        th_d = _dev(w.theta0)
        k.rk4_steps(th_d, w.h, 3)
        torch.cuda.synchronize()
        assert np.array_equal(th_h, th_d.cpu().numpy())


def test_bitwise_deterministic(sbm_mid):
    w = sbm_mid
    g = w.graph
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=1) as k:
        a = _dev(w.theta0)
        b = _dev(w.theta0)
        k.rk4_steps(a, w.h, 5)
        k.rk4_steps(b, w.h, 5)
        torch.cuda.synchronize()
        assert torch.equal(a, b)


# ----------------------------------------------------------------------------- trajectories
def test_rk4_trajectory_complete_512_full_horizon():
    w = G.workload_complete(512)
    g = w.graph
    ref = oracle.rk4_complete(w.omega, w.K, w.theta0, w.h, w.n_steps)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, 1, w.omega, w.K) as k:
        th = _dev(w.theta0)
        k.rk4_steps(th, w.h, w.n_steps)
        k.sync()
        err = np.abs(th.cpu().numpy() - ref).max()
    assert err <= 1e-8, err


def test_rk4_trajectory_sbm_and_conservation(sbm_small):
    w = sbm_small
    g = w.graph
    steps = 40
    ref = oracle.rk4_csr(g.row_ptr, g.col, w.omega, w.K, w.theta0, w.h, steps)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K) as k:
        th = _dev(w.theta0)
        k.rk4_steps(th, w.h, 17)          # two calls: chunked graphs of different lengths
        k.rk4_steps(th, w.h, steps - 17)
        k.sync()
        got = th.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-8
    assert abs(oracle.mean_deviation(got, w.theta0, w.omega, steps * w.h)) < 1e-12   # eq:KuramotoGraphConservation


def test_rk4_mixed_trajectory_error_vs_fp64(sbm_small):
    w = sbm_small
    g = w.graph
    steps = 40
    ref = oracle.rk4_csr(g.row_ptr, g.col, w.omega, w.K, w.theta0, w.h, steps)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=1) as k:
        th = _dev(w.theta0)
        k.rk4_steps(th, w.h, steps)
        k.sync()
        err = np.abs(th.cpu().numpy() - ref).max()
    assert err < 1e-5, err


def test_rk4_synchronised_state_stays_synchronised():
    g = G.sbm(8, [300, 500, 200], 0.8, 0.02)
    omega = np.full(g.n, 0.37)
    th0 = np.full(g.n, 2.0)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, omega, 3.0) as k:
        th = _dev(th0)
        k.rk4_steps(th, 0.01, 50)
        k.sync()
    np.testing.assert_allclose(th.cpu().numpy(), 2.0 + 0.37 * 0.5, rtol=0, atol=1e-13)


# ----------------------------------------------------------------------------- order parameters, baseline
def test_order_params(sbm_small):
    w = sbm_small
    g = w.graph
    r_o, psi_o, rc_o, pc_o = oracle.order_params(w.theta0, g.label, g.n_comm)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K) as k:
        r, psi, rc, pc = k.order_params(_dev(w.theta0), per_community=True)
    assert abs(r - r_o) < 1e-12 and abs(psi - psi_o) < 1e-10
    np.testing.assert_allclose(rc, rc_o, atol=1e-12, rtol=0)
    np.testing.assert_allclose(pc, pc_o, atol=1e-9, rtol=0)


@pytest.mark.parametrize("prec", [0, 1])
def test_direct_baseline(sbm_small, prec):
    w = sbm_small
    g = w.graph
    ref = oracle.rhs_csr(g.row_ptr, g.col, w.omega, w.theta0, w.K)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K) as k:
        th = _dev(w.theta0)
        out = torch.empty_like(th)
        k.direct_rhs(th, out, prec)
        torch.cuda.synchronize()
        f = out.cpu().numpy()
        check_rhs(f, ref, np.diff(g.row_ptr), w.K, g.n, prec, "direct baseline")
        if prec == 0:
            steps = 10
            ref_t = oracle.rk4_csr(g.row_ptr, g.col, w.omega, w.K, w.theta0, w.h, steps)
            k.direct_rk4_steps(th, w.h, steps, 0)
            torch.cuda.synchronize()
            assert np.abs(th.cpu().numpy() - ref_t).max() <= 1e-8


def test_set_param_and_timing(sbm_small):
    w = sbm_small
    g = w.graph
    om2 = G.normal(77, 0, g.n)
    ref = oracle.rhs_csr(g.row_ptr, g.col, om2, w.theta0, 1.25)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K) as k:
        k.set_param(omega=om2, K=1.25)
        check_rhs(_rhs_gpu(k, w.theta0), ref, np.diff(g.row_ptr), 1.25, g.n, 0, "set_param")
        k.set_timing(True)
        th = _dev(w.theta0)
        k.rk4_steps(th, w.h, 3)
        t = k.kernel_times()
        assert t.size == 12 and np.all(t > 0)


def test_nonfinite_state_is_reported(sbm_small):
    w = sbm_small
    g = w.graph
    th0 = w.theta0.copy()
    th0[5] = np.nan
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K) as k:
        th = _dev(th0)
        k.rk4_steps(th, w.h, 1)
        with pytest.raises(kura.KuraError) as e:
            k.sync()
        assert e.value.status == kura.KURA_ENUMERIC
        k.sync()      # latched condition was cleared


# ----------------------------------------------------------------------------- diagnostics (NEXT-2)
@pytest.mark.parametrize("prec,scaling", [(0, 0), (1, 0), (0, 1)])
def test_potential_vs_oracle(sbm_small, prec, scaling):
    """V of eq:ExtendedPotentialConservation from the block method's row sums (cosine identity) against the
    oracle's edge-by-edge sum."""
    w = sbm_small
    g = w.graph
    ref = oracle.potential_csr(g.row_ptr, g.col, w.omega, w.theta0, w.K, scaling)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=prec, scaling=scaling) as k:
        V = k.potential(_dev(w.theta0))
        Vh = k.potential(np.ascontiguousarray(w.theta0))
    assert V == Vh
    tol = (1e-9 if prec == 0 else 1e-5) * max(1.0, abs(ref))
    assert abs(V - ref) <= tol, (V, ref)


def test_potential_decreases_and_mean_is_conserved(sbm_small):
    """Symmetric A, uniform scaling: the flow is a gradient flow of V (V non-increasing along the RK4
    trajectory, up to the integrator's error) and the mean deviation of eq:Means stays zero."""
    w = sbm_small
    g = w.graph
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=0) as k:
        th = _dev(w.theta0)
        th0 = th.clone()
        Vs = [k.potential(th)]
        for _ in range(5):
            k.rk4_steps(th, w.h, 10)
            Vs.append(k.potential(th))
        md = k.mean_deviation(th, th0, 50 * w.h)
    assert all(b <= a + 1e-9 * max(1.0, abs(a)) for a, b in zip(Vs, Vs[1:])), Vs
    assert abs(md) < 1e-10, md
    ref_md = oracle.mean_deviation(th.cpu().numpy(), w.theta0, w.omega, 50 * w.h)
    assert abs(md - ref_md) < 1e-12


# ----------------------------------------------------------------------------- second-order integrators (NEXT-3)
@pytest.mark.parametrize("method", [1, 2])
def test_second_order_integrators_vs_oracle(sbm_small, method):
    """Explicit midpoint (1) and implicit midpoint (2, 4 sweeps) in FP64 against the oracle's."""
    w = sbm_small
    g = w.graph
    steps = 30
    ref = oracle.rk2_csr(g.row_ptr, g.col, w.omega, w.K, w.theta0, w.h, steps, method - 1, 4)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=0) as k:
        th = _dev(w.theta0)
        k.integrate(th, w.h, steps, method, 4)
        k.sync()
        out = th.cpu().numpy()
        # host pointer path
        thh = np.ascontiguousarray(w.theta0).copy()
        k.integrate(thh, w.h, steps, method, 4)
    assert np.abs(out - ref).max() < 1e-8
    assert np.array_equal(out, thh)


def test_long_horizon_mean_deviation_second_order():
    """Classical all-to-all model (N = 512, K = 5, the paper's long-term setting shape): both second-order
    methods keep the linear invariant of eq:5c to rounding over 20000 steps; the drift is measured."""
    w = G.workload_complete(512)
    g = w.graph
    h, steps = 0.01, 20000
    drift = {}
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, 5.0, precision=0) as k:
        for method in (1, 2):
            th = _dev(w.theta0)
            k.integrate(th, h, steps, method, 4)
            drift[method] = abs(k.mean_deviation(th, _dev(w.theta0), h * steps))
    assert drift[1] < 1e-9 and drift[2] < 1e-9, drift


@pytest.mark.parametrize("prec,scaling", [(0, 0), (1, 0), (0, 1)])
def test_small_graph_cluster_step_loop_vs_oracle(prec, scaling):
    """Small graphs run every RK4 step in one launch of one thread-block cluster (8 CTAs, the table spread over
    their shared memory): a 2000-node SBM with dense and sparse blocks (listed missing and present entries
    gathered across CTAs) and the complete graph, against the oracle and against the CUDA-graph step loop."""
    cases = [G.workload_sbm_small(n=2000, n_comm=8, min_size=128, seed=12), G.workload_complete(512)]
    for w in cases:
        g = w.graph
        steps = 40
        ref = oracle.rk4_csr(g.row_ptr, g.col, w.omega, w.K, w.theta0, w.h, steps, scaling)
        out = {}
        for ps in (1, 0):
            with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=prec,
                               persistent_small=ps, scaling=scaling) as k:
                th = _dev(w.theta0)
                k.rk4_steps(th, w.h, steps)
                k.sync()
                out[ps] = th.cpu().numpy()
        deg = np.diff(g.row_ptr)
        calm = np.maximum(deg, 1) if scaling else g.n
        bound = 1e-8 if prec == 0 else 2 * 1e-6 * np.max(w.K / calm * (1 + deg)) * w.h * steps
        for ps in (1, 0):
            assert np.abs(out[ps] - ref).max() <= bound, (w.name, ps, np.abs(out[ps] - ref).max(), bound)
        if prec == 0:
            # both loops use exact fixed-point sums of the same FP64 sin/cos: the same trajectory
            assert np.abs(out[1] - out[0]).max() <= 1e-12
