"""Pins for the FP64 CPU oracle: it is checked against what the paper and the
mathematics fix (hand-derived values, closed forms, invariants, special cases,
brute force on tiny inputs), never against itself.  CPU only."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_2102_07167_gb300 import gen as G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _csr_from_edges(n, edges):
    A = np.zeros((n, n), dtype=np.uint8)
    for m, l in edges:
        A[m, l] = 1
    return A, G.from_dense(A)


def _random_directed(rng, n, p_one, symmetric=False):
    A = (rng.random((n, n)) < p_one).astype(np.uint8)
    np.fill_diagonal(A, 0)
    if symmetric:
        A = np.triu(A, 1)
        A = A + A.T
    return A


# ----------------------------------------------------------------------------- hand-derived values
@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLDEN, "hand_examples.json")))["cases"],
                         ids=lambda c: c["name"])
def test_hand_worked_examples(case):
    """eq:KuramotoGraph on graphs small enough to evaluate by hand."""
    n = case["n"]
    A, g = _csr_from_edges(n, case["edges"])
    theta = (np.array(case["theta_over_half_pi"], float) * np.pi / 2) if "theta_over_half_pi" in case \
        else np.array(case["theta"], float)
    omega = np.array(case["omega"], float)
    exp = np.array(case["expected"])
    for f in (oracle.rhs_dense(A, omega, theta, case["K"], case["scaling"]),
              oracle.rhs_csr(g.row_ptr, g.col, omega, theta, case["K"], case["scaling"])):
        np.testing.assert_allclose(f, exp, rtol=0, atol=2e-15)
    if case["scaling"] == 0:
        fb, _ = oracle.rhs_block(g.row_ptr, g.col, np.zeros(n, np.int32), 1, omega, theta, case["K"])
        np.testing.assert_allclose(fb, exp, rtol=0, atol=2e-15)


# ----------------------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [2, 7, 64, 301])
def test_complete_graph_matches_order_parameter_closed_form(n):
    """eq:OrderParameter: (1/M) sum_l sin(theta_l - theta_m) = r sin(psi - theta_m), so on the complete
    graph f_m - omega_m = K r sin(psi - theta_m); r, psi from numpy's complex mean (independent route)."""
    rng = np.random.default_rng(n)
    theta = rng.uniform(-10, 10, n)
    omega = rng.normal(size=n)
    K = 2.5
    z = np.mean(np.exp(1j * theta))
    expect = omega + K * np.abs(z) * np.sin(np.angle(z) - theta)
    g = G.complete(n)
    np.testing.assert_allclose(oracle.rhs_csr(g.row_ptr, g.col, omega, theta, K), expect, rtol=0, atol=1e-13)
    np.testing.assert_allclose(oracle.rhs_complete_op(omega, theta, K), expect, rtol=0, atol=1e-13)
    fb, st = oracle.rhs_block(g.row_ptr, g.col, g.label, 1, omega, theta, K)
    np.testing.assert_allclose(fb, expect, rtol=0, atol=1e-13)
    if n > 2:  # n = 2: zero fraction exactly 1/2 (the diagonal), a tie, which goes to the sparse rule
        assert st["dense_blocks"] == 1 and st["nonzero_terms"] == 0 and st["zero_terms"] == n  # the diagonal


def test_order_parameters_against_complex_mean():
    rng = np.random.default_rng(3)
    theta = rng.uniform(0, 2 * np.pi, 1000)
    label = rng.integers(0, 5, 1000).astype(np.int32)
    r, psi, rc, pc = oracle.order_params(theta, label, 5)
    z = np.mean(np.exp(1j * theta))
    assert abs(r - abs(z)) < 1e-14 and abs(psi - np.angle(z)) < 1e-13
    for I in range(5):
        zi = np.mean(np.exp(1j * theta[label == I]))
        assert abs(rc[I] - abs(zi)) < 1e-14 and abs(pc[I] - np.angle(zi)) < 1e-13
    # splay state: r = 0 exactly in exact arithmetic, psi reported as 0 when r == 0
    r0, _ = oracle.order_params(np.array([0.0, np.pi / 2, np.pi, 3 * np.pi / 2]))
    assert r0 < 1e-15


def test_trig_counts_table1():
    """Table 1 / eq:EulerCost: the original formulation costs M(M-1) sine evaluations per right-hand side,
    the reformulation with precomputed sums 4M."""
    M = 40
    g = G.complete(M)
    th, om = np.linspace(0, 3, M), np.zeros(M)
    oracle.trig_count_reset()
    oracle.rhs_csr(g.row_ptr, g.col, om, th, 1.0)
    assert oracle.trig_count() == M * (M - 1)
    oracle.trig_count_reset()
    oracle.rhs_complete_op(om, th, 1.0)
    assert oracle.trig_count() == 4 * M


# ----------------------------------------------------------------------------- brute force, tiny inputs
def test_all_symmetric_graphs_n4_all_labellings():
    """Every symmetric 0/1 graph on 4 nodes (64 graphs) x every labelling into <= 2 communities x several tau:
    the block rule equals the brute-force definition."""
    n = 4
    pairs = list(itertools.combinations(range(n), 2))
    rng = np.random.default_rng(11)
    theta = rng.uniform(0, 2 * np.pi, n)
    omega = rng.normal(size=n)
    for bits in range(1 << len(pairs)):
        A = np.zeros((n, n), np.uint8)
        for k, (a, b) in enumerate(pairs):
            if bits >> k & 1:
                A[a, b] = A[b, a] = 1
        g = G.from_dense(A)
        f_ref = oracle.rhs_dense(A, omega, theta, 1.7, 0)
        np.testing.assert_allclose(oracle.rhs_csr(g.row_ptr, g.col, omega, theta, 1.7), f_ref, atol=1e-15, rtol=0)
        for lab in itertools.product(range(2), repeat=n):
            for tau in (0.0, 0.5, 1.01):
                fb, _ = oracle.rhs_block(g.row_ptr, g.col, np.array(lab, np.int32), 2, omega, theta, 1.7, 0, tau)
                np.testing.assert_allclose(fb, f_ref, atol=1e-14, rtol=0)


@pytest.mark.parametrize("seed", range(12))
def test_random_directed_graphs_three_ways(seed):
    """Random directed graphs, 6..16 nodes, random labels, random density: dense brute force, CSR and block
    rule agree; both scalings."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(6, 17))
    A = _random_directed(rng, n, rng.uniform(0.05, 0.95))
    g = G.from_dense(A)
    nc = int(rng.integers(1, 5))
    lab = rng.integers(0, nc, n).astype(np.int32)
    theta = rng.uniform(-20, 20, n)
    omega = rng.normal(size=n)
    deg = A.sum(1)
    for scaling in (0, 1):
        f_ref = oracle.rhs_dense(A, omega, theta, 3.0, scaling)
        np.testing.assert_allclose(oracle.rhs_csr(g.row_ptr, g.col, omega, theta, 3.0, scaling), f_ref,
                                   atol=1e-14, rtol=0)
        for tau in (0.0, 0.3, 0.5, 0.7, 1.01):
            fb, _ = oracle.rhs_block(g.row_ptr, g.col, lab, nc, omega, theta, 3.0, scaling, tau)
            assert np.all(np.abs(fb - f_ref) <= 1e-14 * (1 + deg) * 4)


def test_four_block_flip_matrix_block_rule():
    """The paper's community-detection test matrix (Sec. 3): block diagonal with sizes (5-k)M/10, entries
    flipped with probability p; the block rule over the planted communities equals the CSR definition."""
    M, p = 200, 0.15
    rng = np.random.default_rng(5)
    sizes = [(5 - k) * M // 10 for k in range(1, 5)]
    lab = np.repeat(np.arange(4), sizes).astype(np.int32)
    B = (lab[:, None] == lab[None, :]).astype(np.uint8)
    A = np.where(rng.random((M, M)) < p, 1 - B, B).astype(np.uint8)
    np.fill_diagonal(A, 0)
    g = G.from_dense(A, lab, 4)
    theta = rng.uniform(0, 2 * np.pi, M)
    omega = rng.normal(size=M)
    f_ref = oracle.rhs_csr(g.row_ptr, g.col, omega, theta, 4.0)
    fb, st = oracle.rhs_block(g.row_ptr, g.col, lab, 4, omega, theta, 4.0)
    np.testing.assert_allclose(fb, f_ref, atol=1e-13, rtol=0)
    assert st["dense_blocks"] == 4 and st["sparse_blocks"] == 12
    # stored work equals the entries of C = A - B (flips) plus the diagonal zeros: cost measure eq:QuantityPerformance
    flips = int(np.abs(A.astype(int) - B.astype(int)).sum())
    assert st["zero_terms"] + st["nonzero_terms"] == flips


@pytest.mark.parametrize("p", [0.1, 0.3, 0.45, 0.55, 0.7, 0.9])
def test_unstructured_matrix_dense_sparse_crossover(p):
    """Unstructured random matrices, A = 1 iff z > p (Sec. 3): the block rule takes the dense route exactly
    when ones outnumber zeros, and then its stored work is the zeros, else the ones (crossover at 0.5)."""
    rng = np.random.default_rng(int(p * 1000))
    M = 120
    A = (rng.random((M, M)) > p).astype(np.uint8)
    np.fill_diagonal(A, 0)
    g = G.from_dense(A)
    theta = 2 * np.pi * np.arange(1, M + 1) / M
    omega = np.zeros(M)
    fb, st = oracle.rhs_block(g.row_ptr, g.col, np.zeros(M, np.int32), 1, omega, theta, 1.0)
    np.testing.assert_allclose(fb, oracle.rhs_dense(A, omega, theta, 1.0), atol=1e-13, rtol=0)
    ones = int(A.sum())
    zeros = M * M - ones
    if zeros < ones:
        assert st["dense_blocks"] == 1 and st["zero_terms"] == zeros and st["nonzero_terms"] == 0
    else:
        assert st["sparse_blocks"] == 1 and st["nonzero_terms"] == ones and st["zero_terms"] == 0


# ----------------------------------------------------------------------------- invariants
@pytest.mark.parametrize("seed", range(4))
def test_symmetric_uniform_coupling_sums_to_zero(seed):
    """Sec. 3, uniform scaling: A = A^T makes the coupling terms cancel pairwise, sum_m (f_m - omega_m) = 0;
    a directed graph does not (the test can tell the two apart)."""
    rng = np.random.default_rng(seed)
    n = 150
    theta = rng.uniform(0, 2 * np.pi, n)
    omega = rng.normal(size=n)
    gs = G.from_dense(_random_directed(rng, n, 0.3, symmetric=True))
    fs = oracle.rhs_csr(gs.row_ptr, gs.col, omega, theta, 5.0)
    assert abs(np.sum(fs - omega)) < 1e-12
    gd = G.from_dense(_random_directed(rng, n, 0.3))
    fd = oracle.rhs_csr(gd.row_ptr, gd.col, omega, theta, 5.0)
    assert abs(np.sum(fd - omega)) > 1e-3


def test_synchronised_state_has_no_coupling():
    """Identical phases: every sin(theta_l - theta_m) is sin(0) = 0, so f = omega exactly, on any graph."""
    w = G.workload_sbm_small(n=3000, n_comm=6, min_size=100)
    th = np.full(w.graph.n, 1.234)
    f = oracle.rhs_csr(w.graph.row_ptr, w.graph.col, w.omega, th, 4.0)
    assert np.array_equal(f, w.omega)
    fb, _ = oracle.rhs_block(w.graph.row_ptr, w.graph.col, w.graph.label, w.graph.n_comm, w.omega, th, 4.0)
    np.testing.assert_allclose(fb, w.omega, atol=1e-12, rtol=0)


def test_decoupled_block_degree_scaling():
    """Sec. 3 non-uniform scaling example: an all-ones block on the first M0 nodes, zero elsewhere.  The rest
    is decoupled (f = omega exactly); the block is the classical model on M0 oscillators with the degree
    M0 - 1 as scaling, i.e. eq:KuramotoReformulation with K' = K M0 / (M0 - 1)."""
    M, M0, K = 50, 20, 3.0
    A = np.zeros((M, M), np.uint8)
    A[:M0, :M0] = 1
    np.fill_diagonal(A, 0)
    g = G.from_dense(A)
    rng = np.random.default_rng(2)
    theta, omega = rng.uniform(0, 6, M), rng.normal(size=M)
    f = oracle.rhs_csr(g.row_ptr, g.col, omega, theta, K, 1)
    assert np.array_equal(f[M0:], omega[M0:])
    np.testing.assert_allclose(f[:M0], oracle.rhs_complete_op(omega[:M0], theta[:M0], K * M0 / (M0 - 1)),
                               atol=1e-14, rtol=0)


def test_gradient_structure_of_potential():
    """Sec. 2-3: for symmetric A with uniform scaling the right-hand side is -grad V with V of
    eq:ExtendedPotentialConservation; central differences of the oracle's V reproduce the oracle's f."""
    rng = np.random.default_rng(9)
    n = 40
    g = G.from_dense(_random_directed(rng, n, 0.4, symmetric=True))
    theta, omega, K = rng.uniform(0, 2 * np.pi, n), rng.normal(size=n), 2.0
    f = oracle.rhs_csr(g.row_ptr, g.col, omega, theta, K)
    eps = 1e-6
    grad = np.empty(n)
    for k in range(n):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        grad[k] = (oracle.potential_csr(g.row_ptr, g.col, omega, tp, K)
                   - oracle.potential_csr(g.row_ptr, g.col, omega, tm, K)) / (2 * eps)
    np.testing.assert_allclose(-grad, f, atol=1e-7, rtol=0)


def test_classical_potential_closed_form():
    """eq:Potential: on the complete graph V = -omega^T theta + (K M / 2)(1 - C_M^2 - S_M^2)."""
    M = 64
    rng = np.random.default_rng(4)
    theta, omega, K = rng.uniform(0, 2 * np.pi, M), rng.normal(size=M), 1.5
    g = G.complete(M)
    z = np.mean(np.exp(1j * theta))
    V_closed = -omega @ theta + 0.5 * K * M * (1 - abs(z) ** 2)
    assert abs(oracle.potential_csr(g.row_ptr, g.col, omega, theta, K) - V_closed) < 1e-11


# ----------------------------------------------------------------------------- time integration
def test_rk4_free_rotation_when_uncoupled():
    """K = 0: theta(t) = theta0 + omega t."""
    w = G.workload_sbm_small(n=2000, n_comm=4, min_size=100)
    th = oracle.rk4_csr(w.graph.row_ptr, w.graph.col, w.omega, 0.0, w.theta0, 0.01, 50)
    np.testing.assert_allclose(th, w.theta0 + 0.5 * w.omega, atol=1e-13, rtol=0)


def _adler_phi(phi0, a, b, t):
    """Exact solution of phi' = a - b sin(phi) (two coupled oscillators, phi = theta_2 - theta_1)."""
    if a * a > b * b:
        s = np.sqrt(a * a - b * b)
        # tan(phi/2) = (b + s tan(s (t + c)/2)) / a
        c = 2 * np.arctan((a * np.tan(phi0 / 2) - b) / s) / s
        x = (b + s * np.tan(s * (t + c) / 2)) / a
        return 2 * np.arctan(x)
    s = np.sqrt(b * b - a * a)
    # tan(phi/2) = (b - s tanh(s (t + c)/2)) / a
    c = 2 * np.arctanh((b - a * np.tan(phi0 / 2)) / s) / s
    return 2 * np.arctan((b - s * np.tanh(s * (t + c) / 2)) / a)


@pytest.mark.parametrize("dw", [0.5, 3.0])
def test_rk4_two_oscillators_adler_closed_form(dw):
    """M = 2, uniform scaling: phi = theta_2 - theta_1 obeys phi' = dw - K sin(phi) (Adler equation, closed form),
    theta_1 + theta_2 advances as (omega_1 + omega_2) t (eq:5c).  RK4 error shrinks ~16x when h halves."""
    K, T = 2.0, 1.0
    omega = np.array([0.3, 0.3 + dw])
    th0 = np.array([0.2, 0.9])
    g = G.complete(2)
    phi_ex = _adler_phi(th0[1] - th0[0], dw, K, T)
    errs = []
    for nst in (40, 80, 160, 320):
        th = oracle.rk4_csr(g.row_ptr, g.col, omega, K, th0, T / nst, nst)
        assert abs((th[0] + th[1]) - (th0.sum() + omega.sum() * T)) < 1e-13
        errs.append(abs((th[1] - th[0]) - phi_ex))
    assert errs[-1] < 1e-11
    ratios = [e1 / e2 for e1, e2 in zip(errs, errs[1:])]
    assert all(r > 10 for r in ratios) and 14 < ratios[-1] < 18, errs  # fourth order: ratio -> 16


def test_rk4_conserves_mean_symmetric_uniform():
    """eq:KuramotoGraphConservation: symmetric A, uniform scaling keep (1/M) sum (theta(t) - theta(0) - t omega)
    at zero; RK4 preserves linear invariants, so only rounding remains."""
    w = G.workload_sbm_small(n=3000, n_comm=6, min_size=100)
    n_steps, h = 40, 0.01
    th = oracle.rk4_csr(w.graph.row_ptr, w.graph.col, w.omega, w.K, w.theta0, h, n_steps)
    assert abs(oracle.mean_deviation(th, w.theta0, w.omega, n_steps * h)) < 1e-13


def test_rk4_potential_nonincreasing():
    """Sec. 2: V(theta(t)) decreases in time for the gradient system (symmetric A, uniform scaling)."""
    w = G.workload_sbm_small(n=1500, n_comm=5, min_size=100)
    g = w.graph
    th = w.theta0.copy()
    V = [oracle.potential_csr(g.row_ptr, g.col, w.omega, th, w.K)]
    for _ in range(20):
        th = oracle.rk4_csr(g.row_ptr, g.col, w.omega, w.K, th, 0.01, 1)
        V.append(oracle.potential_csr(g.row_ptr, g.col, w.omega, th, w.K))
    assert np.all(np.diff(V) < 0)


def test_rk4_complete_vs_csr_paths():
    """The two integrator front ends (order-parameter RHS, CSR RHS) follow the same trajectory."""
    w = G.workload_complete(n=64)
    a = oracle.rk4_complete(w.omega, w.K, w.theta0, w.h, 30)
    b = oracle.rk4_csr(w.graph.row_ptr, w.graph.col, w.omega, w.K, w.theta0, w.h, 30)
    np.testing.assert_allclose(a, b, atol=1e-12, rtol=0)


def _locked_r(K, gamma):
    """Fully locked state for frequencies uniform on an interval of half-width gamma: with u = gamma/(K r),
    1 = (K / (2 gamma)) (u sqrt(1 - u^2) + asin u) (self-consistency of eq:OrderParameter)."""
    from scipy.optimize import brentq
    u = brentq(lambda u: K / (2 * gamma) * (u * np.sqrt(1 - u * u) + np.arcsin(u)) - 1, 1e-9, 1.0)
    return gamma / (K * u)


@pytest.mark.parametrize("K", [3.0, 5.0])
def test_paper_classical_runs_synchronise(K):
    """Sec. 2 numerical integration with the paper's inputs (omega_0 = 2, theta_m(0) = 2 pi m / M, T = 200):
    for K = 3 and 5 the oscillators lock and r(T) approaches the locked-state value of the uniform frequency
    density on [1 - 2, 1 + 2]; K = 1 stays incoherent."""
    M = 400
    omega, theta0 = G.paper_e2_inputs(M, 2.0)
    th = oracle.rk4_complete(omega, K, theta0, 0.05, 4000)
    r, _ = oracle.order_params(th)
    assert abs(r - _locked_r(K, 2.0)) < 0.01
    th1 = oracle.rk4_complete(omega, 1.0, theta0, 0.05, 4000)
    assert oracle.order_params(th1)[0] < 0.1


# ----------------------------------------------------------------------------- discrete adjoint
@pytest.mark.parametrize("directed", [False, True])
@pytest.mark.parametrize("loss_kind", [0, 1])
def test_adjoint_matches_central_finite_differences(loss_kind, directed):
    """The oracle's discrete RK4 adjoint against central differences of the oracle's own forward loss
    (eps = 1e-6): directional derivatives in theta0 and omega, and the K derivative; on a symmetric SBM and
    on a directed one (each edge kept in one direction with probability 0.6), where J^T differs from J."""
    rng = np.random.default_rng(21 + loss_kind)
    g = G.sbm(5, [30, 25, 20], [0.8, 0.7, 0.9], 0.1)
    if directed:
        A = np.zeros((g.n, g.n), np.uint8)
        for u in range(g.n):
            A[u, g.col[g.row_ptr[u]:g.row_ptr[u + 1]]] = 1
        A[np.random.default_rng(7).random(A.shape) < 0.4] = 0
        assert (A != A.T).any()
        g = G.from_dense(A, g.label, g.n_comm)
    n = g.n
    omega, theta0 = rng.normal(size=n), rng.uniform(0, 2 * np.pi, n)
    K, h, steps = 3.0, 0.02, 15
    target = theta0 + 0.3 * rng.normal(size=n) if loss_kind == 1 else None
    L, g_om, g_K, g_th = oracle.adjoint_rk4_csr(g.row_ptr, g.col, omega, K, theta0, h, steps, loss_kind, target)
    f = lambda om, KK, th: oracle.loss_rk4_csr(g.row_ptr, g.col, om, KK, th, h, steps, loss_kind, target)
    assert abs(L - f(omega, K, theta0)) < 1e-13
    eps = 1e-6
    for _ in range(4):
        d = rng.normal(size=n)
        fd = (f(omega, K, theta0 + eps * d) - f(omega, K, theta0 - eps * d)) / (2 * eps)
        assert abs(fd - g_th @ d) <= 1e-7 * (1 + abs(fd))
        fd = (f(omega + eps * d, K, theta0) - f(omega - eps * d, K, theta0)) / (2 * eps)
        assert abs(fd - g_om @ d) <= 1e-7 * (1 + abs(fd))
    fd = (f(omega, K + eps, theta0) - f(omega, K - eps, theta0)) / (2 * eps)
    assert abs(fd - g_K) <= 1e-7 * (1 + abs(fd))


def test_adjoint_uncoupled_closed_form():
    """K = 0: theta(T) = theta0 + T omega, so for L = 1/2 ||theta(T) - target||^2 the gradients are
    dL/dtheta0 = theta(T) - target and dL/domega = T (theta(T) - target) exactly."""
    rng = np.random.default_rng(3)
    g = G.sbm(6, [40, 30], 0.5, 0.1)
    n = g.n
    omega, theta0, target = rng.normal(size=n), rng.uniform(0, 6, n), rng.normal(size=n)
    h, steps = 0.05, 20
    T = h * steps
    L, g_om, g_K, g_th = oracle.adjoint_rk4_csr(g.row_ptr, g.col, omega, 0.0, theta0, h, steps, 1, target)
    resid = theta0 + T * omega - target
    np.testing.assert_allclose(g_th, resid, atol=1e-12, rtol=0)
    np.testing.assert_allclose(g_om, T * resid, atol=1e-12, rtol=0)
    assert abs(L - 0.5 * resid @ resid) < 1e-11


# ----------------------------------------------------------------------------- second-order integrators (NEXT-3)
@pytest.mark.parametrize("method", [0, 1])
def test_rk2_free_rotation_when_uncoupled(method):
    """K = 0: both second-order methods integrate theta' = omega exactly."""
    w = G.workload_sbm_small(n=1000, n_comm=4, min_size=100)
    th = oracle.rk2_csr(w.graph.row_ptr, w.graph.col, w.omega, 0.0, w.theta0, 0.01, 50, method, 3)
    np.testing.assert_allclose(th, w.theta0 + 0.5 * w.omega, atol=1e-13, rtol=0)


@pytest.mark.parametrize("method", [0, 1])
def test_rk2_two_oscillators_adler_second_order(method):
    """M = 2 against the Adler closed form: the error shrinks ~4x when h halves (second order), and
    theta_1 + theta_2 advances exactly as (omega_1 + omega_2) t (linear invariant, eq:5c)."""
    K, T, dw = 2.0, 1.0, 0.5
    omega = np.array([0.3, 0.3 + dw])
    th0 = np.array([0.2, 0.9])
    g = G.complete(2)
    phi_ex = _adler_phi(th0[1] - th0[0], dw, K, T)
    errs = []
    for nst in (40, 80, 160, 320):
        th = oracle.rk2_csr(g.row_ptr, g.col, omega, K, th0, T / nst, nst, method, 12)
        assert abs((th[0] + th[1]) - (th0.sum() + omega.sum() * T)) < 1e-13
        errs.append(abs((th[1] - th[0]) - phi_ex))
    ratios = [e1 / e2 for e1, e2 in zip(errs, errs[1:])]
    assert all(3.5 < r < 4.5 for r in ratios), (errs, ratios)


def test_implicit_midpoint_solves_its_stage_equation_and_is_symmetric():
    """Implicit midpoint: the step satisfies y' = y + h f((y + y')/2) (residual at rounding level after enough
    sweeps), and a step with h followed by one with -h returns to y (a symmetric method); explicit midpoint
    does not return."""
    w = G.workload_sbm_small(n=800, n_comm=4, min_size=100)
    g, h = w.graph, 0.02
    y1 = oracle.rk2_csr(g.row_ptr, g.col, w.omega, w.K, w.theta0, h, 1, 1, 30)
    f_mid = oracle.rhs_csr(g.row_ptr, g.col, w.omega, 0.5 * (w.theta0 + y1), w.K)
    assert np.max(np.abs(y1 - w.theta0 - h * f_mid)) < 1e-13
    back = oracle.rk2_csr(g.row_ptr, g.col, w.omega, w.K, y1, -h, 1, 1, 30)
    assert np.max(np.abs(back - w.theta0)) < 1e-12
    ye = oracle.rk2_csr(g.row_ptr, g.col, w.omega, w.K, w.theta0, h, 1, 0, 1)
    backe = oracle.rk2_csr(g.row_ptr, g.col, w.omega, w.K, ye, -h, 1, 0, 1)
    assert np.max(np.abs(backe - w.theta0)) > 1e-9


# ----------------------------------------------------------------------------- finite-valued adjacency (NEXT-4)
def _valued_block_matrix(rng, sizes, vals, noise, max_val):
    """Block matrix whose block (I, J) mostly holds vals[I][J] (0..max_val), with a fraction `noise` of entries
    replaced by uniform values in 0..max_val; zero diagonal."""
    sizes = np.asarray(sizes)
    lab = np.repeat(np.arange(len(sizes)), sizes)
    n = lab.size
    A = np.asarray(vals, dtype=np.int32)[lab][:, lab]
    flip = rng.random((n, n)) < noise
    A[flip] = rng.integers(0, max_val + 1, int(flip.sum()))
    np.fill_diagonal(A, 0)
    return A.astype(np.int32), lab.astype(np.int32)


def _csr_values(A):
    rows, cols = np.nonzero(A)
    row_ptr = np.zeros(A.shape[0] + 1, np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    return np.cumsum(row_ptr), cols.astype(np.int32), A[rows, cols].astype(np.int32)


@pytest.mark.parametrize("seed", range(4))
def test_valued_block_rule_matches_definition(seed):
    """Sec. 1 (Generalisations): for A in {0..3} with one prevalent value per block, the prevalent-value block
    rule equals the definition (CSR and brute force) for every tau; the detected block values are the planted
    ones where the noise leaves them prevalent."""
    rng = np.random.default_rng(seed)
    vals = [[2, 0, 1], [0, 3, 0], [1, 0, 1]]
    A, lab = _valued_block_matrix(rng, [20, 15, 25], vals, 0.2, 3)
    perm = rng.permutation(A.shape[0])
    A, lab = A[perm][:, perm], lab[perm]
    rp, cl, vl = _csr_values(A)
    omega, theta = rng.normal(size=A.shape[0]), rng.uniform(-20, 20, A.shape[0])
    ref = oracle.rhs_valued_dense(A, omega, theta, 1.7)
    np.testing.assert_allclose(oracle.rhs_valued_csr(rp, cl, vl, omega, theta, 1.7), ref, atol=1e-13, rtol=0)
    for tau in (0.0, 0.3, 0.5, 0.8, 1.0):
        f, bv = oracle.rhs_block_valued(rp, cl, vl, 3, lab, 3, omega, theta, 1.7, tau)
        np.testing.assert_allclose(f, ref, atol=1e-12, rtol=0)
        if tau == 0.5:
            assert np.array_equal(bv, np.asarray(vals))


def test_valued_rule_reduces_to_binary_rule():
    """With values in {0, 1} the valued rule is the 0/1 block rule of eq:KuramotoGraphApproach."""
    w = G.workload_sbm_small(n=600, n_comm=4, min_size=80)
    g = w.graph
    val = np.ones(g.col.shape[0], np.int32)
    f, _ = oracle.rhs_block_valued(g.row_ptr, g.col, val, 1, g.label, g.n_comm, w.omega, w.theta0, w.K)
    f01, _ = oracle.rhs_block(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.theta0, w.K)
    np.testing.assert_allclose(f, f01, atol=1e-12, rtol=0)
