"""GPU parity for finite-valued adjacency (Sec. 1, Generalisations: A_ml in {0..J}, one prevalent value per
block; kura_create_valued) against the oracle's definition."""
import numpy as np
import pytest

import oracle
from _parity import check_rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2102_07167_gb300 import kura


def _valued_graph(seed, sizes, max_val, noise):
    rng = np.random.default_rng(seed)
    k = len(sizes)
    V = rng.integers(0, max_val + 1, (k, k))
    V = np.maximum(V, V.T)                                   # symmetric block values
    lab = np.repeat(np.arange(k), sizes)
    A = V[lab][:, lab].astype(np.int32)
    flip = np.triu(rng.random(A.shape) < noise, 1)
    vals = rng.integers(0, max_val + 1, A.shape)
    A[flip] = vals[flip]
    A = np.triu(A, 1)
    A = A + A.T
    perm = rng.permutation(A.shape[0])
    A, lab = A[perm][:, perm], lab[perm].astype(np.int32)
    rows, cols = np.nonzero(A)
    rp = np.zeros(A.shape[0] + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    return np.cumsum(rp), cols.astype(np.int32), A[rows, cols].astype(np.int32), lab, k


@pytest.fixture(scope="module")
def valued():
    return _valued_graph(3, [300, 513, 129, 700, 60, 1030], 5, 0.2)


def _dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda:0")


@pytest.mark.parametrize("prec", [0, 1])
def test_valued_rhs_vs_oracle(valued, prec):
    rp, cl, vl, lab, k = valued
    n = rp.shape[0] - 1
    rng = np.random.default_rng(prec)
    omega, theta, K = rng.normal(size=n), rng.uniform(-30, 30, n), 2.0
    ref = oracle.rhs_valued_csr(rp, cl, vl, omega, theta, K)
    with kura.Kuramoto(rp, cl, lab, k, omega, K, precision=prec, val=vl) as h:
        st = h.stats()
        assert st["dense_blocks"] > 0 and st["tc_tiles"] == 0
        th = _dev(theta)
        out = torch.empty_like(th)
        h.rhs(th, out)
        h.sync()
        f = out.cpu().numpy()
        # re-classification with another tau keeps the values
        h.classify_blocks(0.3)
        h.rhs(th, out)
        h.sync()
        f2 = out.cpu().numpy()
    # weighted degree sum_l A_ml: the largest coupling a row can have is (K/n) times it
    wdeg = np.add.reduceat(vl, rp[:-1]) if vl.size else np.zeros(n)
    check_rhs(f, ref, wdeg, K, n, prec, "valued")
    check_rhs(f2, ref, wdeg, K, n, prec, "valued after re-classification")


def test_valued_rk4_and_refused_calls(valued):
    rp, cl, vl, lab, k = valued
    n = rp.shape[0] - 1
    rng = np.random.default_rng(7)
    omega, theta = rng.normal(size=n), rng.uniform(0, 2 * np.pi, n)
    K, h, steps = 1.5, 0.01, 15
    # classical RK4 with the oracle's valued right-hand side
    y = theta.copy()
    f = lambda x: oracle.rhs_valued_csr(rp, cl, vl, omega, x, K)
    for _ in range(steps):
        k1 = f(y); k2 = f(y + 0.5 * h * k1); k3 = f(y + 0.5 * h * k2); k4 = f(y + h * k3)
        y = y + (h / 6) * (k1 + 2 * k2 + 2 * k3 + k4)
    with kura.Kuramoto(rp, cl, lab, k, omega, K, precision=0, val=vl) as hd:
        th = _dev(theta)
        hd.rk4_steps(th, h, steps)
        hd.sync()
        assert np.abs(th.cpu().numpy() - y).max() < 1e-8
        with pytest.raises(Exception):
            hd.potential(th)
        with pytest.raises(Exception):
            hd.direct_rhs(th, torch.empty_like(th))
