"""Seeded synthetic inputs: the generators produce what their recipes state (CPU only)."""
import numpy as np

from paper_2102_07167_gb300 import gen as G


def test_dirichlet_sizes_bounds_and_sum():
    s = G.dirichlet_sizes(0, 1 << 20, 1024, 2, 256, 4096)
    assert s.sum() == 1 << 20 and s.min() >= 256 and s.max() <= 4096
    s2 = G.dirichlet_sizes(0, 65536, 64, 2, 128, 0)
    assert s2.sum() == 65536 and s2.min() >= 128
    assert np.array_equal(s2, G.dirichlet_sizes(0, 65536, 64, 2, 128, 0))      # deterministic
    assert not np.array_equal(s2, G.dirichlet_sizes(1, 65536, 64, 2, 128, 0))  # seed matters


def test_sbm_structure():
    sizes = np.array([50, 80, 120, 30])
    g = G.sbm(3, sizes, [0.9, 0.8, 0.95, 0.7], 0.02)
    n = g.n
    assert n == 280 and g.row_ptr[0] == 0 and g.row_ptr[-1] == g.col.size
    A = np.zeros((n, n), np.uint8)
    for i in range(n):
        c = g.col[g.row_ptr[i]:g.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)            # sorted, no duplicates
        A[i, c] = 1
    assert np.array_equal(A, A.T) and A.diagonal().sum() == 0
    assert np.array_equal(np.bincount(g.label, minlength=4), sizes)
    same = g.label[:, None] == g.label[None, :]
    intra_density = A[same].sum() / (same.sum() - n)
    inter_density = A[~same].sum() / (~same).sum()
    assert 0.8 < intra_density < 0.92 and 0.01 < inter_density < 0.03
    # relabelled: the user numbering does not list communities contiguously
    assert np.any(np.diff(g.label) < 0)


def test_sbm_deterministic_across_calls():
    a = G.sbm(11, [300, 200], 0.6, 0.01)
    b = G.sbm(11, [300, 200], 0.6, 0.01)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)


def test_node_draws():
    x = G.normal(0, 0, 200000)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1) < 0.01
    u = G.uniform(0, 1, 100000, 0, 2 * np.pi)
    assert u.min() >= 0 and u.max() < 2 * np.pi
    c = G.cauchy(0, 0, 100000, 0.0, 0.5, 10.0)
    assert c.min() >= -10 and c.max() <= 10 and abs(np.median(c)) < 0.02
    om, th = G.paper_e2_inputs(5, 2.0)
    np.testing.assert_allclose(om, [-1, 0, 1, 2, 3])
    np.testing.assert_allclose(th, 2 * np.pi * np.arange(1, 6) / 5)
