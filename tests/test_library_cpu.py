"""libkura on the CPU: the library loads and exports every declared symbol,
argument errors come back as status codes, and the host-side block plan
(permutation, dense/sparse classification, correction streams) reconstructs
the permuted adjacency matrix exactly.  No GPU computation here."""
import ctypes as C

import numpy as np
import pytest

from paper_2102_07167_gb300 import gen as G
from paper_2102_07167_gb300 import kura


def test_library_exports_every_declared_symbol():
    L = kura.load()
    names = kura.header_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert kura.kura_version() >= 100


def test_create_without_gpu_reports_cuda_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    g = G.complete(8)
    with pytest.raises(kura.KuraError) as e:
        kura.kura_create(8, g.row_ptr, g.col, g.label, 1, np.zeros(8), 1.0)
    assert e.value.status == kura.KURA_ECUDA


@pytest.mark.parametrize("bad", ["unsorted", "duplicate", "range", "label", "tau", "rowptr"])
def test_invalid_input_is_rejected(bad):
    g = G.sbm(1, [20, 30], 0.8, 0.05)
    row_ptr, col, label, tau = g.row_ptr.copy(), g.col.copy(), g.label.copy(), 0.5
    r = int(np.argmax(np.diff(row_ptr) >= 2))
    b = int(row_ptr[r])
    if bad == "unsorted":
        col[b], col[b + 1] = col[b + 1], col[b]
    elif bad == "duplicate":
        col[b + 1] = col[b]
    elif bad == "range":
        col[b] = g.n
    elif bad == "label":
        label[3] = 2
    elif bad == "tau":
        tau = 1.5
    elif bad == "rowptr":
        row_ptr[5] = row_ptr[6] + 1
    with pytest.raises(kura.KuraError) as e:
        kura.kura_plan_build(g.n, row_ptr, col, label, 2, tau)
    assert e.value.status == kura.KURA_EINVAL
    assert kura.kura_last_error(None)


def _reconstruct_and_check(g, tau):
    n, nc = g.n, g.n_comm
    p = kura.kura_plan_build(n, g.row_ptr, g.col, g.label, nc, tau)
    try:
        perm, off = kura.kura_plan_perm(p, n, nc)
        st = kura.kura_plan_stats(p)
        # permutation: a bijection, stable sort by label
        assert np.array_equal(np.sort(perm), np.arange(n))
        assert np.array_equal(perm, np.argsort(g.label, kind="stable"))
        inv = np.empty(n, np.int64)
        inv[perm] = np.arange(n)
        comm = np.empty(n, np.int64)
        for I in range(nc):
            comm[off[I]:off[I + 1]] = I
        sizes = np.diff(off)
        # independent classification: non-zeros per block of P A P^T (no self loops)
        A = np.zeros((n, n), np.uint8)
        for u in range(n):
            cs = g.col[g.row_ptr[u]:g.row_ptr[u + 1]]
            cs = cs[cs != u]
            A[inv[u], inv[cs]] = 1
        dense = np.zeros((nc, nc), bool)
        n_dense = n_nonempty = 0
        for I in range(nc):
            for J in range(nc):
                nnz = A[off[I]:off[I + 1], off[J]:off[J + 1]].sum()
                if nnz == 0:
                    continue
                n_nonempty += 1
                entries = sizes[I] * (sizes[I] - 1) if I == J else sizes[I] * sizes[J]
                dense[I, J] = (1 - nnz / entries) < tau
                n_dense += int(dense[I, J])
        assert st["dense_blocks"] == n_dense and st["nonempty_blocks"] == n_nonempty
        for I in range(nc):
            assert np.array_equal(kura.kura_plan_dense_blocks(p, I), np.nonzero(dense[I])[0])
        # streams reconstruct every row exactly
        tot_m = tot_p = 0
        for v in range(n):
            miss, pres = kura.kura_plan_row(p, v, n)
            I = comm[v]
            row = np.zeros(n, np.uint8)
            for J in np.nonzero(dense[I])[0]:
                row[off[J]:off[J + 1]] = 1
            if dense[I, I]:
                row[v] = 0           # diagonal: don't-care, never stored
            assert np.all(row[miss] == 1), "missing entry outside a dense block"
            row[miss] = 0
            assert np.all(row[pres] == 0), "present entry inside a dense block"
            row[pres] = 1
            assert np.array_equal(row, A[v]), f"row {v} differs"
            assert np.all(np.diff(miss) > 0) and np.all(np.diff(pres) > 0)
            assert not dense[I][comm[pres]].any()
            tot_m += miss.size
            tot_p += pres.size
        assert st["missing_entries"] == tot_m and st["sparse_entries"] == tot_p
        return st
    finally:
        kura.kura_plan_destroy(p)


@pytest.mark.parametrize("seed", range(6))
def test_plan_reconstructs_random_graphs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 70))
    nc = int(rng.integers(1, 6))
    A = (rng.random((n, n)) < rng.uniform(0.05, 0.95)).astype(np.uint8)
    lab = rng.integers(0, nc, n).astype(np.int32)
    if seed % 2:
        np.fill_diagonal(A, 1)           # self-loops must be dropped
    g = G.from_dense(A, lab, nc)
    for tau in (0.0, 0.25, 0.5, 0.75, 1.0):
        _reconstruct_and_check(g, tau)


def test_plan_reconstructs_sbm_and_extremes():
    g = G.sbm(4, [40, 25, 60, 13], [0.9, 0.6, 0.95, 0.3], 0.04)
    st = _reconstruct_and_check(g, 0.5)
    assert st["dense_blocks"] == 3          # the p_in = 0.3 community stays sparse
    st0 = _reconstruct_and_check(g, 0.0)
    assert st0["dense_blocks"] == 0 and st0["missing_entries"] == 0 and st0["sparse_entries"] == g.nnz
    st1 = _reconstruct_and_check(g, 1.0)
    assert st1["sparse_blocks"] == 0 and st1["sparse_entries"] == 0


def test_plan_complete_graph_needs_no_corrections():
    g = G.complete(300)
    p = kura.kura_plan_build(g.n, g.row_ptr, g.col, g.label, 1, 0.5)
    st = kura.kura_plan_stats(p)
    kura.kura_plan_destroy(p)
    assert st["dense_blocks"] == 1 and st["missing_entries"] == 0 and st["sparse_entries"] == 0


def test_plan_empty_communities_and_isolated_nodes():
    A = np.zeros((6, 6), np.uint8)
    A[0, 1] = A[1, 0] = 1
    g = G.from_dense(A, np.array([0, 0, 2, 2, 4, 4], np.int32), 5)
    _reconstruct_and_check(g, 0.5)
