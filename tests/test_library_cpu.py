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


def _reconstruct_and_check(g, tau, bitmap_zmin=-1.0, precision=1, tensor_cores=1):
    n, nc = g.n, g.n_comm
    p = kura.kura_plan_build(n, g.row_ptr, g.col, g.label, nc, tau, precision, bitmap_zmin, tensor_cores)
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
        for zmin, prec, tcm in ((-1.0, 1, 0), (0.0, 1, 0), (-1.0, 0, 0), (-1.0, 1, 1), (-1.0, 0, 2)):
            _reconstruct_and_check(g, tau, zmin, prec, tcm)


def test_plan_reconstructs_sbm_and_extremes():
    g = G.sbm(4, [40, 25, 60, 13], [0.9, 0.6, 0.95, 0.3], 0.04)
    _reconstruct_and_check(g, 0.5, 0.0, tensor_cores=0)
    st2 = _reconstruct_and_check(g, 0.5, tensor_cores=2)
    assert st2["tc_tiles"] >= 3 and st2["tc_rows"] == 40 + 25 + 60      # every dense community on the tensor cores
    st = _reconstruct_and_check(g, 0.5, tensor_cores=0)
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


@pytest.mark.parametrize("tau,p_one", [(0.0, 0.6), (1.0, 0.3)])
def test_plan_splits_long_rows_into_subrows(tau, p_one):
    """Rows with more than 508 stored entries are cut into several sub-rows; the streams still reconstruct
    every row (tau = 0 forces ~720 present entries per row, tau = 1 ~840 missing entries)."""
    rng = np.random.default_rng(7)
    n = 1200
    A = (rng.random((n, n)) < p_one).astype(np.uint8)
    np.fill_diagonal(A, 0)
    g = G.from_dense(A)
    st = _reconstruct_and_check(g, tau, tensor_cores=0)
    _reconstruct_and_check(g, tau, 0.0, tensor_cores=0)
    _reconstruct_and_check(g, tau, tensor_cores=2)
    assert st["max_row_entries"] > 508


def _tc_digits(v):
    """Balanced base-16 digits (16 of them, each in [-8, 7]) of integers v, as the trig kernel writes them."""
    v = np.asarray(v, dtype=np.int64).copy()
    out = np.empty((16,) + v.shape, np.int64)
    for k in range(16):
        d = ((v + 8) & 15) - 8
        out[k] = d
        v = (v - d) >> 4
    assert np.all(v == 0)
    return out


def _emulate_row_kernel(g, tau, omega, theta, K, bitmap_zmin=-1.0, precision=1, tensor_cores=1):
    """Consumes the packed stream exactly as the row kernel does (groups -> sub-row headers -> padded int4
    segments -> window-or-table gathers, padding resolving to zero entries; tensor-core tiles: 128 x 128 mask
    blocks times the base-16 digits of the fixed-point table, summed as exact integers), in float64, and
    returns f in user order."""
    n, nc = g.n, g.n_comm
    p = kura.kura_plan_build(n, g.row_ptr, g.col, g.label, nc, tau, precision, bitmap_zmin, tensor_cores)
    try:
        perm, off = kura.kura_plan_perm(p, n, nc)
        gstream, groups, tiles, row_sub0, bitmap = kura.kura_plan_export(p, n)
        dense = [kura.kura_plan_dense_blocks(p, I) for I in range(nc)]
    finally:
        kura.kura_plan_destroy(p)
    th = theta[perm]
    s_tab = np.append(np.sin(th), [0.0, 0.0])      # entries n, n+1 are the table's zero padding
    c_tab = np.append(np.cos(th), [0.0, 0.0])
    S = np.array([s_tab[off[J]:off[J + 1]].sum() for J in range(nc)])
    C = np.array([c_tab[off[J]:off[J + 1]].sum() for J in range(nc)])
    # fixed point with q = 61 - ceil(log2 n) fraction bits, and its digits per column (padded to 128)
    qb = 61 - int(np.ceil(np.log2(max(n, 2))))
    npad = (n + 127) // 128 * 128
    sf = np.zeros(npad, np.int64)
    cf = np.zeros(npad, np.int64)
    sf[:n] = np.rint(s_tab[:n] * 2.0 ** qb).astype(np.int64)
    cf[:n] = np.rint(c_tab[:n] * 2.0 ** qb).astype(np.int64)
    dsf, dcf = _tc_digits(sf), _tc_digits(cf)
    f = np.empty(n)
    for t in tiles:
        wbeg, wlen = int(t["wbeg"]), int(t["wlen"])

        def gather(idx, missing):
            # the window [wbeg, wbeg + wlen) holds copies of the table entries; padding is n (the table's
            # zero entry) or, for missing parts of tiles whose dense columns all lie in the window, wbeg - 1
            # (the zero entry kept just before the staged window)
            zero = idx == wbeg - 1 if (missing and t["flags"] & 2) else np.zeros(idx.shape, bool)
            assert np.all(((idx >= 0) & (idx <= n)) | zero)
            safe = np.where(zero, n, idx)
            return s_tab[safe], c_tab[safe]
        stash = {}
        for gi in range(t["g0"], t["g1"]):
            G_ = groups[gi]
            base = int(G_["off"])
            for j in range(G_["nsub"]):
                mrel, nm, prel, npr = gstream[base + 4 * j: base + 4 * j + 4]
                m = gstream[base + mrel: base + mrel + 4 * ((nm + 3) // 4)]
                q = gstream[base + prel: base + prel + 4 * ((npr + 3) // 4)]
                ms, mc = gather(m, True)
                ps, pc = gather(q, False)
                stash[int(G_["sub0"]) + j] = (ps.sum() - ms.sum(), pc.sum() - mc.sum())
        for r in range(t["r0"], t["r1"]):
            a_s = sum(stash[s][0] for s in range(row_sub0[r], row_sub0[r + 1]))
            a_c = sum(stash[s][1] for s in range(row_sub0[r], row_sub0[r + 1]))
            if t["flags"] & kura.TILE_BITMAP:
                # lane-major bitmap: bit j of word q of super-word w <-> window column 1024 w + 32 j + q
                nsw = int(t["nsw"])
                words = bitmap[int(t["bm_off"]) + (r - t["r0"]) * nsw * 32: int(t["bm_off"]) + (r - t["r0"] + 1) * nsw * 32]
                k = np.arange(wlen)
                bits = (words[(k >> 10) * 32 + (k & 31)] >> ((k >> 5) & 31).astype(np.uint32)) & 1
                cols = wbeg + k[bits == 1]
                a_s -= s_tab[cols].sum()
                a_c -= c_tab[cols].sum()
            if t["flags"] & kura.TILE_TC:
                # block (kb, m) of 128 x 128 bits; D_k = mask . digit_k, sum_k D_k 16^k in integers
                lr, nM = r - t["r0"], (t["r1"] - t["r0"] + 127) // 128
                ms = mc = 0
                for kb in range(int(t["nsw"])):
                    w = bitmap[int(t["bm_off"]) + ((kb * nM + lr // 128) * 128 + lr % 128) * 4:][:4]
                    c = np.arange(128)
                    bits = ((w[c >> 5] >> (c & 31).astype(np.uint32)) & 1).astype(np.int64)
                    cols = wbeg + 128 * kb + c
                    assert np.all(cols[bits == 1] < n)
                    Ds = dsf[:, cols] @ bits
                    Dc = dcf[:, cols] @ bits
                    assert np.all(np.abs(Ds) < 2 ** 24) and np.all(np.abs(Dc) < 2 ** 24)   # exact in FP32
                    ms += sum(int(Ds[k]) << (4 * k) for k in range(16))
                    mc += sum(int(Dc[k]) << (4 * k) for k in range(16))
                a_s -= ms * 2.0 ** -qb
                a_c -= mc * 2.0 ** -qb
            I = t["comm"]
            Ts, Tc = S[dense[I]].sum(), C[dense[I]].sum()
            f[r] = omega[perm[r]] + (K / n) * (c_tab[r] * (Ts + a_s) - s_tab[r] * (Tc + a_c))
    out = np.empty(n)
    out[perm] = f
    return out


@pytest.mark.parametrize("zmin,prec,tcm", [(-1.0, 1, 0), (0.05, 1, 0), (-1.0, 0, 0), (-1.0, 1, 1), (-1.0, 0, 2)])
@pytest.mark.parametrize("case", ["sbm", "long_rows_sparse", "long_rows_dense", "big_community"])
def test_packed_stream_emulation_matches_oracle(case, zmin, prec, tcm):
    """The packed stream (headers, padding, windows, sub-rows) read the way the row kernel reads it gives
    the right-hand side of the FP64 oracle."""
    import oracle
    rng = np.random.default_rng(11)
    if case == "sbm":
        g, tau = G.sbm(3, [300, 45, 1, 700, 130], [0.9, 0.6, 1.0, 0.75, 0.3], 0.02), 0.5
    elif case == "big_community":
        g, tau = G.sbm(5, [5000, 257], [0.93, 0.8], 0.003), 0.5        # window cap exceeded
    else:
        n = 1100
        A = (rng.random((n, n)) < (0.6 if case == "long_rows_sparse" else 0.3)).astype(np.uint8)
        np.fill_diagonal(A, 0)
        g = G.from_dense(A)
        tau = 0.0 if case == "long_rows_sparse" else 1.0
    omega, theta = rng.normal(size=g.n), rng.uniform(-30, 30, g.n)
    f = _emulate_row_kernel(g, tau, omega, theta, 2.0, zmin, prec, tcm)
    ref = oracle.rhs_csr(g.row_ptr, g.col, omega, theta, 2.0)
    np.testing.assert_allclose(f, ref, rtol=0, atol=1e-10)


@pytest.mark.parametrize("prec", [0, 1])
def test_missing_entries_are_bank_balanced(prec):
    """Each warp-wide gather of missing entries (positions 128 i + 4 l + t, l = 0..31) touches every shared
    memory bank group about equally: on average at most 2.5 (of 32) entries per group of 128 / entry-size
    bytes (the ideal is 32 / groups = 2 or 4); only a row's tail can be lopsided."""
    g = G.sbm(2, [900, 700, 1200], [0.6, 0.7, 0.8], 0.01)
    p = kura.kura_plan_build(g.n, g.row_ptr, g.col, g.label, g.n_comm, 0.5, prec, tensor_cores=0)
    try:
        gstream, groups, tiles, row_sub0, _ = kura.kura_plan_export(p, g.n)
    finally:
        kura.kura_plan_destroy(p)
    K = 16 if prec == 1 else 8
    maxima = []
    for t in tiles:
        for gi in range(t["g0"], t["g1"]):
            G_ = groups[gi]
            base = int(G_["off"])
            for j in range(G_["nsub"]):
                mrel, nm = gstream[base + 4 * j], gstream[base + 4 * j + 1]
                seg = gstream[base + mrel: base + mrel + nm]
                for i in range(0, (nm + 127) // 128):
                    for tt in range(4):
                        pos = [128 * i + 4 * l + tt for l in range(32) if 128 * i + 4 * l + tt < nm]
                        if len(pos) < 32:
                            continue
                        keys = (seg[pos] - t["wbeg"]) % K
                        maxima.append(np.bincount(keys, minlength=K).max())
    ideal = 32 // K
    maxima = np.array(maxima)
    assert maxima.size > 100 and maxima.mean() <= ideal + 0.5 and np.percentile(maxima, 99) <= ideal + 3, \
        (maxima.size, maxima.mean(), np.percentile(maxima, 99))


def test_gather_rate_probe_rejects_bad_sizes():
    """Argument checks of the roofline probe run before any CUDA call."""
    import ctypes as C
    L = kura.load()
    r = C.c_double()
    for args in ((0, 1 << 20, 8), (1 << 20, 100, 8), (1 << 20, 1 << 20, 12), (1 << 31, 1 << 20, 8)):
        assert L.kura_measure_gather_rate(*args, None, C.byref(r)) == kura.KURA_EINVAL
    assert L.kura_measure_gather_rate(1 << 20, 1 << 20, 8, None, None) == kura.KURA_EINVAL


def test_probes_and_batch_queries_reject_bad_arguments():
    """Argument checks of the L2-bandwidth and launch-floor probes and of the batch queries run before any
    CUDA call."""
    import ctypes as C
    L = kura.load()
    r = C.c_double()
    for nbytes in (0, (1 << 20) - 1, (1 << 30) + 1):
        assert L.kura_measure_l2_bandwidth(nbytes, None, C.byref(r)) == kura.KURA_EINVAL
    assert L.kura_measure_l2_bandwidth(1 << 24, None, None) == kura.KURA_EINVAL
    for k, reps in ((0, 10), (4097, 10), (8, 0), (8, 100001)):
        assert L.kura_measure_graph_launch_floor(k, reps, None, C.byref(r)) == kura.KURA_EINVAL
    info = kura.KuraBatchInfo()
    assert L.kura_batch_info(None, C.byref(info)) == kura.KURA_EINVAL
    assert L.kura_batch_traj_params(None, 0, None, None, None) == kura.KURA_EINVAL


def test_batch_create_rejects_bad_options_without_a_gpu():
    """Option checks of kura_batch_create come before the device is touched."""
    import ctypes as C
    g = G.complete(8)
    o = kura.kura_default_opts()
    o.precision = kura.PREC_MIXED
    o.row_lanes = 12
    with pytest.raises(kura.KuraError) as e:
        kura.kura_batch_create([(None, None, None, 1, np.zeros(8), 1.0)], o)
    assert e.value.status == kura.KURA_EINVAL
    o.row_lanes, o.tau = 0, 1.5
    with pytest.raises(kura.KuraError) as e:
        kura.kura_batch_create([(None, None, None, 1, np.zeros(8), 1.0)], o)
    assert e.value.status == kura.KURA_EINVAL


# ----------------------------------------------------------------------------- finite-valued matrices
def _valued_case(seed, sizes=(40, 70, 25, 130), max_val=3, noise=0.25):
    rng = np.random.default_rng(seed)
    k = len(sizes)
    V = rng.integers(0, max_val + 1, (k, k))
    lab = np.repeat(np.arange(k), sizes)
    A = V[lab][:, lab].astype(np.int32)
    flip = rng.random(A.shape) < noise
    A[flip] = rng.integers(0, max_val + 1, int(flip.sum()))
    np.fill_diagonal(A, 0)
    perm = rng.permutation(A.shape[0])
    A, lab = A[perm][:, perm], lab[perm].astype(np.int32)
    rows, cols = np.nonzero(A)
    rp = np.zeros(A.shape[0] + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    return A, np.cumsum(rp), cols.astype(np.int32), A[rows, cols].astype(np.int32), lab, k


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("prec", [0, 1])
def test_valued_plan_stream_emulation_matches_oracle(seed, prec):
    """A finite-valued plan (Sec. 1, Generalisations) read the way the row kernel reads it: block values times
    the block sums, plus every packed (column, weight) entry times its (sin, cos); equals the oracle's
    definition, and the dense-block values are the oracle block rule's."""
    import oracle
    A, rp, cl, vl, lab, k = _valued_case(seed)
    n = A.shape[0]
    rng = np.random.default_rng(100 + seed)
    omega, theta, K = rng.normal(size=n), rng.uniform(-20, 20, n), 1.3
    p = kura.kura_plan_build_valued(n, rp, cl, vl, lab, k, 0.5, prec)
    try:
        perm, off = kura.kura_plan_perm(p, n, k)
        gstream, groups, tiles, row_sub0, _ = kura.kura_plan_export(p, n)
        dense = [kura.kura_plan_dense_blocks(p, I) for I in range(k)]
        dvals = [kura.kura_plan_dense_values(p, I) for I in range(k)]
    finally:
        kura.kura_plan_destroy(p)
    _, bv = oracle.rhs_block_valued(rp, cl, vl, 3, lab, k, omega, theta, K)
    for I in range(k):
        expect = np.nonzero(bv[I])[0]
        assert np.array_equal(dense[I], expect) and np.array_equal(dvals[I], bv[I][expect])
    th = theta[perm]
    s_tab, c_tab = np.append(np.sin(th), [0, 0]), np.append(np.cos(th), [0, 0])
    S = np.array([s_tab[off[J]:off[J + 1]].sum() for J in range(k)])
    C = np.array([c_tab[off[J]:off[J + 1]].sum() for J in range(k)])
    f = np.empty(n)
    for t in tiles:
        assert t["flags"] & kura.TILE_VALUED
        stash = {}
        for gi in range(t["g0"], t["g1"]):
            G_ = groups[gi]
            base = int(G_["off"])
            for j in range(G_["nsub"]):
                mrel, nm, prel, npr = gstream[base + 4 * j: base + 4 * j + 4]
                seg = np.concatenate([gstream[base + mrel: base + mrel + 4 * ((nm + 3) // 4)],
                                      gstream[base + prel: base + prel + 4 * ((npr + 3) // 4)]]).astype(np.uint32)
                col, w = (seg & 0xFFFFFF).astype(np.int64), (seg >> 24).astype(np.int64) - 128
                assert np.all(col <= n)
                stash[int(G_["sub0"]) + j] = ((w * s_tab[col]).sum(), (w * c_tab[col]).sum())
        for r in range(t["r0"], t["r1"]):
            a_s = sum(stash[s][0] for s in range(row_sub0[r], row_sub0[r + 1]))
            a_c = sum(stash[s][1] for s in range(row_sub0[r], row_sub0[r + 1]))
            I = t["comm"]
            Ts = sum(v * S[J] for J, v in zip(dense[I], dvals[I]))
            Tc = sum(v * C[J] for J, v in zip(dense[I], dvals[I]))
            f[r] = omega[perm[r]] + (K / n) * (c_tab[r] * (Ts + a_s) - s_tab[r] * (Tc + a_c))
    out = np.empty(n)
    out[perm] = f
    np.testing.assert_allclose(out, oracle.rhs_valued_csr(rp, cl, vl, omega, theta, K), atol=1e-11, rtol=0)


def test_valued_plan_rejects_bad_values():
    A, rp, cl, vl, lab, k = _valued_case(0)
    for bad in (0, 128):
        vb = vl.copy()
        vb[3] = bad
        with pytest.raises(Exception):
            kura.kura_plan_build_valued(A.shape[0], rp, cl, vb, lab, k)


# ----------------------------------------------------------------------------- digit and rounding identities
# The trig/block-sum kernel forms the tensor-core digit image and the mixed-precision fixed point with two
# shortcuts. These tests pin the arithmetic of both, in integer and float32 numpy, against the plain
# definitions.

def _balanced_digits_sequential(v):
    """Balanced base-16 digits in [-8, 7] by the definition: d = ((v + 8) mod 16) - 8, v <- (v - d) / 16."""
    out = []
    for _ in range(16):
        d = ((v + 8) & 15) - 8
        out.append(d)
        v = (v - d) >> 4
    return out


def _balanced_digits_bias(v):
    """The kernel's form: nibble k of (v + 0x8888888888888888) mod 2^64, minus 8."""
    u = (v + 0x8888888888888888) & 0xFFFFFFFFFFFFFFFF
    return [((u >> (4 * k)) & 15) - 8 for k in range(16)]


def test_balanced_digits_by_bias_equal_sequential_and_sum_back():
    rng = np.random.default_rng(11)
    vals = [0, 1, -1, 7, 8, -8, -9, 2**41, -2**41, 2**62, -2**63, 2**63 - 1]
    vals += [int(x) for x in rng.integers(-2**62, 2**62, 2000)]
    vals += [int(x) for x in rng.integers(-2**42, 2**42, 2000)]
    for v in vals:
        d = _balanced_digits_bias(v)
        assert d == _balanced_digits_sequential(v), v
        assert all(-8 <= x <= 7 for x in d)
        assert sum(x * 16**k for k, x in enumerate(d)) % 2**64 == v % 2**64


def _f32_to_ll_rn_split(x):
    """The kernel's 64-bit rounding with FP32 operations only: xi = rint(x); hi = floor(xi 2^-24);
    lo = fma(-hi, 2^24, xi) (exact: an integer in [0, 2^24)); result hi 2^24 + lo."""
    x = np.float32(x)
    xi = np.rint(x)                                   # round half to even, float32
    hi = np.floor(np.float32(xi * np.float32(2.0**-24)))
    lo = np.float32(np.float64(xi) - np.float64(hi) * 2.0**24)   # the exact fma result, representable
    assert float(lo) == float(np.float64(xi) - np.float64(hi) * 2.0**24)
    assert 0.0 <= float(lo) < 2.0**24
    return int(hi) * 2**24 + int(lo)


def test_fp32_split_rounding_equals_round_half_even():
    rng = np.random.default_rng(12)
    q = 41
    s = rng.uniform(-1, 1, 20000).astype(np.float32)
    s = np.concatenate([s, np.float32([0.0, -0.0, 1.0, -1.0, 2.0**-30, -2.0**-30, 2.0**-41, 1.5 * 2.0**-41,
                                       2.5 * 2.0**-41, -2.5 * 2.0**-41, 0.5 * 2.0**-41])])
    for v in s:
        x = np.float32(v * np.float32(2.0**q))        # the kernel's FP32 product
        want = int(np.rint(np.float64(x)))           # round half to even of the same float32 value
        assert _f32_to_ll_rn_split(x) == want, v


def test_fixed_point_turn_constants_match_pi():
    """The mixed-mode phase reduction multiplies by round(2^64 / (2 pi)) and scales by 2 pi 2^-32 and
    2 pi 2^-64 in FP32: the constants in the kernel source against a 60-digit pi."""
    import os
    import re
    sp = pytest.importorskip("sympy")
    src = open(os.path.join(os.path.dirname(kura.__file__), "csrc", "kura_kernels.cuh")).read()
    q64 = int(re.search(r"#define KURA_TURN_Q64 (0x[0-9A-Fa-f]+)ull", src).group(1), 16)
    assert q64 == int(sp.floor(sp.Integer(2) ** 63 / sp.pi + sp.Rational(1, 2)))
    for name, e in (("KURA_TWO_PI_2M32", -32), ("KURA_TWO_PI_2M64", -64)):
        v = float(re.search(rf"#define {name} ([0-9.e+-]+)f", src).group(1))
        assert np.float32(v) == np.float32(float(sp.N(2 * sp.pi * sp.Integer(2) ** e, 40)))
