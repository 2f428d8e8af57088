"""kura_order_params_static: order parameters for callers that must not allocate device memory
(plug-ins inside an application that owns the whole device-memory budget, real-time loops that may
not block on cudaMalloc/cudaFree).  The entry point keeps its scratch in a static device array of
the library; the caller passes only its own inputs and outputs.

Checked, on two calls in a row (the scratch must come back zeroed), against the handle-based
kura_order_params on the same phases and against the FP64 CPU oracle's eq:OrderParameter, global and
per community; then a call with one label out of range must give NaN everywhere without touching
memory outside the scratch, and the next call must be correct again.  This file is collected last,
so a run that stops at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_2102_07167_gb300 import gen as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12      # both sides are FP64; the library's sums are exact fixed point (2^-41 per term here)


def _case():
    w = G.workload_sbm_small(n=20000, n_comm=24, min_size=128, seed=4)
    theta = w.theta0 + 3.0 * G.uniform(8, 2, w.graph.n, -1, 1)
    return w.graph, w, theta


def _expected_oracle(g, theta):
    import oracle
    r, psi, rc, pc = oracle.order_params(theta, g.label, g.n_comm)
    return np.concatenate([[r, psi], np.stack([rc, pc], 1).ravel()])


def _angle_close(got, ref, tol):
    """Arguments compared modulo 2 pi (atan2 near +-pi)."""
    d = np.abs(np.angle(np.exp(1j * (got - ref))))
    return np.all(d <= tol)


def _check(got, ref, tol, what):
    r_got, r_ref = got[0::2], ref[0::2]
    np.testing.assert_allclose(r_got, r_ref, rtol=0, atol=tol, err_msg=f"{what}: moduli")
    # arguments are well defined where the modulus is not tiny; their error is about the sums' / r
    ok = r_ref > 1e-3
    assert _angle_close(got[1::2][ok], ref[1::2][ok], 1e-9), f"{what}: arguments"


def test_static_order_params_match_handle_api_and_oracle_twice():
    from paper_2102_07167_gb300 import kura
    g, w, theta_h = _case()
    dev = torch.device("cuda", 0)
    theta = torch.tensor(theta_h, device=dev)
    label = torch.tensor(g.label, device=dev, dtype=torch.int32)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K) as k:
        r_ref, psi_ref, rc_ref, pc_ref = k.order_params(theta, per_community=True)
    ref_api = np.concatenate([[r_ref, psi_ref], np.stack([rc_ref, pc_ref], 1).ravel()])
    ref_orc = _expected_oracle(g, theta_h)
    for call in range(2):
        out = torch.full((2 + 2 * g.n_comm,), -7.0, dtype=torch.float64, device=dev)
        kura.kura_order_params_static(g.n, theta, label, g.n_comm, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref_api, rtol=0, atol=TOL, err_msg=f"call {call} vs kura_order_params")
        _check(got, ref_orc, TOL, f"call {call} vs oracle")
    # one community without labels: the global order parameter
    out1 = torch.zeros(4, dtype=torch.float64, device=dev)
    kura.kura_order_params_static(g.n, theta, None, 1, out1)
    torch.cuda.synchronize()
    got1 = out1.cpu().numpy()
    _check(got1[:2], ref_orc[:2], TOL, "no labels, global")
    _check(got1[2:], ref_orc[:2], TOL, "no labels, community 0")


def test_static_order_params_bad_label_gives_nan_then_recovers():
    from paper_2102_07167_gb300 import kura
    g, w, theta_h = _case()
    dev = torch.device("cuda", 0)
    theta = torch.tensor(theta_h, device=dev)
    n_comm = g.n_comm
    for bad_value in (n_comm, -1, 10 ** 6):
        lab = g.label.copy()
        lab[g.n // 2] = bad_value
        label_bad = torch.tensor(lab, device=dev, dtype=torch.int32)
        # a guard row past out's end must stay untouched
        buf = torch.full((2 + 2 * n_comm + 2,), 5.0, dtype=torch.float64, device=dev)
        kura.kura_order_params_static(g.n, theta, label_bad, n_comm, buf[:2 + 2 * n_comm])
        torch.cuda.synchronize()
        got = buf.cpu().numpy()
        assert np.all(np.isnan(got[:2 + 2 * n_comm])), f"label {bad_value}: expected NaN everywhere"
        assert np.all(got[2 + 2 * n_comm:] == 5.0)
        # the scratch is clean again: a correct call right after gives the oracle's values
        label = torch.tensor(g.label, device=dev, dtype=torch.int32)
        out = torch.zeros(2 + 2 * n_comm, dtype=torch.float64, device=dev)
        kura.kura_order_params_static(g.n, theta, label, n_comm, out)
        torch.cuda.synchronize()
        _check(out.cpu().numpy(), _expected_oracle(g, theta_h), TOL, f"after label {bad_value}")


def test_static_order_params_rejects_too_many_communities():
    from paper_2102_07167_gb300 import kura
    dev = torch.device("cuda", 0)
    n = 64
    theta = torch.zeros(n, dtype=torch.float64, device=dev)
    label = torch.zeros(n, dtype=torch.int32, device=dev)
    big = kura.STATIC_MAX_COMM + 1
    out = torch.zeros(2 + 2 * big, dtype=torch.float64, device=dev)
    with pytest.raises(kura.KuraError) as e:
        kura.kura_order_params_static(n, theta, label, big, out)
    assert e.value.status == kura.KURA_EINVAL
