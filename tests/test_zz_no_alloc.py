"""kura_order_params_static: order parameters for callers that must not allocate device memory
(plug-ins inside an application that owns a fixed device-memory budget, code that runs while a stream
capture is open, real-time loops).  The entry point keeps its scratch in a static device array of the
library; the caller passes only its own inputs and outputs.  Checked against the handle-based
kura_order_params on the same phases, twice in a row (the scratch must come back zeroed)."""
import numpy as np
import pytest

from paper_2102_07167_gb300 import gen as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_static_order_params_match_handle_api_twice():
    from paper_2102_07167_gb300 import kura
    w = G.workload_sbm_small(n=20000, n_comm=24, min_size=128, seed=4)
    g = w.graph
    dev = torch.device("cuda", 0)
    theta = torch.tensor(w.theta0 + 3.0 * G.uniform(8, 2, g.n, -1, 1), device=dev)
    label = torch.tensor(g.label, device=dev, dtype=torch.int32)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K) as k:
        r_ref, psi_ref, rc_ref, pc_ref = k.order_params(theta, per_community=True)
    ref = np.concatenate([[r_ref, psi_ref], np.stack([rc_ref, pc_ref], 1).ravel()])
    free = []
    for call in range(2):
        out = torch.full((2 + 2 * g.n_comm,), -7.0, dtype=torch.float64, device=dev)
        kura.kura_order_params_static(g.n, theta, label, g.n_comm, out)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info(dev)[0])
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12, err_msg=f"call {call}")
    assert free[0] == free[1]          # the second call allocated nothing on the device
    # one community without labels: the global order parameter
    out1 = torch.zeros(4, dtype=torch.float64, device=dev)
    kura.kura_order_params_static(g.n, theta, None, 1, out1)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out1.cpu().numpy()[:2], ref[:2], rtol=0, atol=1e-12)
    np.testing.assert_allclose(out1.cpu().numpy()[2:], ref[:2], rtol=0, atol=1e-12)


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
