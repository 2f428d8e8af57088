"""Sharding a batch of independent trajectories across GPUs (host only, no GPU): kura_batch_costs gives the
work-queue cost of each trajectory, kura_partition_lpt splits them by the longest-processing-time rule.

Pins that do not come from the implementation:
- Graham's bound for LPT, max load <= (4/3 - 1/(3m)) OPT, against the optimum found by brute force over
  every assignment of small random instances;
- Graham's tight instance (costs 5,5,4,4,3,3,3 on three parts), whose LPT schedule is worked out by hand;
- the cost of a trajectory is 24 n plus its listed corrections, which an independent host plan counts."""
import itertools

import numpy as np
import pytest

from paper_2102_07167_gb300 import gen as G
from paper_2102_07167_gb300 import kura


def _brute_force_opt(cost, m):
    n = len(cost)
    assign = np.array(list(itertools.product(range(m), repeat=n)), dtype=np.int64)     # m^n x n
    loads = (assign[:, :, None] == np.arange(m)[None, None, :]).astype(np.float64)
    loads = np.einsum("ain,i->an", loads, np.asarray(cost, dtype=np.float64))
    return loads.max(axis=1).min()


def test_lpt_graham_tight_instance_by_hand():
    # decreasing order 5,5,4,4,3,3,3: 5->0, 5->1, 4->2, 4->2 (load 4 < 5), 3->0, 3->1, then all parts hold 8
    # and the last 3 goes to part 0; the optimum 9 is (5,4), (5,4), (3,3,3)
    part, load = kura.kura_partition_lpt([5, 5, 4, 4, 3, 3, 3], 3)
    assert part.tolist() == [0, 1, 2, 2, 0, 1, 0]
    assert load.tolist() == [11.0, 8.0, 8.0]
    assert _brute_force_opt([5, 5, 4, 4, 3, 3, 3], 3) == 9.0
    assert load.max() <= (4 / 3 - 1 / 9) * 9 + 1e-12          # the bound is attained


@pytest.mark.parametrize("m", [2, 3])
def test_lpt_within_graham_bound_of_brute_force_optimum(m):
    rng = np.random.default_rng(10 + m)
    for trial in range(25):
        n = int(rng.integers(1, 9))
        cost = rng.integers(1, 40, size=n).astype(np.float64)
        part, load = kura.kura_partition_lpt(cost, m)
        assert part.shape == (n,) and ((part >= 0) & (part < m)).all()
        # loads are the sums of the assigned costs, every item counted once
        assert np.allclose(load, [cost[part == q].sum() for q in range(m)])
        opt = _brute_force_opt(cost, m)
        assert opt - 1e-9 <= load.max() <= (4 / 3 - 1 / (3 * m)) * opt + 1e-9
        assert load.max() <= cost.sum() / m + cost.max() + 1e-9


def test_lpt_ties_and_edge_cases():
    # equal costs: lower index first, and on equal loads the lower part
    part, load = kura.kura_partition_lpt([1.0] * 5, 2)
    assert part.tolist() == [0, 1, 0, 1, 0] and load.tolist() == [3.0, 2.0]
    # more parts than items: one item per part, the rest empty
    part, load = kura.kura_partition_lpt([2.0, 7.0], 4)
    assert part.tolist() == [1, 0] and load.tolist() == [7.0, 2.0, 0.0, 0.0]
    # one part takes everything; no items gives empty loads
    part, load = kura.kura_partition_lpt([3.0, 1.0, 2.0], 1)
    assert part.tolist() == [0, 0, 0] and load.tolist() == [6.0]
    part, load = kura.kura_partition_lpt([], 3)
    assert part.size == 0 and load.tolist() == [0.0, 0.0, 0.0]
    # zero costs are allowed: the 5 goes first, to part 0; both zeros then go to the empty part 1
    part, load = kura.kura_partition_lpt([0.0, 0.0, 5.0], 2)
    assert part.tolist() == [1, 1, 0] and load.tolist() == [5.0, 0.0]


def test_lpt_is_deterministic():
    cost = np.random.default_rng(3).exponential(size=500)
    a, la = kura.kura_partition_lpt(cost, 8)
    b, lb = kura.kura_partition_lpt(cost.copy(), 8)
    assert (a == b).all() and (la == lb).all()
    assert la.max() <= cost.sum() / 8 + cost.max()


@pytest.mark.parametrize("bad", [[1.0, -1.0], [1.0, float("nan")], [float("inf")]])
def test_lpt_rejects_bad_costs(bad):
    with pytest.raises(kura.KuraError):
        kura.kura_partition_lpt(bad, 2)


def test_lpt_rejects_no_parts():
    with pytest.raises(kura.KuraError):
        kura.kura_partition_lpt([1.0], 0)


def test_batch_costs_count_nodes_and_listed_corrections():
    ens = G.workload_batch(n_traj=12, n_max=3000, seed=4)
    graphs = G.batch_graphs(ens)
    cost = kura.kura_batch_costs(graphs)                   # FP64 defaults: index lists, tau 0.5
    for (g, n, om, th, K), c in zip(ens, cost):
        if g is None:
            assert c == 24.0 * n                           # complete graph: nothing stored
            continue
        p = kura.kura_plan_build(g.n, g.row_ptr, g.col, g.label, g.n_comm, tau=0.5, tensor_cores=0)
        st = kura.kura_plan_stats(p)
        kura.kura_plan_destroy(p)
        assert c == 24.0 * n + st["missing_entries"] + st["sparse_entries"]
    # the tensor-core mask product (mixed only) adds its operand-block term to the SBMs only
    o = kura.kura_default_opts()
    o.precision, o.tensor_cores = kura.PREC_MIXED, 2
    tc = kura.kura_batch_costs(graphs, o)
    for (g, n, om, th, K), c0, c2 in zip(ens, cost, tc):
        assert (c2 == c0) if g is None else (c2 > 24.0 * n)


def test_batch_costs_reject_what_batch_create_rejects():
    big = (None, None, None, 1, np.zeros(20000), 1.0)         # above the mixed per-trajectory maximum
    o = kura.kura_default_opts()
    o.precision = kura.PREC_MIXED
    with pytest.raises(kura.KuraError, match="trajectory 0"):
        kura.kura_batch_costs([big], o)
    empty = (np.zeros(3, np.int64), np.zeros(0, np.int32), np.zeros(2, np.int32), 0, np.zeros(2), 1.0)
    with pytest.raises(kura.KuraError, match="trajectory 1"):      # n_comm = 0
        kura.kura_batch_costs([(None, None, None, 1, np.zeros(10), 1.0), empty], o)
