"""The N > 1 path of bench.py on CPU: two gloo ranks run bench.timed_replicas (the replica protocol of the GPU
run: warm-up, barriers, exactly K timed steps, max over ranks) with a host stand-in for the device step, and
bench.core_line turns the ranks' times into the JSON line's fields.  Each rank also builds the host-only block
plan of its replica (kura_plan_build, no GPU) and the ranks check that they hold identical plans: a single graph
does not shard on this path, every rank integrates a full replica.  A batch of independent trajectories
does shard: bench.shard_trajectories splits it by LPT on kura_batch_costs with no collective, and
bench.timed_shards times the shares (host stand-ins for the device steps)."""
import os
import socket
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2102_07167_gb300 import gen as G
    from paper_2102_07167_gb300 import kura
    w = G.workload_sbm_small(n=3000, n_comm=6, min_size=128, seed=2)
    g = w.graph
    p = kura.kura_plan_build(g.n, g.row_ptr, g.col, g.label, g.n_comm)
    st = kura.kura_plan_stats(p)
    kura.kura_plan_destroy(p)
    mine = torch.tensor([st["missing_entries"], st["sparse_entries"], st["dense_blocks"], st["tiles"]],
                        dtype=torch.int64)
    all_st = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(all_st, mine)
    steps_run = []

    def run_steps(k):                              # the host stand-in for k RK4 steps; rank 1 is slower
        steps_run.append(k)
        time.sleep(k * (0.004 + 0.004 * rank))

    value, el_max = bench.timed_replicas(run_steps, g.n, 10, 2, dist.barrier, bench.WallTimer(), dist, "cpu")
    line = bench.core_line(value, dist.get_world_size(), 10, 2, el_max, "f64", {"workload": w.name})
    out[rank] = (value, el_max, line, [t.tolist() for t in all_st], steps_run)
    dist.destroy_process_group()


def test_replicas_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert set(out.keys()) == {0, 1}
    v0, el0, line0, st0, steps0 = out[0]
    v1, el1, line1, st1, steps1 = out[1]
    # identical replicas: every rank planned the same graph
    assert st0 == st1 and st0[0] == st0[1]
    # warm-up of max(W, 3) steps, then exactly K timed steps on every rank
    assert steps0 == [3, 10] and steps1 == [3, 10]
    # the slowest rank's time, agreed on by both ranks; rank 1 sleeps 8 ms per step
    assert el0 == el1 and el0 >= 80.0
    n = 3000
    assert abs(v0 - world * n * 10 / (el0 / 1e3)) < 1e-6 * v0 and v0 == v1
    assert line0["n_gpus"] == 2 and line0["value"] == v0 and line0["scaling"] == "weak"
    assert line0["config"]["parallelism"] == "replicas"
    assert abs(line0["ms_per_step"] - el0 / 10) < 1e-12


def test_single_rank_line_fields():
    import bench
    line = bench.core_line(5.0e8, 1, 300, 1, 600.0, "f32+f64", {"workload": "x"})
    assert line["warmup"] == 3 and line["ms_per_step"] == 2.0 and line["config"]["parallelism"] == "single-gpu"
    assert line["higher_is_better"] is True and np.isclose(line["value"], 5.0e8)


def _shard_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2102_07167_gb300 import gen as G
    from paper_2102_07167_gb300 import kura
    ens = G.workload_batch(n_traj=40, n_max=2000, seed=5)
    graphs = G.batch_graphs(ens)
    o = kura.kura_default_opts()
    o.precision = kura.PREC_MIXED
    mine, part, load = bench.shard_trajectories(graphs, world, rank, o)
    # the costs of this rank's share, planned on their own, are the ones the split used
    own_cost = kura.kura_batch_costs([graphs[int(t)] for t in mine], o)
    n_local = int(sum(ens[int(t)][1] for t in mine))
    steps_run = []

    def run_steps(k):                              # host stand-in: time proportional to the share's cost
        steps_run.append(k)
        time.sleep(k * float(own_cost.sum()) * 2e-8)

    value, el_max, n_all = bench.timed_shards(run_steps, n_local, 10, 2, dist.barrier, bench.WallTimer(), dist,
                                              "cpu")
    parts = [torch.zeros(len(ens), dtype=torch.int32) for _ in range(world)]
    dist.all_gather(parts, torch.from_numpy(part))
    out[rank] = (mine.tolist(), load.tolist(), own_cost.tolist(), n_local, value, el_max, n_all,
                 [p.tolist() for p in parts], steps_run)
    dist.destroy_process_group()


def test_batch_shards_two_gloo_ranks():
    """Batched trajectories shard across ranks by LPT with no data-path collective: both ranks compute the
    same partition on their own, their shares are disjoint and cover the batch, and the line's value is
    the whole batch's oscillator-steps over the slowest rank's time."""
    from paper_2102_07167_gb300 import gen as G
    from paper_2102_07167_gb300 import kura
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_shard_worker, args=(world, port, out), nprocs=world, join=True)
    ens = G.workload_batch(n_traj=40, n_max=2000, seed=5)
    o = kura.kura_default_opts()
    o.precision = kura.PREC_MIXED
    cost = kura.kura_batch_costs(G.batch_graphs(ens), o)
    r0, r1 = out[0], out[1]
    # identical partitions, computed independently on each rank
    assert r0[7][0] == r0[7][1] == r1[7][0] == r1[7][1]
    part = np.array(r0[7][0])
    # disjoint shares covering every trajectory, each the rank's part
    assert sorted(r0[0] + r1[0]) == list(range(len(ens)))
    assert all(part[t] == 0 for t in r0[0]) and all(part[t] == 1 for t in r1[0])
    # each share's costs, planned alone, are the batch's; the loads are their sums
    assert np.allclose(r0[2], cost[r0[0]]) and np.allclose(r1[2], cost[r1[0]])
    assert np.allclose(r0[1], [cost[r0[0]].sum(), cost[r1[0]].sum()]) and r0[1] == r1[1]
    assert max(r0[1]) <= cost.sum() / world + cost.max()
    # the timing protocol: warm-up, exactly K timed steps, the slowest rank's time and all oscillators
    assert r0[8] == [3, 10] and r1[8] == [3, 10]
    n_total = sum(n for (_, n, _, _, _) in ens)
    assert r0[3] + r1[3] == n_total and r0[6] == r1[6] == n_total
    assert r0[5] == r1[5] and abs(r0[4] - n_total * 10 / (r0[5] / 1e3)) < 1e-6 * r0[4]


def test_single_rank_shard_aggregate():
    """One rank, no process group: the whole batch's oscillator-steps over that rank's time."""
    import bench
    value, el, n_all = bench.aggregate_shards(10.0, 1000, 5)
    assert n_all == 1000 and el == 10.0 and abs(value - 1000 * 5 / 0.010) < 1e-9
