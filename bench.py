"""Benchmark: RK4 oscillator-steps/s of the localised-order-parameter block path.

Default workload: the 2^20-node SBM (1024 communities, Dirichlet sizes in
[256, 4096], p_in ~ U[0.5, 0.99], p_out = 1e-4, omega ~ Cauchy(0, 0.5)
clipped at +-10, K = 3, h = 0.01), mixed precision (FP32 sin/cos and
per-edge corrections, exact fixed-point block sums, FP64 epilogue and state).
One "step" is one classical RK4 step over the whole graph (4 right-hand-side
evaluations).  Inputs are resident in HBM; the 1.85 GB correction stream of
every stage is larger than the 126 MiB L2, so no L2 flush is needed.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(the reference implementation of the method for this build) on the host
cores on a bounded sample of the same workload.

Multi-GPU: a single graph does not shard on this path (no exchange step is
cheaper than the stage itself), so N > 1 runs N independent replicas
("weak" scaling); value = total oscillator-steps of all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RK4 oscillator-steps/s (N*steps/s) vs GPU direct sum at stated FP64/FP32 error"
UNIT = "oscillator-steps/s"
FALLBACK_HBM_GBS = 6800.0


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate_replicas(el_ms_local: float, n: int, steps: int, dist=None, device=None):
    """Replica runs: every rank integrates its own copy of the workload.  Returns (value, max elapsed ms):
    value = total oscillator-steps of all ranks / the slowest rank's time."""
    import torch
    world = 1
    el = float(el_ms_local)
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        t = torch.tensor([el], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el = float(t.item())
    return world * n * steps / (el / 1e3), el


# kernels per RK4 step of the CUDA-graph step loop: four row kernels, and one trig/block-sum launch per
# 8-step graph (the fused trig makes every other stage's table inside the row kernel)
LAUNCHES_PER_STEP = 4 + 1 / 8


def aggregate_shards(el_ms_local: float, n_local: int, steps: int, dist=None, device=None):
    """Shard runs: every rank integrates its own share of one batch.  Returns (value, max elapsed ms, total
    oscillators): value = oscillator-steps of all ranks' shares / the slowest rank's time."""
    import torch
    el, n = float(el_ms_local), int(n_local)
    if dist is not None and dist.is_initialized():
        t = torch.tensor([el], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        c = torch.tensor([n], dtype=torch.int64, device=device)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        el, n = float(t.item()), int(c.item())
    return n * steps / (el / 1e3), el, n


def timed_shards(run_steps, n_local: int, steps: int, warmup: int, barrier, timer, dist=None, device=None):
    """The shard protocol: as timed_replicas, but each rank integrates a different share of the work."""
    run_steps(max(warmup, 3))
    barrier()
    barrier()
    t0 = timer.mark()
    run_steps(steps)
    t1 = timer.mark()
    barrier()
    return aggregate_shards(timer.ms(t0, t1), n_local, steps, dist, device)


def shard_trajectories(graphs, world: int, rank: int, opts=None):
    """This rank's trajectories of a batch split over `world` GPUs by the longest-processing-time rule on the
    work-queue costs (kura_batch_costs, kura_partition_lpt).  Every rank computes the same partition from
    the same graphs, so the split needs no communication.  Returns (indices of this rank's trajectories,
    part of every trajectory, cost load of every part)."""
    from paper_2102_07167_gb300 import kura
    cost = kura.kura_batch_costs(graphs, opts)
    part, load = kura.kura_partition_lpt(cost, world)
    return np.flatnonzero(part == rank), part, load


class EventTimer:
    """Marks on the current CUDA stream (CUDA events)."""

    def mark(self):
        import torch
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        return e

    def ms(self, a, b):
        return a.elapsed_time(b)


class WallTimer:
    """Host wall-clock marks (for replicas whose step runs on the host)."""

    def mark(self):
        return time.perf_counter()

    def ms(self, a, b):
        return (b - a) * 1e3


def timed_replicas(run_steps, n: int, steps: int, warmup: int, barrier, timer, dist=None, device=None):
    """The replica protocol of the N-GPU run: max(warmup, 3) untimed steps, then exactly `steps` steps between
    barriers, timed on each rank; returns (value, slowest rank's ms) from aggregate_replicas."""
    run_steps(max(warmup, 3))
    barrier()
    barrier()
    t0 = timer.mark()
    run_steps(steps)
    t1 = timer.mark()
    barrier()
    return aggregate_replicas(timer.ms(t0, t1), n, steps, dist, device)


def core_line(value: float, world: int, steps: int, warmup: int, el_ms: float, dtype: str, config: dict) -> dict:
    """The fields of the JSON line that follow from the replicas' times."""
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": max(warmup, 3), "ms_per_step": el_ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": dict(config, parallelism="replicas" if world > 1 else "single-gpu")}


def _workload(name: str):
    from paper_2102_07167_gb300 import gen as G
    if name == "sbm-2p20":
        return G.workload_sbm_large()
    if name == "sbm-2p18":     # same recipe at a quarter of the nodes and communities (profiling size)
        return G.workload_sbm_large(n=1 << 18, n_comm=256)
    if name == "sbm-2p19":     # half the nodes and communities, p_out doubled: rows keep ~105 sparse entries
        return G.workload_sbm_large(n=1 << 19, n_comm=512, p_out=2e-4)
    if name == "sbm-65536":
        return G.workload_sbm_small()
    if name == "complete-512":
        return G.workload_complete(512)
    raise SystemExit(f"unknown workload {name}")


def _workload_desc(w, st):
    g = w.graph
    return {"workload": f"{w.name}: SBM N={g.n}, {g.n_comm} communities" if g.n_comm > 1 else
            f"{w.name}: complete graph N={g.n}",
            "n": g.n, "edges": g.nnz, "communities": g.n_comm, "K": w.K, "h": w.h,
            "dense_blocks": st["dense_blocks"], "missing_entries": st["missing_entries"],
            "sparse_entries": st["sparse_entries"],
            "l2": "inputs larger than L2 (correction stream %.2f GB per stage vs 126 MiB L2)" %
                  (st["stream_bytes"] / 1e9)}


def cpu_baseline_oracle(w, seconds: float = 12.0, keep_values: bool = False):
    """The FP64 oracle as it stands (CSR definition, one sine per edge, one core) on a bounded sample of
    rows of the same graph; 4 right-hand-side evaluations per RK4 step.  With keep_values the sampled rows
    and the oracle's values there are returned too (keys "_rows", "_ref"), so that the GPU's right-hand
    side at the same phases can be compared with them."""
    import oracle
    from paper_2102_07167_gb300 import gen as G
    g = w.graph
    order = G.permutation(123, g.n).astype(np.int64)
    done, t0, pos, batch = 0, time.perf_counter(), 0, 2048
    vals = []
    while time.perf_counter() - t0 < seconds and pos < g.n:
        rows = order[pos:pos + batch]
        v = oracle.rhs_csr(g.row_ptr, g.col, w.omega, w.theta0, w.K, rows=rows)
        if keep_values:
            vals.append(v)
        pos += rows.size
        done += rows.size
    el = time.perf_counter() - t0
    rows_per_s = done / el
    out = {"value": rows_per_s / 4.0, "unit": UNIT, "cores": 1, "kind": "oracle",
           "nproc": os.cpu_count(), "cpu_model": _cpu_model(),
           "sample": f"FP64 oracle right-hand side (CSR definition) on {done} random rows of the "
                     f"{g.n}-node graph in {el:.1f} s on one core; RK4 step = 4 evaluations, extrapolated to "
                     "N rows"}
    if keep_values:
        out["_rows"] = order[:done]
        out["_ref"] = np.concatenate(vals) if vals else np.zeros(0)
    return out


_CPB = None


def cpu_block_lib():
    """The OpenMP CPU block method (baseline/cpu_block.c), compiled with gcc on first use."""
    global _CPB
    if _CPB is not None:
        return _CPB
    import ctypes as C
    src = os.path.join(ROOT, "baseline", "cpu_block.c")
    lib = os.path.join(ROOT, "baseline", "_cpu_block.so")
    if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fPIC", "-shared", "-fopenmp", "-o", tmp, src, "-lm"])
        os.replace(tmp, lib)
    L = C.CDLL(lib)
    P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    L.cpb_create.restype = P
    L.cpb_create.argtypes = [I64, P, P, P, I32, P, D, D]
    L.cpb_rk4.argtypes = [P, P, D, I64]
    L.cpb_rhs.argtypes = [P, P, P]
    L.cpb_threads.restype = C.c_int
    L.cpb_destroy.argtypes = [P]
    _CPB = L
    return L


class CpuBlock:
    """Handle of the OpenMP CPU block method on one graph (host arrays, user order)."""

    def __init__(self, g, omega, K, tau=0.5):
        L = cpu_block_lib()
        self._keep = [np.ascontiguousarray(g.row_ptr, dtype=np.int64), np.ascontiguousarray(g.col, dtype=np.int32),
                      np.ascontiguousarray(g.label, dtype=np.int32), np.ascontiguousarray(omega, dtype=np.float64)]
        rp, cl, lb, om = self._keep
        self.n = g.n
        self.h = L.cpb_create(g.n, rp.ctypes.data, cl.ctypes.data, lb.ctypes.data, int(g.n_comm), om.ctypes.data,
                              float(K), float(tau))
        if not self.h:
            raise RuntimeError("cpb_create failed")

    def rhs(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        f = np.empty(self.n)
        cpu_block_lib().cpb_rhs(self.h, th.ctypes.data, f.ctypes.data)
        return f

    def rk4(self, theta, h, steps):
        cpu_block_lib().cpb_rk4(self.h, theta.ctypes.data, float(h), int(steps))

    def close(self):
        if self.h:
            cpu_block_lib().cpb_destroy(self.h)
            self.h = None


def cpu_block_baseline(w, seconds: float = 10.0, steps_full: int = 0):
    """The block method on all host cores (OpenMP), timed over whole RK4 steps of the workload (about
    `seconds` of work, at least one step; steps_full > 0 times that many steps instead)."""
    t0 = time.perf_counter()
    cb = CpuBlock(w.graph, w.omega, w.K)
    t_setup = time.perf_counter() - t0
    th = np.array(w.theta0, dtype=np.float64)
    t0 = time.perf_counter()
    cb.rk4(th, w.h, 1)
    t1 = time.perf_counter() - t0
    steps = steps_full if steps_full > 0 else max(1, min(int(seconds / max(t1, 1e-9)), 1000))
    t0 = time.perf_counter()
    cb.rk4(th, w.h, steps)
    el = time.perf_counter() - t0
    cb.close()
    return {"value": w.graph.n * steps / el, "unit": UNIT, "cores": cpu_block_lib().cpb_threads(),
            "kind": "cpu block method (OpenMP, FP64)", "nproc": os.cpu_count(), "cpu_model": _cpu_model(),
            "steps": steps, "seconds": el, "setup_s": t_setup,
            "sample": f"{steps} whole RK4 steps of the {w.graph.n}-node workload, all host cores"}


def _cpu_model() -> str:
    """Host CPU model name (lscpu, else /proc/cpuinfo)."""
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for ln in r.stdout.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model Name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def scale_free_errors(f_gpu, rows, ref, w) -> dict:
    """max over the sampled rows of e_i = |f_i - o_i| / ((K/N)(1 + deg_i)) and of |f_i - o_i|."""
    g = w.graph
    deg = np.diff(g.row_ptr)[rows]
    d = np.abs(np.asarray(f_gpu)[rows] - ref)
    e = d / ((abs(w.K) / g.n) * (1.0 + deg))
    return {"max_scale_free": float(e.max()) if e.size else None, "max_abs": float(d.max()) if d.size else None,
            "rows": int(rows.size)}


def bench_adjoint(dev):
    """Loss 1 - r(T) and its gradients on the 65536-node SBM: T = 20, h = 0.01 (2000 steps), a checkpoint every
    64 steps, FP32 right-hand side, FP64 state.  Reports forward-only and forward+backward wall time."""
    import torch
    from paper_2102_07167_gb300 import gen as G
    from paper_2102_07167_gb300 import kura
    w = G.workload_sbm_small()
    g = w.graph
    h, steps, M = 0.01, 2000, 64

    def measure(k):
        th0 = torch.tensor(w.theta0, device=dev)
        k.adjoint(th0, h, 3 * M, M, 0)                    # warm-up (buffers, captured segments)
        th = th0.clone()
        k.rk4_steps(th, h, 8)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        th = th0.clone()
        e0.record()
        k.rk4_steps(th, h, steps)
        e1.record()
        torch.cuda.synchronize()
        fwd_ms = e0.elapsed_time(e1)
        e0.record()
        L, gom, gK, gth = k.adjoint(th0, h, steps, M, 0)
        e1.record()
        torch.cuda.synchronize()
        adj_ms = e0.elapsed_time(e1)
        return {"forward_ms": fwd_ms, "forward_backward_ms": adj_ms, "ratio": adj_ms / fwd_ms, "loss": L,
                "g_K": gK, "g_theta0_norm": float(torch.linalg.norm(gth)),
                "g_omega_norm": float(torch.linalg.norm(gom))}
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=kura.PREC_MIXED) as k:
        default = measure(k)
        tune = k.autotune(torch.tensor(w.theta0, device=dev), budget_s=20.0)
        tuned = measure(k)
        tuned["autotune"] = tune
    out = {"workload": "SBM N=65536 (64 communities, p_in 0.95, p_out 0.001), loss 1 - r(T), T = 20, "
                       "h = 0.01, 2000 RK4 steps, checkpoint every 64", "precision": "mixed (FP32 RHS, FP64 state)",
           "timing": "CUDA events around each library call (the adjoint call synchronises at its end)"}
    out.update(tuned)
    out["default_plan"] = default
    return out


def adjoint_launches(dev):
    """A short adjoint for a launch list: the adjoint workload's graph with the autotuner's plan for it (index
    lists, tau 0.35), 192 steps with a checkpoint every 64; a warm-up call, then one call inside the NVTX
    range "profiled" (for ncu --nvtx --nvtx-include "profiled/")."""
    import torch
    from paper_2102_07167_gb300 import gen as G
    from paper_2102_07167_gb300 import kura
    w = G.workload_sbm_small()
    g = w.graph
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=kura.PREC_MIXED, tau=0.35,
                       tensor_cores=0) as k:
        th0 = torch.tensor(w.theta0, device=dev)
        k.adjoint(th0, 0.01, 192, 64, 0)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("profiled")
        L, gom, gK, gth = k.adjoint(th0, 0.01, 192, 64, 0)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    return {"workload": "SBM N=65536, loss 1 - r(T), h = 0.01, 192 steps, checkpoint every 64, index lists, "
                        "tau 0.35", "loss": L, "g_K": gK}


def bench_batch(dev, steps: int = 1000, tc_steps: int = 50, dist=None):
    """2048 independent trajectories of uneven size in one persistent launch (half complete graphs, half SBMs),
    h = 0.01, mixed precision: the dense-block zeros as index lists (1000 steps), and as 0/1 masks multiplied
    on the tensor cores with split BF16 (sin, cos) (tc_steps steps).  With more than one rank, every rank
    takes its LPT share of the trajectories and integrates it (index lists), with no collective in the
    data path; the line is the whole batch's oscillator-steps over the slowest rank's time."""
    import torch
    from paper_2102_07167_gb300 import gen as G
    from paper_2102_07167_gb300 import kura
    t0 = time.perf_counter()
    ens = G.workload_batch()
    t_gen = time.perf_counter() - t0
    world = dist.get_world_size() if dist is not None and dist.is_initialized() else 1
    if world > 1:
        o = kura.kura_default_opts()
        o.precision = kura.PREC_MIXED
        rank = dist.get_rank()
        mine, part, load = shard_trajectories(G.batch_graphs(ens), world, rank, o)
        sub = [ens[int(t)] for t in mine]
        theta0 = np.concatenate([th for (_, _, _, th, _) in sub])

        def barrier():
            dist.barrier()
            torch.cuda.synchronize()

        with kura.KuramotoBatch(G.batch_graphs(sub), tensor_cores=0) as b:
            th = torch.tensor(theta0, device=dev)
            value, el_ms, n_all = timed_shards(lambda k: b.rk4_steps(th, 0.01, k), theta0.size, steps, 3, barrier,
                                               EventTimer(), dist, dev)
        return {"workload": "2048 trajectories, n log-uniform in [256, 16384], half complete graphs, half SBMs "
                            "(8-32 communities, p_in 0.9, p_out 0.005), K ~ U[0.5, 5], h = 0.01",
                "n_total": n_all, "value": value, "unit": UNIT, "steps": steps, "ms_per_step": el_ms / steps,
                "scaling": "strong", "sharding": {
                    "ranks": world, "rule": "LPT on kura_batch_costs (kura_partition_lpt), no collective",
                    "trajectories_per_rank": np.bincount(part, minlength=world).tolist(),
                    "cost_per_rank": load.tolist(), "max_over_mean_cost": float(load.max() / load.mean())},
                "precision": "mixed, index lists"}
    theta0 = np.concatenate([th for (_, _, _, th, _) in ens])

    def run(tcm, nsteps):
        t0 = time.perf_counter()
        with kura.KuramotoBatch(G.batch_graphs(ens), tensor_cores=tcm) as b:
            t_create = time.perf_counter() - t0
            st, info = b.stats(), b.info()
            th = torch.tensor(theta0, device=dev)
            b.rk4_steps(th, 0.01, 3)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.rk4_steps(th, 0.01, nsteps)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
        return {"steps": nsteps, "ms": ms, "ms_per_step": ms / nsteps,
                "value": info["n_total"] * nsteps / (ms / 1e3), "unit": UNIT, "create_s": t_create,
                "listed_corrections": st["missing_entries"] + st["sparse_entries"],
                "tc_trajectories": info["tc_traj"], "tc_tiles": info["tc_tiles"], "tc_mask_bits": info["tc_mask_bits"],
                "gpu_launches": 3}
    lists = run(0, steps)
    tc = run(2, tc_steps)
    # the batch autotuner: per size class, dense-zero encoding, row tile and tau (30 s budget)
    t0 = time.perf_counter()
    with kura.KuramotoBatch(G.batch_graphs(ens), tensor_cores=0) as b:
        tune = b.autotune(theta0, budget_s=30.0)
        t_tune = time.perf_counter() - t0
        choices = {}
        for t in range(len(ens)):
            if ens[t][0] is not None:
                key = str(b.traj_params(t))
                choices[key] = choices.get(key, 0) + 1
        info = b.info()
        th = torch.tensor(theta0, device=dev)
        b.rk4_steps(th, 0.01, 3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.rk4_steps(th, 0.01, steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    tuned = {"steps": steps, "ms_per_step": ms / steps, "value": info["n_total"] * steps / (ms / 1e3), "unit": UNIT,
             "tune_seconds": t_tune, "candidates": tune["candidates"],
             "sbm_trajectories_by_choice_tau_tc_lanes": choices, "tc_trajectories": info["tc_traj"]}
    return {"workload": "2048 trajectories, n log-uniform in [256, 16384], half complete graphs, half SBMs "
                        "(8-32 communities, p_in 0.9, p_out 0.005), K ~ U[0.5, 5], h = 0.01",
            "n_total": int(theta0.size), "value": max(lists["value"], tuned["value"]), "unit": UNIT,
            "generate_s": t_gen, "autotuned": tuned,
            "precision": "mixed (FP32 sin/cos and corrections, exact fixed-point block sums, FP64 epilogue/state)",
            "cuda_cores_index_lists": lists,
            "tensor_cores_split_bf16": dict(tc, note="dense-block zeros as a BF16 0/1 mask x split BF16 (sin_hi, "
                                            "sin_lo, cos_hi, cos_lo) per trajectory: M = 128, N = 16 (4 useful), "
                                            "tcgen05.mma.kind::f16, FP32 accumulation; a matrix-vector product "
                                            "per trajectory, so the tensor cores are 1/4 used"),
            "tc_over_lists_time": tc["ms_per_step"] / lists["ms_per_step"]}


def bench_complete_512(dev):
    """Classical all-to-all model, N = 512, K = 2, h = 0.01, 200 steps, FP64 (the latency-bound case): the
    CUDA-graph step loop (4 row kernels per step and one trig launch per 8-step graph) against the measured
    graph launch floor for that many kernels, the persistent
    single-CTA form (a batch of one trajectory: one launch runs all 200 steps), the GPU direct sum, and the
    CPU baselines on the whole trajectory."""
    import torch
    from paper_2102_07167_gb300 import gen as G
    from paper_2102_07167_gb300 import kura
    w = G.workload_complete(512)
    g = w.graph

    def timed(fn, reps=5):
        out = []
        for _ in range(reps):
            th = torch.tensor(w.theta0, device=dev)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn(th)
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return float(np.median(out)), th.cpu().numpy()
    with kura.Kuramoto(g.row_ptr, g.col, g.label, 1, w.omega, w.K, precision=kura.PREC_FP64,
                       persistent_small=0) as k:
        k.rk4_steps(torch.tensor(w.theta0, device=dev), w.h, w.n_steps)
        ms_graph, th_graph = timed(lambda th: k.rk4_steps(th, w.h, w.n_steps))
        ms_direct, _ = timed(lambda th: k.direct_rk4_steps(th, w.h, w.n_steps, kura.PREC_FP64), reps=3)
    with kura.Kuramoto(g.row_ptr, g.col, g.label, 1, w.omega, w.K, precision=kura.PREC_FP64) as kc:
        kc.rk4_steps(torch.tensor(w.theta0, device=dev), w.h, w.n_steps)
        ms_cluster, th_cluster = timed(lambda th: kc.rk4_steps(th, w.h, w.n_steps))
    with kura.KuramotoBatch([(None, None, None, 1, w.omega, w.K)], precision=kura.PREC_FP64) as b:
        b.rk4_steps(torch.tensor(w.theta0, device=dev), w.h, w.n_steps)
        ms_pers, th_pers = timed(lambda th: b.rk4_steps(th, w.h, w.n_steps))
    floor_us = kura.kura_measure_graph_launch_floor(8, 2000)
    st = w.n_steps
    per_step = LAUNCHES_PER_STEP
    res = {"workload": "complete graph N=512, K = 2, h = 0.01, 200 RK4 steps, FP64",
           "graph_step_loop": {"us_per_step": ms_graph * 1e3 / st, "value": g.n * st / (ms_graph / 1e3),
                               "launches_per_step": per_step},
           "launch_floor": {"us_per_kernel": floor_us, "us_per_step": per_step * floor_us,
                            "how": "CUDA graph of 8 empty dependent kernels, replayed 2000 times; per step "
                                   "times the step loop's launches per step"},
           "graph_over_floor": (ms_graph * 1e3 / st) / (per_step * floor_us),
           "persistent_single_cta": {"us_per_step": ms_pers * 1e3 / st, "value": g.n * st / (ms_pers / 1e3),
                                     "launches": 1},
           "persistent_cluster": {"us_per_step": ms_cluster * 1e3 / st, "value": g.n * st / (ms_cluster / 1e3),
                                  "launches": 1, "how": "kura_rk4_steps on a small graph: one launch of one "
                                                        "8-CTA thread-block cluster for all 200 steps"},
           "direct_fp64": {"us_per_step": ms_direct * 1e3 / st, "value": g.n * st / (ms_direct / 1e3)}}
    # CPU legs: the oracle as it stands (CSR definition, one core) on the whole trajectory, and the
    # OpenMP block method; the oracle's final phases also give the GPU paths' error
    import oracle
    t0 = time.perf_counter()
    ref = oracle.rk4_csr(g.row_ptr, g.col, w.omega, w.K, w.theta0, w.h, st)
    t_orc = time.perf_counter() - t0
    res["cpu_baseline"] = {"value": g.n * st / t_orc, "unit": UNIT, "cores": 1, "kind": "oracle",
                           "sample": f"whole trajectory ({st} steps) by oracle.rk4_csr in {t_orc:.1f} s"}
    res["cpu_block_baseline"] = cpu_block_baseline(w, steps_full=st)
    res["max_abs_err_vs_oracle"] = {"graph_step_loop": float(np.abs(th_graph - ref).max()),
                                    "persistent_single_cta": float(np.abs(th_pers - ref).max()),
                                    "persistent_cluster": float(np.abs(th_cluster - ref).max())}
    res["value"] = g.n * st / (ms_cluster / 1e3)
    res["unit"] = UNIT
    return res


def bench_sbm_65536(dev, cpu_seconds: float = 8.0):
    """SBM N = 65536 (64 communities, p_in 0.95, p_out 0.001), K = 4, FP64, h = 0.005, its 1000 steps: the
    correction stream (~35 MB) and node data stay in L2, so the row kernel is measured against the L2 read
    bandwidth (measured here) as well as HBM."""
    import torch
    from paper_2102_07167_gb300 import gen as G
    from paper_2102_07167_gb300 import kura
    w = G.workload_sbm_small()
    g = w.graph
    l2 = kura.kura_measure_l2_bandwidth(48 << 20)
    hbm, _ = _peaks()
    floor_us = kura.kura_measure_graph_launch_floor(8, 2000)

    def measure(k):
        st = k.stats()
        th = torch.tensor(w.theta0, device=dev)
        k.set_timing(True)
        k.rk4_steps(th, w.h, 8)
        torch.cuda.synchronize()
        th = torch.tensor(w.theta0, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        k.rk4_steps(th, w.h, w.n_steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        kt = k.kernel_times()
        alg = 4 * (st["missing_entries"] + st["sparse_entries"]) + st["node_bytes_row"]
        row_ms = float(np.mean(kt)) if kt.size else None
        ach = alg / (row_ms * 1e-3) / 1e9 if row_ms else None
        return {"value": g.n * w.n_steps / (ms / 1e3), "unit": UNIT, "us_per_step": ms * 1e3 / w.n_steps,
                "tensor_core_tiles": int(st["tc_tiles"]), "tiles": int(st["tiles"]), "tau": st["tau"],
                "roofline": {"bound": "l2", "kernel": "k_row_stage", "achieved": ach, "peak": l2, "unit": "GB/s",
                             "frac": ach / l2 if ach else None, "hbm_frac": ach / hbm if ach else None,
                             "algorithmic_bytes_per_launch": alg, "row_kernel_ms": row_ms,
                             "peak_source": "kura_measure_l2_bandwidth(48 MiB), measured in this run"}}
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=kura.PREC_FP64) as k:
        default = measure(k)
        tune = k.autotune(torch.tensor(w.theta0, device=dev), budget_s=20.0)
        tuned = measure(k)
        tuned["autotune"] = tune
    res = {"workload": "SBM N=65536, 64 communities, p_in 0.95, p_out 0.001, K = 4, FP64, h = 0.005, 1000 steps",
           "value": tuned["value"], "unit": UNIT, "us_per_step": tuned["us_per_step"],
           "launch_floor_us_per_step": LAUNCHES_PER_STEP * floor_us, "roofline": tuned["roofline"],
           "default_plan": default, "autotuned_plan": tuned}
    res["cpu_baseline"] = cpu_baseline_oracle(w, seconds=cpu_seconds)
    res["cpu_block_baseline"] = cpu_block_baseline(w, seconds=cpu_seconds)
    return res


def bench_ensemble(dev, n_traj: int = 64, steps: int = 200):
    """64 trajectories sharing the 65536-node SBM (64 communities, p_in 0.95, p_out 0.001): own omega ~ N(0,1),
    K ~ U[0.5, 5] and theta0 ~ U[0, 2 pi) each; the dense-block product is a BF16 tensor-core GEMM over the
    trajectories; h = 0.005. Next to it, one single-trajectory mixed-precision handle on the same graph."""
    import torch
    from paper_2102_07167_gb300 import gen as G
    from paper_2102_07167_gb300 import kura
    w = G.workload_sbm_small()
    g = w.graph
    rng = np.random.default_rng(0)
    omega = rng.normal(size=(n_traj, g.n))
    K = rng.uniform(0.5, 5.0, n_traj)
    theta = rng.uniform(0.0, 2 * np.pi, (n_traj, g.n))

    def timed(obj, th, h):
        obj.rk4_steps(th, h, 3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        obj.rk4_steps(th, h, steps)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)
    t0 = time.perf_counter()
    with kura.KuramotoEnsemble(g.row_ptr, g.col, g.label, g.n_comm, omega, K) as e:
        t_create = time.perf_counter() - t0
        st = e.stats()
        ms = timed(e, torch.tensor(theta, device=dev), 0.005)
        # error of one right-hand side against the library's FP64 mode, a few trajectories
        th = torch.tensor(theta, device=dev)
        out = torch.empty_like(th)
        e.rhs(th, out)
        f = out.cpu().numpy()
    errs = []
    for b in (0, n_traj // 2, n_traj - 1):
        with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, omega[b], K[b], precision=kura.PREC_FP64) as k64:
            t64 = torch.tensor(theta[b], device=dev)
            o64 = torch.empty_like(t64)
            k64.rhs(t64, o64)
            ref = o64.cpu().numpy()
        errs.append(float(np.max(np.abs(f[b] - ref) / (1 + np.diff(g.row_ptr)))))
    with kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, omega[0], K[0], precision=kura.PREC_MIXED) as k:
        ms1 = timed(k, torch.tensor(theta[0], device=dev), 0.005)
    v = g.n * n_traj * steps / (ms / 1e3)
    v1 = g.n * steps / (ms1 / 1e3)
    return {"workload": f"{n_traj} trajectories sharing the SBM N=65536 (64 communities, p_in 0.95, p_out 0.001); "
                        "own omega, K ~ U[0.5, 5], theta0; h = 0.005",
            "steps": steps, "ms": ms, "value": v, "unit": UNIT, "create_s": t_create,
            "tensor_core_tiles": int(st["tc_tiles"]), "tiles": int(st["tiles"]),
            "gemm": "per 128-row tile and 16 trajectories: BF16 0/1 mask x split BF16 (sin_hi, sin_lo, cos_hi, cos_lo), "
                    "N = 64, FP32 accumulation (tcgen05.mma.kind::f16)",
            "rhs_max_abs_err_over_1_plus_deg_vs_fp64_mode": max(errs),
            "single_trajectory_handle": {"value": v1, "ms_per_step": ms1 / steps},
            "speedup_per_oscillator_vs_single": v / v1}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    w = _workload(args.workload)
    per_step = []
    for _ in range(args.warmup):
        cpu_baseline_oracle(w, seconds=0.5)
    for _ in range(args.steps):
        per_step.append(cpu_baseline_oracle(w, seconds=max(1.0, 60.0 / max(args.steps, 1))))
    vals = [p["value"] for p in per_step]
    v = float(np.mean(vals))
    ms = w.graph.n / v * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n": w.graph.n},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": per_step[-1]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    from paper_2102_07167_gb300 import kura

    world, rank, local = _dist()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    prec = kura.PREC_MIXED if args.precision == "mixed" else kura.PREC_FP64

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w = _workload(args.workload)
    g = w.graph
    n = g.n
    k = kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=prec)
    st = k.stats()
    theta = torch.tensor(w.theta0, device=dev)

    # ---- warm-up, then the timed region: K RK4 steps through one library call
    k.set_timing(True)
    with ClockSampler(local) as clk:
        value, el_ms = timed_replicas(lambda ks: k.rk4_steps(theta, w.h, ks), n, args.steps, args.warmup,
                                      barrier, EventTimer(), dist, dev)
    launch_ms = k.kernel_times()
    ms_step = el_ms / args.steps
    # per 8-step graph: one trig/block-sum launch and 32 row kernels (the fused trig); two permutations
    gpu_launches = 4 * args.steps + -(-args.steps // 8) + 2

    # ---- roofline of the dominant kernel (row kernel): algorithmic bytes / mean launch time
    peak, peak_kind = _peaks()
    # algorithmic bytes of the method: 4 B per stored correction index (a missing entry of a dense block or
    # a present entry of a sparse block, int32) plus the row kernel's per-node traffic; the bytes the
    # chosen encoding streams (tensor-core mask images, headers, digits) are reported beside them
    alg_bytes = 4 * (st["missing_entries"] + st["sparse_entries"]) + st["node_bytes_row"]
    enc_bytes = st["stream_bytes"] + st["node_bytes_row"]
    row_ms = float(np.mean(launch_ms)) if launch_ms.size else None
    achieved = alg_bytes / (row_ms * 1e-3) / 1e9 if row_ms else None
    achieved_enc = enc_bytes / (row_ms * 1e-3) / 1e9 if row_ms else None
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "row_kernel_traffic.json")
    if os.path.exists(tpath):
        try:
            from paper_2102_07167_gb300 import _build
            rec = json.load(open(tpath))
            if rec.get("source_hash") == _build.kernel_source_hash() and rec.get("workload") == w.name \
                    and rec.get("precision") == args.precision:
                traffic = rec.get("traffic_bytes_per_launch")
        except Exception:
            traffic = None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured"
                else "fallback 6.8 TB/s", "kernel": "k_row_stage",
                "algorithmic_bytes_per_launch": alg_bytes,
                "algorithmic_bytes_def": "4 B per stored correction index (missing + present entries) + "
                                         f"{st['node_bytes_row'] // max(n, 1)} B per node (row kernel node traffic)",
                "encoding_bytes_per_launch": enc_bytes, "encoding_achieved": achieved_enc,
                "encoding_frac": (achieved_enc / peak) if achieved_enc else None,
                "row_kernel_ms": row_ms,
                "launches_timed": int(launch_ms.size),
                # the kernel's actual limiter: random L2 gathers of the present (sparse-block) entries
                "present_gathers_per_launch": int(st["sparse_entries"]),
                "present_gather_rate_per_s": (st["sparse_entries"] / (row_ms * 1e-3)) if row_ms else None,
                "tensor_core_tiles": int(st["tc_tiles"]), "tiles": int(st["tiles"])}

    # ---- the bound the row kernel actually meets: random L2 gathers of its sparse-block entries,
    # against the rate this device reaches on the same kind of gathers (measured now, same process)
    gather_peak = kura.kura_measure_gather_rate(1 << 20, 1 << 28, 8 if args.precision == "mixed" else 16)
    gather_rate = (st["sparse_entries"] / (row_ms * 1e-3)) if row_ms else None
    gather_roofline = {"bound": "l2_random_gather", "achieved": gather_rate, "peak": gather_peak,
                       "unit": "gathers/s", "frac": (gather_rate / gather_peak) if gather_rate else None,
                       "peak_source": "measured in this run (kura_measure_gather_rate): 2^28 random "
                                      f"{8 if args.precision == 'mixed' else 16}-byte gathers from an L2-resident "
                                      "2^20-entry table, four per 16-byte index load, full occupancy, median of 3",
                       "kernel": "k_row_stage"}

    # ---- e2e: the public call with pinned HOST phases, copies inside every step
    e2e = None
    if not args.no_e2e:
        host = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        host[:] = w.theta0
        k.rk4_steps(host, w.h, 1)
        ke = max(5, min(args.steps, 50))
        barrier()
        t0 = time.perf_counter()
        for _ in range(ke):
            k.rk4_steps(host, w.h, 1)
        el = time.perf_counter() - t0
        e2e = {"value": n * ke / el, "unit": UNIT, "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
               "steps": ke, "note": "kura_rk4_steps(host pointer, n_steps=1) per step: H2D, permute, 1 RK4 "
                                    "step, un-permute, D2H, synchronise"}

    extra = {}
    f_host = {}
    if not args.quick and rank == 0:
        # mixed vs FP64 path error on one right-hand side (both through the library)
        th0 = torch.tensor(w.theta0, device=dev)
        f_a = torch.empty_like(th0)
        k.rhs(th0, f_a)
        other = kura.PREC_FP64 if prec == kura.PREC_MIXED else kura.PREC_MIXED
        k.close()
        k = None
        k2 = kura.Kuramoto(g.row_ptr, g.col, g.label, g.n_comm, w.omega, w.K, precision=other)
        f_b = torch.empty_like(th0)
        k2.rhs(th0, f_b)
        f_host = {args.precision: f_a.cpu().numpy(), ("fp64" if other == kura.PREC_FP64 else "mixed"): f_b.cpu().numpy()}
        deg = torch.tensor(np.diff(g.row_ptr), device=dev, dtype=torch.float64)
        err = (f_a - f_b).abs()
        extra["rhs_error_vs_other_precision"] = {
            "max_abs": float(err.max()), "max_scaled": float((err / (1 + deg)).max()),
            "note": "|f_mixed - f_fp64|, and divided by (1 + deg_i); both through the library"}
        # the other precision's throughput
        th = th0.clone()
        k2.rk4_steps(th, w.h, 3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ks = max(10, args.steps // 4)
        e0.record()
        k2.rk4_steps(th, w.h, ks)
        e1.record()
        torch.cuda.synchronize()
        mso = e0.elapsed_time(e1) / ks
        extra["fp64_mode" if other == kura.PREC_FP64 else "mixed_mode"] = {
            "value": n / mso * 1e3, "ms_per_step": mso, "steps": ks}
        # GPU direct-summation baselines (one sine per edge)
        direct = {}
        for dp, name in ((kura.PREC_MIXED, "fp32"), (kura.PREC_FP64, "fp64")):
            th = th0.clone()
            k2.direct_rk4_steps(th, w.h, 1, dp)
            torch.cuda.synchronize()
            nd = 2 if dp == kura.PREC_FP64 else 5
            e0.record()
            k2.direct_rk4_steps(th, w.h, nd, dp)
            e1.record()
            torch.cuda.synchronize()
            msd = e0.elapsed_time(e1) / nd
            direct[name] = {"value": n / msd * 1e3, "ms_per_step": msd, "steps": nd}
        direct["speedup_vs_fp64_direct"] = value / world / direct["fp64"]["value"]
        direct["speedup_vs_fp32_direct"] = value / world / direct["fp32"]["value"]
        extra["direct_baseline"] = direct
        k2.close()
    if k is not None:
        k.close()
    if not args.quick and not args.no_batch:
        # every rank: with more than one, the batch is sharded across them (before the rank-0-only extras,
        # so that no rank waits at a barrier while another runs them)
        b = bench_batch(dev, dist=dist)
        if rank == 0:
            extra["batch"] = b
    if not args.quick and rank == 0 and not args.no_adjoint:
        extra["adjoint"] = bench_adjoint(dev)
    if not args.quick and rank == 0 and not args.no_configs:
        extra["configs"] = {"complete_512": bench_complete_512(dev), "sbm_65536": bench_sbm_65536(dev)}
    if not args.quick and rank == 0 and not args.no_ensemble:
        extra["ensemble_shared_graph"] = bench_ensemble(dev)

    cpu = cpu_baseline_oracle(w, seconds=args.cpu_seconds, keep_values=True) \
        if (rank == 0 and world == 1 and not args.quick) else None
    if cpu is not None:
        extra["cpu_block_baseline"] = cpu_block_baseline(w, seconds=args.cpu_seconds)
        rows, ref = cpu.pop("_rows"), cpu.pop("_ref")
        # the rows the CPU-baseline leg evaluated with the oracle give the GPU's error at the same phases
        extra["rhs_error_vs_oracle"] = {
            p: scale_free_errors(f, rows, ref, w) for p, f in f_host.items()}
        extra["rhs_error_vs_oracle"]["definition"] = (
            "e_i = |f_i - o_i| / ((K/N)(1 + deg_i)) on the rows of the cpu_baseline sample, o = FP64 oracle "
            "(CSR definition); bound 1e-6 mixed, 1e-10 FP64")
    if rank == 0:
        line = core_line(value, world, args.steps, args.warmup, el_ms,
                         "f32+f64" if prec == kura.PREC_MIXED else "f64",
                         dict(_workload_desc(w, st), precision=args.precision))
        line.update({"e2e": e2e, "gpu_launches": gpu_launches, "roofline": roofline,
                     "gather_roofline": gather_roofline, "cpu_baseline": cpu, "clocks": clk.summary()})
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="sbm-2p20", choices=["sbm-2p20", "sbm-2p19", "sbm-2p18", "sbm-65536", "complete-512"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--quick", action="store_true", help="skip the extra comparisons and the CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-configs", action="store_true")
    ap.add_argument("--only", choices=["ensemble", "batch", "complete-512", "sbm-65536", "adjoint", "adjoint-launches"],
                    default=None,
                    help="run one of the extra measurements alone (for profiling) and print its JSON")
    args = ap.parse_args()
    if args.only is not None:
        import torch
        dev = torch.device("cuda", 0)
        if args.only == "ensemble":
            out = bench_ensemble(dev, steps=args.steps)
        elif args.only == "batch":
            out = bench_batch(dev, steps=args.steps, tc_steps=max(1, args.steps // 5))
        elif args.only == "complete-512":
            out = bench_complete_512(dev)
        elif args.only == "adjoint":
            out = bench_adjoint(dev)
        elif args.only == "adjoint-launches":
            out = adjoint_launches(dev)
        else:
            out = bench_sbm_65536(dev)
        print(json.dumps(out))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
