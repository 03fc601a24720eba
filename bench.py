"""Benchmark: exact (k+1)-subsets tested per second (and degrees per second) on one GB300.

Workload: the single larger system (n = 24 variables, 16 random binomials with exponents in
{0,1,2} and at most 4 nonzeros per monomial, seed 0; rank 16, so k = 8): 25 kernel points in
Z^8 and C(25, 9) = 2,042,975 subsets per degree.  A step is one complete exact volume pass
(lift, enumerate every subset with the exact lower-facet test, reduce, read the result and
re-lift on a tie) with the reduced points resident in device memory.  The e2e figure runs the
public call bd_degree(A) from a host matrix per step (Smith form, kernel basis, device copies,
enumeration, result read).  L2 is flushed (a 256 MB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "single_n24_k8"

# DRAM bytes (read + write) of one enumeration launch, from an ncu capture of the kernel built
# from exactly these sources (profiles/k_enumerate_*.md); reported only while the library
# sources still hash to the captured version, null otherwise.
TRAFFIC = {"sources_sha256": "4c5e5db3658ba52d8528820bd46484af652a3b26d5f670e7ce88a46b0fb4ab8d",
           "single_n24_k8": 1138176 + 0, "heavy_quiver_n32_k10": 8020480 + 0}


# the sources that determine the enumeration kernel's code and its work list
KERNEL_SOURCES = ("bd_core.cuh", "bd_kernels.cuh", "bd_kernels.cu", "bd_worklist.cpp", "bd_host.h", "bd_lifts.h")


def sources_sha256() -> str:
    import hashlib
    d = os.path.join(ROOT, "paper_1501_02237_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    from paper_1501_02237_gb300 import build as B  # and the compiler flags (paths relative to the repo)
    h.update(repr((B.ARCH, [f.replace(B.ROOT, "<repo>") for f in B.FLAGS])).encode())
    return h.hexdigest()
METRIC = "exact (k+1)-subsets tested/sec (exact degrees/sec alongside), 1 GB300"
UNIT = "subsets/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch-serve", action="store_true", help="skip the batch and serving sections")
    ap.add_argument("--workload", default=WORKLOAD, help="single system timed (profiling runs use the others)")
    ap.add_argument("--mixed-only", default=None, metavar="WORKLOAD",
                    help="run only the mixed-volume section on this workload (profiling runs)")
    ap.add_argument("--pivot-only", default=None, metavar="M,K",
                    help="run only the pivoting section on the master space W_{M,K} (profiling runs)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_step(system):
    from oracle.degree import degree as oracle_degree

    return oracle_degree(system.A.tolist())


def run_reference(args, rank, world):
    """The oracle (plain exact Python) timed on this host's cores on the same workload."""
    if rank != 0:
        return
    from math import comb

    from workloads import config_system

    s = config_system(args.workload)
    r = oracle_step(s)
    subsets = comb(s.n + 1, r.dim + 1)
    for _ in range(args.warmup):
        oracle_step(s)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(s)
    dt = time.perf_counter() - t0
    value = subsets * args.steps / dt
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * dt / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="exact rationals (Python int)", data="synthetic",
                config=dict(workload=args.workload, n=s.n, m=s.m, k=r.dim, subsets_per_step=subsets,
                            note="each step = one exact degree of the workload by the oracle"),
                degrees_per_s=args.steps / dt,
                cpu_baseline=dict(value=value, unit=UNIT, cores=1, kind="oracle",
                                  sample=f"{args.steps} full exact degrees of the workload, single thread"),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def cpu_baseline(system, subsets, budget_s=15.0):
    t0 = time.perf_counter()
    n = 0
    while True:
        oracle_step(system)
        n += 1
        if time.perf_counter() - t0 > budget_s or n >= 30:
            break
    dt = time.perf_counter() - t0
    return dict(value=subsets * n / dt, unit=UNIT, cores=1, kind="oracle",
                sample=f"{n} full exact degrees of the workload ({dt:.1f} s, single thread)")


def cpu_native(bd, P, nvol, budget_s=5.0):
    """The library's own C++ emulation of the enumeration walker (the same work list and exact
    tests) on every host core: the native CPU comparison point beside the GPU figure."""
    import numpy as np

    W = np.random.default_rng(0).integers(1, 1 << 20, size=P.shape[0], endpoint=True)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    n = 0
    while True:
        r = bd.host_volume_lifted(P, W, threads=threads)
        n += 1
        if time.perf_counter() - t0 > budget_s or n >= 20:
            break
    dt = time.perf_counter() - t0
    subsets = math.comb(P.shape[0], P.shape[1] + 1)
    return dict(value=subsets * n / dt, unit=UNIT, cores=threads, kind="library host emulation",
                exact_match=r["status"] != 0 or r["nvol"] == nvol,
                sample=f"{n} exact volumes of the workload ({dt:.1f} s, {threads} threads)")


def batch_section(bd, seed=0):
    """The batched form against one launch per system on the uneven 4096-system workload
    (n ~ U[12,28], k ~ U[4,9], exponents in {0,1,2}, seeds 0..4095), exact agreement checked."""
    from workloads import batch_systems

    systems = batch_systems(4096)
    b = bd.Batch()
    for s in systems:
        b.add(s.A, seed=seed)
    b.prepare()
    out = {}
    ref = None
    for label, kw in [("batched", dict(mode=0, autotune=True)), ("batched", dict(mode=0, autotune=True)),
                      ("batched_graph", dict(mode=0, autotune=True, use_graph=True)),
                      ("per_system", dict(mode=1))]:
        st = b.run(**kw)
        res = [(r["degree"], r["nvol"]) for r in b.results()]
        ref = ref or res
        assert res == ref, "batched and per-system results differ"
        out[label] = dict(systems_per_s=len(systems) / (st["wall_ms"] / 1e3), wall_ms=st["wall_ms"],
                          gpu_ms=st["gpu_ms"], subsets_per_s=st["subsets"] / (st["wall_ms"] / 1e3),
                          launches=st["launches"], warps_per_block=st["warps_per_block"],
                          item_factor=st["item_factor"])
    out["systems"] = len(systems)
    out["subsets"] = int(st["subsets"])
    out["host_reduce_ms"] = st["host_ms"]
    out["speedup_batched_vs_per_system"] = out["batched"]["systems_per_s"] / out["per_system"]["systems_per_s"]
    return out


def start_section(bd, P, seed=0, coef_seed=1):
    """The witness-set start solutions of every cell of the workload (Sec. 6), kept on the
    device: solutions/s end to end (cells, per-cell preparation, solutions, residual check)."""
    import torch
    _, vol = bd.cells(P, seed=seed, capacity=1 << 16)
    out = torch.empty((vol["nvol"], P.shape[1]), dtype=torch.complex128, device="cuda")
    bd.start_solutions(P, seed=seed, coef_seed=coef_seed, device_out=out)  # warm-up
    ts = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n, res = bd.start_solutions(P, seed=seed, coef_seed=coef_seed, device_out=out)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    dt = statistics.median(ts)
    return dict(solutions=n, cells=vol["cells"], ms=1e3 * dt, solutions_per_s=n / dt, max_residual=res,
                note="all start solutions of the workload's cells, on the device")


MIXED_WORKLOAD = "mixed_k7_p8"


def mixed_section(bd, name=MIXED_WORKLOAD, seed=0, runs=3, cpu_seconds=5.0):
    """Mixed volume (the BKK bound, Appendix A) of the sparse supports `name` (k = 7 sets of 8
    exponent vectors in {0,1,2}^7: 28^7 = 1.35e10 tuples of pairs): tuples of pairs resolved per
    second by the enumeration kernel (CUDA events) and per public call, against the oracle's
    rational test of single tuples on one host core (a bounded random sample)."""
    import random

    from oracle.lifts import lifts as oracle_lifts
    from oracle.mixed import cell_status
    from workloads import mixed_config

    S = mixed_config(name)
    bd.mixed_volume(S, seed=seed)  # warm-up
    dev, wall = [], []
    r = None
    for _ in range(runs):
        t0 = time.perf_counter()
        r = bd.mixed_volume(S, seed=seed)
        wall.append(time.perf_counter() - t0)
        dev.append(r["device_ms"])
    d, w = statistics.median(dev), statistics.median(wall)
    # the oracle on a sample of random tuples
    SL = [A.tolist() for A in S]
    W = oracle_lifts(sum(len(A) for A in SL), seed)
    pairs = [[(p, q) for p in range(len(A)) for q in range(p + 1, len(A))] for A in SL]
    rng = random.Random(1)
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < cpu_seconds:
        cell_status(SL, W, tuple(rng.choice(P) for P in pairs))
        done += 1
    cpu_rate = done / max(time.perf_counter() - t0, 1e-9)
    return dict(workload=name, k=len(S), points_per_set=len(S[0]), tuples=r["tuples"], mv=r["mv"], cells=r["cells"],
                int_path="int128" if r["flags"] & bd.BD_FLAG_INT128 else "int64", kernel_ms=d,
                tuples_per_s=r["tuples"] / (d / 1e3), call_ms=1e3 * w, call_tuples_per_s=r["tuples"] / w,
                cpu_baseline=dict(value=cpu_rate, unit="tuples/s", cores=1, kind="oracle",
                                  sample=f"{done} random tuples through oracle.mixed.cell_status ({cpu_seconds:.0f} s)"))


PIVOT_WORKLOADS = ("4,4", "3,6", "4,5")


def pivot_section(bd, systems=PIVOT_WORKLOADS, seed=0):
    """Output-sensitive degrees by simplicial pivoting (Sec. 4.2) of master spaces of Table
    mspace-deg that the subset enumeration cannot reach (W_{4,4}: 1.9e13 subsets, W_{3,6}: 8.4e14,
    W_{4,5}: 3.7e16): per system the exact degree against the table, cells walked per second on
    the GPU and the time of the public call bd_degree_pivot(A)."""
    from workloads import master_space_system

    table = json.load(open(os.path.join(ROOT, "tests", "golden", "master_space_table.json")))["degree"]
    out = {}
    for mk in systems:
        m, k = map(int, mk.split(","))
        s = master_space_system(m, k)
        red = bd.reduce(s.A)
        P = red["points"]
        v = bd.volume_pivot(P, seed=seed)  # warm-up and device time
        t0 = time.perf_counter()
        r = bd.degree_pivot(s.A, s.coef, seed=seed)
        call = time.perf_counter() - t0
        out[f"W{m},{k}"] = dict(points=int(P.shape[0]), dim=int(P.shape[1]),
                               subsets=float(math.comb(P.shape[0], P.shape[1] + 1)), degree=r["degree"],
                               table=table.get(mk), exact_match=r["degree"] == table.get(mk), cells=v["cells"],
                               relifts=v["relifts"], device_ms=v["device_ms"],
                               cells_per_s=v["cells"] / (v["device_ms"] / 1e3), call_s=call)
    return out


def serve_section(bd, rate=200.0, count=1000, train_count=20000):
    """Cost model trained on method-generated runs, then a Poisson stream served with continuous
    batching (n ~ U[12,30], k ~ U[4,10]); p50/p99 latency and degrees/s per admission policy."""
    import numpy as np

    from workloads import batch_systems, poisson_arrivals

    t0 = time.perf_counter()
    train = batch_systems(train_count, first_seed=200000, n_range=(12, 30), k_range=(4, 10))
    b = bd.Batch()
    for s in train:
        b.add(s.A)
    b.prepare()
    b.run(mode=0)
    cyc = np.array([r["cycles"] for r in b.results()], dtype=np.float64)
    X = b.features()
    keep = cyc > 0
    X, y = X[keep], np.log2(cyc[keep]).astype(np.float32)
    ntr = int(0.8 * len(y))
    model = bd.CostModel(0)
    model.train(X[:ntr], y[:ntr], epochs=150, batch=256, lr=2e-3, seed=1)
    mae_model = float(np.mean(np.abs(model.predict(X[ntr:]) - y[ntr:])))
    cf = X[:, 3].astype(np.float64)
    A = np.stack([np.ones(ntr), cf[:ntr]], 1)
    coef, *_ = np.linalg.lstsq(A, y[:ntr], rcond=None)
    mae_cf = float(np.mean(np.abs(coef[0] + coef[1] * cf[ntr:] - y[ntr:])))
    train_s = time.perf_counter() - t0

    stream = batch_systems(count, first_seed=300000, n_range=(12, 30), k_range=(4, 10))
    sb = bd.Batch()
    for s in stream:
        sb.add(s.A)
    sb.prepare()
    pred = np.exp2(model.predict(sb.features()))
    arrivals = poisson_arrivals(rate, count, 7)
    res = {}
    for label, order, costs in [("fifo", 0, None), ("cost_model_order", 1, pred)]:
        srv = bd.Server(order=order)
        lat = []
        skipped = 0
        i = 0
        t1 = time.perf_counter()
        while i < count or len(lat) + skipped < count:
            now = time.perf_counter() - t1
            if i < count and now >= arrivals[i]:
                try:
                    srv.submit(stream[i].A, seed=0, predicted_cost=float(costs[i]) if costs is not None else 0.0)
                except bd.BinodegError:
                    skipped += 1
                i += 1
                continue
            got = srv.poll()
            if got:
                lat.append(got[2])
            else:
                time.sleep(0.0001)
        el = time.perf_counter() - t1
        srv.stop()
        lat = np.array(lat)
        res[label] = dict(degrees_per_s=len(lat) / el, p50_ms=float(np.percentile(lat, 50)),
                          p99_ms=float(np.percentile(lat, 99)), mean_ms=float(lat.mean()), served=len(lat),
                          not_served_128bit=skipped)
    res.update(rate_per_s=rate, requests=count, cost_model=dict(
        train_runs=int(keep.sum()), mae_log2_runtime_model=mae_model, mae_log2_runtime_closed_form=mae_cf,
        train_and_data_s=train_s))
    return res


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    import paper_1501_02237_gb300 as bd
    from workloads import config_system

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    bd.set_stream(stream)
    if args.pivot_only:
        print(json.dumps(pivot_section(bd, systems=(args.pivot_only,), seed=args.seed)), flush=True)
        return
    if args.mixed_only:
        print(json.dumps(mixed_section(bd, name=args.mixed_only, seed=args.seed, runs=1, cpu_seconds=0.0)), flush=True)
        return

    s = config_system(args.workload)
    red = bd.reduce(s.A)
    P = red["points"]
    N, k = P.shape
    subsets = math.comb(N, k + 1)
    plan = bd.Plan(P)
    info = plan.info()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    seed = args.seed  # every rank lifts alike: with N GPUs each enumerates 1/N of the work list
    if world > 1:
        from paper_1501_02237_gb300 import shard

    # correctness of the timed configuration before timing it
    if world > 1:
        with torch.cuda.stream(stream):
            res = shard.volume(plan, seed=seed, stream=stream)
    else:
        res = plan.volume(seed=seed)
    expect_nvol = res["nvol"]

    def step(i, timing=None):
        # one exact volume pass; a tie (none expected) re-lifts.  Device time is taken with CUDA
        # events on the launching stream around memset + enumeration kernel + 48-byte result copy;
        # with N GPUs the step is this rank's shard plus the all-reduce of the partial sums.
        attempt, ms = 0, 0.0
        while True:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                a.record(stream)
                if world > 1:
                    plan.launch(seed=seed + i, attempt=attempt, stream=stream, shard=rank, shards=world)
                    out = shard.combine(plan.read())
                else:
                    plan.launch(seed=seed + i, attempt=attempt, stream=stream)
                b.record(stream)
                if world == 1:
                    out = plan.read()
            b.synchronize()
            ms += a.elapsed_time(b)
            if out["ties"] == 0:
                return out, attempt + 1, ms
            attempt += 1

    for i in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    total_ms, launches, kernel_ms = 0.0, 0, []
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        out, nl, ms = step(args.warmup + i)
        kernel_ms.append(ms)
        launches += nl
        assert out["nvol"] == expect_nvol, "volume changed between liftings"
    torch.cuda.synchronize()
    total_ms = sum(kernel_ms)
    clk = clocks.stop()
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = subsets * args.steps / (total_ms / 1e3)  # one volume per step across all ranks

    # end to end through the public calls from a host matrix (pinned copy of A each step): with
    # one GPU bd_degree(A); with N, the host reduction, a plan and the sharded volume
    A_host = torch.from_numpy(np.ascontiguousarray(s.A)).pin_memory()
    e2e_ms = []
    for i in range(max(3, args.steps // 5)):
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        if world > 1:
            p_i = bd.Plan(bd.reduce(A_host.numpy())["points"])
            with torch.cuda.stream(stream):
                r = shard.volume(p_i, seed=seed + i, stream=stream)
            p_i.close()
        else:
            r = bd.degree(A_host.numpy(), seed=seed + i)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        assert r["nvol"] == expect_nvol
    e2e_ms = e2e_ms[1:]
    if world > 1:
        t = torch.tensor([statistics.mean(e2e_ms)], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_ms = [float(t.item())]
    e2e_value = subsets / (statistics.mean(e2e_ms) / 1e3)
    h2d = N * k * 8  # the reduced points; the work list stays on the device after the first call
    d2h = 48

    # roofline: the algorithmic int64 work of the plain per-subset method (differences,
    # Bareiss on the k x (k+1) lifted system with 2 multiplies, 1 subtract, 1 exact division
    # per entry, back substitution) per subset, against the INT32 lane peak of the GPU
    E = sum((k - p) * (k + 1 - p) for p in range(1, k))
    ops_per_subset = k * (k + 1) + 4 * E + k * k
    props = torch.cuda.get_device_properties(dev)
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak_int32 = props.multi_processor_count * 128 * sm_max * 1e6
    achieved = ops_per_subset * (subsets / world) / (ms_per_step / 1e3)  # one GPU's shard
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms_per_step, higher_is_better=True, scaling="strong", vs_baseline=None, dtype="int64",
                data="synthetic",
                config=dict(workload=args.workload, n=s.n, m=s.m, k=k, points=N, subsets_per_step=subsets,
                            l2="flushed before each timed step (256 MB device write)", items=info["items"],
                            blocks=info["blocks"], warps_per_block=info["warps_per_block"],
                            int_path="int128" if info["int128"] else "int64", max_abs_coord=red["max_abs_coord"]),
                degrees_per_s=args.steps / (total_ms / 1e3), nvol=int(expect_nvol), cells=res["cells"],
                clocks=clk, gpu_launches=launches,
                e2e=dict(value=e2e_value, unit=UNIT, h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h,
                         ms_per_step=statistics.mean(e2e_ms), call="bd_degree(A) from host memory"),
                roofline=dict(bound="alu", achieved=achieved / 1e9, peak=peak_int32 / 1e9, unit="Gop/s",
                              frac=achieved / peak_int32,
                              traffic=(TRAFFIC.get(args.workload)
                                       if sources_sha256() == TRAFFIC["sources_sha256"] else None),
                              traffic_unit="bytes per launch (DRAM read + write, ncu)",
                              ops_per_subset=ops_per_subset,
                              note="int64 ops of the plain per-subset method vs INT32 lane peak "
                                   f"({props.multi_processor_count} SMs x 128 lanes x {sm_max:.0f} MHz)"))
    if rank == 0 and world == 1 and not args.no_batch_serve:
        line["batch"] = batch_section(bd)
        line["serve"] = serve_section(bd)
        line["start_solutions"] = start_section(bd, P, seed=seed)
        mx = mixed_section(bd, seed=seed)
        # the same convention for a tuple of pairs: the k x (k+1) lifted system of the pair rows
        # (differences, Bareiss, back substitution) per tuple, against the same INT32 lane peak
        km = mx["k"]
        Em = sum((km - p) * (km + 1 - p) for p in range(1, km))
        ops_t = km * (km + 1) + 4 * Em + km * km
        ach = ops_t * mx["tuples_per_s"]
        mx["roofline"] = dict(bound="alu", achieved=ach / 1e9, peak=peak_int32 / 1e9, unit="Gop/s",
                              frac=ach / peak_int32, ops_per_tuple=ops_t)
        line["mixed_volume"] = mx
        line["pivoting"] = pivot_section(bd, seed=seed)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(s, subsets)
        line["cpu_native"] = cpu_native(bd, P, int(expect_nvol))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
