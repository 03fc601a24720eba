"""Benchmark: exact (k+1)-subsets tested per second (and degrees per second) on one GB300.

Workload (the headline): the heavy quiver system, n = 32 variables and 22 binomials whose
monomials are products of 2-3 distinct variables (0/1 exponents), seed 0; rank 22, so k = 10:
33 kernel points in Z^10 and C(33, 11) = 193,536,720 subsets per degree.  A step is one
complete exact volume pass (lift, enumerate every subset with the exact lower-facet test,
reduce, read the result and re-lift on a tie) with the reduced points resident in device
memory.  The e2e figure runs the public call bd_degree(A) from a host matrix per step (Smith
form, kernel basis, device copies, enumeration, result read).  L2 is flushed (a 256 MB write)
before every timed step.  The n = 24, k = 8 system (2,042,975 subsets) is timed the same way
in its own section of the line.

The roofline's denominator is measured in the same process: bd_issue_peak runs full-occupancy
streams of LOP3, IMAD and FFMA instructions and reports lane operations per second with the SM
clock it saw.

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

WORKLOAD = "heavy_quiver_n32_k10"
SECONDARY = "single_n24_k8"

# Counters of one enumeration launch from an ncu capture of the kernel built from exactly these
# sources: DRAM bytes (read + write), warp instructions issued and the issue-active fraction.
# Reported only while the library sources still hash to the captured version, null otherwise.
PROFILE = {
    "sources_sha256": "7b024fb2ac13dff5495cc8ff5b59430c6ac43f6afd6fd438fe6d49c72eb72965",
    # k_enumerate<int32, int64, 5> (the 5-D stage), 388,070 items
    "heavy_quiver_n32_k10": dict(warp_inst=2408999333, lanes_per_inst=25.77, issue_active=0.5944,
                                 traffic=6700544 + 42496),
    # k_enumerate<int32, int64, 4> (the 4-D stage), 53,196 items
    "single_n24_k8": dict(warp_inst=130995030, lanes_per_inst=23.46, issue_active=0.5992,
                          traffic=1161472 + 19200),
}


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


def profile_of(workload: str):
    """The committed ncu counters of this workload's launch, if the sources still match."""
    if PROFILE.get(workload) is None or sources_sha256() != PROFILE["sources_sha256"]:
        return None
    return PROFILE[workload]


def ops_per_subset(k: int) -> int:
    """Algorithmic int64 operations of the plain per-subset method (Sec. 4): k(k+1) differences,
    Bareiss on the k x (k+1) lifted system (2 multiplies, 1 subtract, 1 exact division per
    entry) and the k^2 back substitution; the scan of the other points is not counted."""
    E = sum((k - p) * (k + 1 - p) for p in range(1, k))
    return k * (k + 1) + 4 * E + k * k


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


def workload_config(name: str, s, points: int, k: int) -> dict:
    """The config object of the line: the same dict in both arms."""
    return dict(workload=name, n=s.n, m=s.m, k=k, points=points, subsets_per_step=math.comb(points, k + 1),
                l2="flushed before each timed step (256 MB device write)")


def host_info() -> dict:
    cpu = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    cpu = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        aff = len(os.sched_getaffinity(0))
    except AttributeError:
        aff = os.cpu_count() or 1
    return dict(cpu_count=os.cpu_count(), affinity=aff, cpu=cpu)


def run_reference(args, rank, world):
    """The oracle (plain exact Python) timed on this host's cores on the same workload: each step
    is one full exact degree of the workload on one core."""
    if rank != 0:
        return
    from workloads import config_system

    s = config_system(args.workload)
    r = oracle_step(s)
    N, k = s.n + 1, r.dim
    subsets = math.comb(N, k + 1)
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
                config=workload_config(args.workload, s, N, k),
                degrees_per_s=args.steps / dt, degree=r.degree,
                cpu_baseline=dict(value=value, unit=UNIT, cores=1, kind="oracle", host=host_info(),
                                  sample=f"{args.steps} full exact degrees of the workload, single thread"),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def cpu_baseline(system, subsets, budget_s=15.0):
    """The oracle on one host core: whole exact degrees of the workload for about budget_s."""
    t0 = time.perf_counter()
    n = 0
    while True:
        oracle_step(system)
        n += 1
        if time.perf_counter() - t0 > budget_s or n >= 30:
            break
    dt = time.perf_counter() - t0
    return dict(value=subsets * n / dt, unit=UNIT, cores=1, kind="oracle", host=host_info(),
                sample=f"{n} full exact degrees of the workload ({dt:.1f} s, single thread)")


def _oracle_system(args):
    """Pool worker: the oracle's degree of one batch system; (index, degree, subsets)."""
    i, A = args
    from oracle.degree import degree as oracle_degree

    r = oracle_degree(A)
    n = len(A)
    return i, r.degree, (math.comb(n + 1, r.dim + 1) if r.dim > 0 else 0)


def cpu_oracle_pool(systems, budget_s=20.0):
    """The oracle on every host core (a spawn pool, one system per task) over the uneven batch,
    in batch order, for about budget_s: systems/s and subsets/s of what it finished."""
    import multiprocessing as mp

    info = host_info()
    procs = info["affinity"]
    ctx = mp.get_context("spawn")
    done, subsets, degs = 0, 0, {}
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_system, [(i, systems[i].A.tolist()) for i in range(procs)])  # workers up
        t0 = time.perf_counter()
        last = t0
        for i, d, sub in pool.imap_unordered(_oracle_system, [(i, s.A.tolist()) for i, s in enumerate(systems)]):
            done += 1
            subsets += sub
            degs[i] = d
            last = time.perf_counter()
            if last - t0 > budget_s:
                break
        pool.terminate()
    dt = last - t0
    return dict(value=done / dt, unit="systems/s", subsets_per_s=subsets / dt, cores=procs, kind="oracle",
                host=info, sample=f"{done} of {len(systems)} batch systems (batch order) by the oracle in "
                                  f"{dt:.1f} s on {procs} processes"), degs


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


def train_cost_model(bd, train_count=20000):
    """The cost model of the batch and serving sections: 20,000 method-generated runs (n ~ U[12,30],
    k ~ U[4,10]) enumerated in one batch, their SM cycles as targets; 80 % train, 20 % held out."""
    import numpy as np

    from workloads import batch_systems

    t0 = time.perf_counter()
    train = batch_systems(train_count, first_seed=200000, n_range=(12, 30), k_range=(4, 10))
    b = bd.Batch()
    for s in train:
        b.add(s.A)
    b.prepare()
    b.run(mode=0)
    cyc = np.array([r["cycles"] for r in b.results()], dtype=np.float64)
    X = b.features()
    b.close()
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
    return model, dict(train_runs=int(keep.sum()), mae_log2_runtime_model=mae_model,
                       mae_log2_runtime_closed_form=mae_cf, train_and_data_s=time.perf_counter() - t0)


def batch_section(bd, model, pool_cpu=None, seed=0):
    """The batched form against one launch per system on the uneven 4096-system workload
    (n ~ U[12,28], k ~ U[4,9], exponents in {0,1,2}, seeds 0..4095), exact agreement checked:
    batched with the closed-form cost, batched with the learned cost model's predictions sizing
    and ordering the work items, the latter captured in a CUDA graph, and per system."""
    import numpy as np

    from workloads import batch_systems

    systems = batch_systems(4096)
    b = bd.Batch()
    for s in systems:
        b.add(s.A, seed=seed)
    b.prepare()
    pred = np.exp2(model.predict(b.features())).astype(np.float32)
    out = {}
    ref = None
    arms = [("batched", dict(mode=0, autotune=True)), ("batched", dict(mode=0, autotune=True)),
            ("batched_mlp", dict(mode=0, autotune=True, cost=pred)),
            ("batched_mlp", dict(mode=0, autotune=True, cost=pred)),
            ("batched_mlp_graph", dict(mode=0, autotune=True, use_graph=True, cost=pred)),
            ("per_system", dict(mode=1))]
    for label, kw in arms:
        st = b.run(**kw)
        res = [(r["degree"], r["nvol"]) for r in b.results()]
        ref = ref or res
        assert res == ref, "batch modes disagree"
        out[label] = dict(systems_per_s=len(systems) / (st["wall_ms"] / 1e3), wall_ms=st["wall_ms"],
                          gpu_ms=st["gpu_ms"], subsets_per_s=st["subsets"] / (st["wall_ms"] / 1e3),
                          launches=st["launches"], warps_per_block=st["warps_per_block"],
                          item_factor=st["item_factor"])
    out["systems"] = len(systems)
    out["subsets"] = int(st["subsets"])
    out["host_reduce_ms"] = st["host_ms"]
    out["speedup_batched_mlp_vs_per_system"] = out["batched_mlp"]["systems_per_s"] / out["per_system"]["systems_per_s"]
    out["speedup_batched_mlp_vs_closed_form"] = out["batched_mlp"]["systems_per_s"] / out["batched"]["systems_per_s"]
    if pool_cpu is not None:
        line, degs = pool_cpu
        line["exact_match"] = all(ref[i][0] == d for i, d in degs.items())
        line["checked"] = len(degs)
        out["cpu_baseline_pool"] = line
    b.close()
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


def serve_stream(bd, stream, arrivals, order, costs):
    """Submit stream[i] at arrivals[i] seconds (this thread) while a second thread polls the
    finished degrees; returns (latencies ms, elapsed s, server stats, degrees by ticket)."""
    srv = bd.Server(order=order)
    lat, degs = [], {}
    count = len(stream)
    stop = threading.Event()

    def poller():
        while not stop.is_set() or len(lat) < count:
            got = srv.poll(wait_ms=20)
            if got:
                degs[got[0]] = got[1]["degree"]
                lat.append(got[2])

    th = threading.Thread(target=poller, daemon=True)
    t1 = time.perf_counter()
    th.start()
    tickets = []
    for i in range(count):
        d = arrivals[i] - (time.perf_counter() - t1)
        if d > 0:
            time.sleep(d)
        tickets.append(srv.submit(stream[i].A, seed=0, predicted_cost=float(costs[i]) if costs is not None else 0.0))
    stop.set()
    th.join()
    el = time.perf_counter() - t1
    st = srv.stats()
    srv.stop()
    return lat, el, st, [degs[t] for t in tickets]


def serve_section(bd, model, cm, rates=(200.0, 2000.0, 5000.0), count=2000):
    """A Poisson stream served with continuous batching (n ~ U[12,30], k ~ U[4,10]) at several
    arrival rates, up to ones that keep the GPU busy: p50/p99 latency and degrees/s for FIFO
    admission and for smallest-predicted-cost-first admission by the closed-form bound and by
    the learned model."""
    import numpy as np

    from workloads import batch_systems, poisson_arrivals

    stream = batch_systems(count, first_seed=300000, n_range=(12, 30), k_range=(4, 10))
    sb = bd.Batch()
    for s in stream:
        sb.add(s.A)
    sb.prepare()
    pred = np.exp2(model.predict(sb.features()))
    sb.run(mode=0)
    ref = [r["degree"] for r in sb.results()]
    sb.close()
    res = dict(requests=count, cost_model=cm)
    for rate in rates:
        arrivals = poisson_arrivals(rate, count, 7)
        per = {}
        # shortest first by the closed-form bound (predicted_cost 0) isolates what the network adds
        for label, order, costs in [("fifo", 0, None), ("closed_form_order", 1, None), ("cost_model_order", 1, pred)]:
            lat, el, st, degs = serve_stream(bd, stream, arrivals, order, costs)
            lat = np.array(lat)
            per[label] = dict(degrees_per_s=len(lat) / el, p50_ms=float(np.percentile(lat, 50)),
                              p99_ms=float(np.percentile(lat, 99)), mean_ms=float(lat.mean()), served=len(lat),
                              exact_match=degs == ref, peak_resident=st["peak_resident"],
                              side_route=st["routed"], kernel_launches=st["launches"])
        res[f"rate_{int(rate)}"] = per
    return res


ISSUE_KINDS = ("lop3", "imad", "lop3_imad", "ffma", "lop3_ffma")
INT_KINDS = ("lop3", "imad", "lop3_imad")


def issue_peaks(bd, reps=3, iters=4096):
    """Full-occupancy instruction streams (bd_issue_peak), best of reps each, after one short
    warm-up launch: lane operations/s, per SM per cycle, and the SM clock each run saw."""
    out = {}
    for kind in ISSUE_KINDS:
        bd.issue_peak(kind, iters=64)
        best = max((bd.issue_peak(kind, iters=iters) for _ in range(reps)), key=lambda r: r["lane_ops_per_s"])
        out[kind] = dict(lane_ops_per_s=best["lane_ops_per_s"], per_sm_per_clk=best["lane_ops_per_sm_clk"],
                         sm_mhz=best["sm_mhz"], ms=best["ms"])
    best_int = max(INT_KINDS, key=lambda k: out[k]["lane_ops_per_s"])
    return out, best_int


def timed_volume(plan, subsets, steps, warmup, stream, flush, seed, world, rank, clocks=None):
    """warmup + steps exact volume passes of a resident plan; each step flushes L2 first and is
    timed on the launching stream with CUDA events (memset + enumeration + result copy; with N
    GPUs this rank's shard plus the all-reduce).  A tie (none expected) re-lifts."""
    import torch

    if world > 1:
        from paper_1501_02237_gb300 import shard

    def step(i):
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

    for i in range(warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    if clocks:
        clocks.start()
    launches, kernel_ms, nvols = 0, [], set()
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        out, nl, ms = step(warmup + i)
        kernel_ms.append(ms)
        launches += nl
        nvols.add(out["nvol"])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if clocks else None
    total_ms = sum(kernel_ms)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    return dict(total_ms=total_ms, ms_per_step=total_ms / steps, launches=launches, nvols=nvols,
                value=subsets * steps / (total_ms / 1e3), clocks=clk, best_ms=min(kernel_ms))


def roofline(k, subsets_per_launch, launch_ms, peak, workload, clocks_note):
    ops = ops_per_subset(k)
    achieved = ops * subsets_per_launch / (launch_ms / 1e3)
    prof = profile_of(workload)
    r = dict(bound="alu", achieved=achieved / 1e9, peak=peak["lane_ops_per_s"] / 1e9, unit="Gop/s",
             frac=achieved / peak["lane_ops_per_s"], traffic=prof["traffic"] if prof else None,
             traffic_unit="bytes per launch (DRAM read + write, ncu)", ops_per_subset=ops,
             peak_kind=peak["kind"], peak_sm_mhz=peak["sm_mhz"],
             note="algorithmic int64 ops of the plain per-subset method (no scan) per second, against the "
                  f"measured {peak['kind']} issue peak (bd_issue_peak, {peak['per_sm_per_clk']:.1f} lane ops per SM "
                  f"per cycle at {peak['sm_mhz']:.0f} MHz, of measured); the walk does less than the plain method "
                  "per subset (prefix eliminations shared by a subtree, singular subsets rejected by one "
                  "single-precision determinant), so frac can exceed 1; the issue view (ncu lane instructions "
                  f"per second against the same peak) is `ncu.lane_inst_frac_of_peak`; {clocks_note}")
    if prof:
        # the issue view: instructions the kernel issued (ncu) per subset and against the peak
        lane_inst = prof["warp_inst"] * prof["lanes_per_inst"]
        r["ncu"] = dict(warp_inst_per_launch=prof["warp_inst"], lanes_per_warp_inst=prof["lanes_per_inst"],
                        issue_active=prof["issue_active"], warp_inst_per_subset=prof["warp_inst"] / subsets_per_launch,
                        lane_inst_frac_of_peak=lane_inst / (launch_ms / 1e3) / peak["lane_ops_per_s"],
                        useful_ops_per_lane_inst=ops * subsets_per_launch / lane_inst)
    return r


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    import paper_1501_02237_gb300 as bd
    from workloads import batch_systems, config_system

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    # the oracle's process pool is spawned before the first GPU call
    pool_cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not (args.pivot_only or args.mixed_only):
        pool_cpu = cpu_oracle_pool(batch_systems(4096))
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

    # the denominator first (a few ms of full-occupancy instruction streams)
    peaks, best_int = issue_peaks(bd)
    peak = dict(peaks[best_int], kind=best_int)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    seed = args.seed  # every rank lifts alike: with N GPUs each enumerates 1/N of the work list

    def prepare(name):
        s = config_system(name)
        red = bd.reduce(s.A)
        P = red["points"]
        plan = bd.Plan(P)
        # correctness of the timed configuration before timing it
        if world > 1:
            from paper_1501_02237_gb300 import shard

            with torch.cuda.stream(stream):
                res = shard.volume(plan, seed=seed, stream=stream)
        else:
            res = plan.volume(seed=seed)
        return s, red, P, plan, res

    s, red, P, plan, res = prepare(args.workload)
    N, k = P.shape
    subsets = math.comb(N, k + 1)
    info = plan.info()
    expect_nvol = res["nvol"]
    t = timed_volume(plan, subsets, args.steps, args.warmup, stream, flush, seed, world, rank,
                     clocks=ClockSampler(local))
    assert t["nvols"] == {expect_nvol}, "volume changed between liftings"
    clk = t["clocks"]
    value = t["value"]

    # end to end through the public calls from a host matrix (pinned copy of A each step): with
    # one GPU bd_degree(A); with N, the host reduction, a plan and the sharded volume
    A_host = torch.from_numpy(np.ascontiguousarray(s.A)).pin_memory()
    e2e_ms = []
    for i in range(max(3, args.steps // 5)):
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        if world > 1:
            from paper_1501_02237_gb300 import shard

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
        tt = torch.tensor([statistics.mean(e2e_ms)], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        e2e_ms = [float(tt.item())]
    e2e_value = subsets / (statistics.mean(e2e_ms) / 1e3)
    h2d = N * k * 8  # the reduced points; the work list stays on the device after the first call
    d2h = 48

    clocks_note = (f"kernel timed at a median {clk['sm_mhz']:.0f} MHz" if clk and clk.get("sm_mhz") else "no clock samples")
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=t["ms_per_step"], higher_is_better=True, scaling="strong", vs_baseline=None,
                dtype="int64", data="synthetic", config=workload_config(args.workload, s, N, k),
                launch=dict(items=info["items"], blocks=info["blocks"], warps_per_block=info["warps_per_block"],
                            int_path="int128" if info["int128"] else "int64", max_abs_coord=red["max_abs_coord"]),
                degrees_per_s=args.steps / (t["total_ms"] / 1e3), nvol=int(expect_nvol), cells=res["cells"],
                singular=res["singular"], full_dimensional=subsets - res["singular"],
                clocks=clk, gpu_launches=t["launches"],
                e2e=dict(value=e2e_value, unit=UNIT, h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h,
                         ms_per_step=statistics.mean(e2e_ms), call="bd_degree(A) from host memory"),
                roofline=roofline(k, subsets / world, t["ms_per_step"], peak, args.workload, clocks_note),
                issue_peaks=dict(peaks, note="bd_issue_peak: 152-SM full-occupancy streams, lane ops/s"))
    if rank == 0 and world == 1 and not args.no_batch_serve:
        # the n = 24, k = 8 system, timed the same way
        s2, red2, P2, plan2, res2 = prepare(SECONDARY)
        N2, k2 = P2.shape
        sub2 = math.comb(N2, k2 + 1)
        t2 = timed_volume(plan2, sub2, args.steps, args.warmup, stream, flush, seed, 1, 0)
        assert t2["nvols"] == {res2["nvol"]}
        line[SECONDARY] = dict(config=workload_config(SECONDARY, s2, N2, k2), value=t2["value"], unit=UNIT,
                               ms_per_step=t2["ms_per_step"], degrees_per_s=args.steps / (t2["total_ms"] / 1e3),
                               nvol=int(res2["nvol"]), singular=res2["singular"], full_dimensional=sub2 - res2["singular"],
                               roofline=roofline(k2, sub2, t2["ms_per_step"], peak, SECONDARY, ""))
        plan2.close()
        model, cm = train_cost_model(bd)
        line["batch"] = batch_section(bd, model, pool_cpu)
        line["serve"] = serve_section(bd, model, cm)
        line["start_solutions"] = start_section(bd, P2, seed=seed)
        mx = mixed_section(bd, seed=seed)
        # the same convention for a tuple of pairs: the k x (k+1) lifted system of the pair rows
        # (differences, Bareiss, back substitution) per tuple, against the same measured peak
        ops_t = ops_per_subset(mx["k"])
        ach = ops_t * mx["tuples_per_s"]
        mx["roofline"] = dict(bound="alu", achieved=ach / 1e9, peak=peak["lane_ops_per_s"] / 1e9, unit="Gop/s",
                              frac=ach / peak["lane_ops_per_s"], ops_per_tuple=ops_t, peak_kind=peak["kind"])
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
