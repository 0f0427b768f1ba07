"""Benchmark: batched Roaring set operations on one GB300 (or N replicas).

Workload (the batched configuration): a pool of 4096 seeded bitmaps over
[0, 2^32), cardinalities log-uniform 10..1e7, classes 40% uniform-sparse /
30% dense-clustered / 30% runs; 65,536 query pairs (a != b) with ops AND 40% /
OR 30% / ANDNOT 15% / XOR 15%, materialised as canonical Roaring bitmaps,
plus a count-only Jaccard batch over the same pairs.

One step = one run of both batches (two persistent launches replayed from
CUDA graphs, plus compaction).  value = sum over pairs of (|A| + |B|) per
step / device time of the step, in Gints/s (the paper's per-input-value
normalisation inverted); pairs are counted once per step although the Jaccard
batch reads them again.  The pool (3+ GB) and the outputs (tens of GB) are far
larger than L2, so no flush is needed between steps.

--impl reference times the CPU oracle (test infrastructure, plain C) on the
host cores over a bounded sample of the same pairs.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_PAIRS = 65536
# the workload both arms name in their JSON line
WORKLOAD = ("batched: 4096-bitmap pool over [0,2^32), c log-uniform 10..1e7, 40/30/30 sparse/dense/runs; "
            "65,536 pairs AND/OR/ANDNOT/XOR 40/30/15/15 materialised + Jaccard count batch")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_sha256():
    """SHA-256 of the device code of the pairwise kernels without comment-only
    lines: csrc/rb_pairs.cu and csrc/rb_internal.h up to their "host side"
    marker line, and csrc/rb_device.cuh, in that order.  Host-only edits
    leave it unchanged."""
    import hashlib
    h = hashlib.sha256()
    for f in ("rb_pairs.cu", "rb_device.cuh", "rb_internal.h"):
        with open(os.path.join(ROOT, "paper_1709_07821_gb300", "csrc", f)) as fh:
            for line in fh:
                t = line.strip()
                if t.startswith("//") and t.endswith("host side"):
                    break
                if not t.startswith("//"):
                    h.update(line.encode())
    return h.hexdigest()


def kernel_traffic(kernel, alg_bytes):
    """DRAM bytes of one launch of `kernel` in the materialising batch: the
    dram/algorithmic byte ratio of its ncu capture summarised in profiles/
    (a file named <kernel>_batched_*.md with "traffic_ratio:" and
    "source_sha256:" lines) times this launch's algorithmic bytes, or None
    when the kernel sources differ from those the capture was taken from (or
    there is no capture)."""
    import glob
    import re
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{kernel}_batched_*.md"))):
        try:
            txt = open(path).read()
            ratio = float(re.search(r"^traffic_ratio: ([0-9.]+)", txt, re.M).group(1))
            want = re.search(r"^source_sha256: ([0-9a-f]{64})", txt, re.M).group(1)
        except Exception:
            continue
        if kernel_source_sha256() == want:
            return ratio * alg_bytes
    return None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _reduce(value, op):
    """value reduced over the ranks of the default process group (as is
    when there is none); tensors live on the backend's device."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    dist.barrier()
    return float(t.item())


def reduce_max(value):
    """Slowest rank's value: the whole job ends when its last replica does."""
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.MAX)


def reduce_sum(value):
    """Sum over ranks: replicas draw different seeded workloads, so the
    job's units are the sum of every rank's units."""
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.SUM)


def job_value(units_total, max_ms_per_step):
    """Whole-job Gints/s: all ranks' input values per step over the slowest
    rank's step time."""
    return units_total / (max_ms_per_step / 1e3) / 1e9


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index: int):
        import tempfile
        # raw samples go to a scratch file (RB_BENCH_CLOCKS_DIR if set); the
        # JSON line carries their summary
        d = os.environ.get("RB_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        os.makedirs(d, exist_ok=True)
        self.path = os.path.join(d, f"rb_bench_clocks_gpu{gpu_index}_{os.getpid()}.csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(seed_offset=0, args=None):
    import workloads as W
    t0 = time.time()
    spec = W.SPECS["batched"]
    if args is not None and (args.pool or args.log10_hi):
        spec = W.scaled(spec, n_bitmaps=args.pool or None, log10_hi=args.log10_hi or None)
    pool = W.make_pool(spec)
    n_pairs = args.pairs if args is not None and args.pairs else N_PAIRS
    ops, a, b = W.pairs(4 + seed_offset, n_pairs, pool.n)
    log(f"generated pool of {pool.n} bitmaps ({int(pool.sizes().sum()):,} values) in {time.time() - t0:.1f}s")
    return pool, ops, a, b


class OracleSample:
    """The CPU oracle (as it stands, test infrastructure) over a bounded
    sample of the pairs: its bitmaps are built once (untimed), then time()
    runs the materialised op plus the Jaccard counts of each pair on the host
    cores, pairs spread over a thread pool (ctypes releases the GIL)."""

    def __init__(self, pool, ops, a, b, sample_values=2e10, threads=None):
        import oracle
        oracle.build()
        self.threads = threads or os.cpu_count() or 1
        self.sizes = pool.sizes()
        self.ops, self.a, self.b, self.n_total = ops, a, b, len(ops)
        self.sample, need, est = [], set(), 0
        for i in range(len(ops)):
            self.sample.append(i)
            need.update([int(a[i]), int(b[i])])
            est += int(self.sizes[a[i]]) + int(self.sizes[b[i]])
            if est > sample_values or len(self.sample) >= 16384:
                break
        need = sorted(need)
        with cf.ThreadPoolExecutor(self.threads) as ex:
            self.built = dict(zip(need, ex.map(lambda j: oracle.Bitmap.from_sorted(pool.values(j)), need)))

    def _one(self, i):
        A, B = self.built[int(self.a[i])], self.built[int(self.b[i])]
        r = A.op(int(self.ops[i]), B)
        r.close()
        A.jaccard(B)
        return int(self.sizes[self.a[i]]) + int(self.sizes[self.b[i]])

    def time(self, budget_s, threads=None):
        threads = threads or self.threads
        done_vals, done_pairs = 0, 0
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(threads) as ex:
            futs = [ex.submit(self._one, i) for i in self.sample]
            for f in futs:
                done_vals += f.result()
                done_pairs += 1
                if time.perf_counter() - t0 > budget_s:
                    for g in futs:
                        g.cancel()
                    break
        dt = time.perf_counter() - t0
        return {"value": done_vals / dt / 1e9, "unit": "Gints/s", "cores": threads, "kind": "oracle",
                "sample": f"first {done_pairs} of the {self.n_total} pairs (materialised op + Jaccard each), "
                          f"{done_vals:,} input values, {dt:.1f}s on {threads} host threads"}

    def close(self):
        for x in self.built.values():
            x.close()


def cpu_oracle_leg(pool, ops, a, b, budget_s=15.0):
    """The oracle on every host core (the reported baseline) and on one core
    (the paper's own figures are single-threaded), same pairs."""
    s = OracleSample(pool, ops, a, b)
    try:
        res = s.time(budget_s)
        one = s.time(max(3.0, budget_s / 3), threads=1)
        res["one_core"] = {"value": one["value"], "unit": one["unit"], "cores": 1, "sample": one["sample"]}
        res["cpu_model"] = cpu_model()
        return res
    finally:
        s.close()


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine() or "unknown"


def time_tasks(tasks, threads, budget_s):
    """Run tasks (callables returning input values processed) in order on
    `threads` host threads until all are done or budget_s has passed;
    returns (values per second, tasks done, seconds)."""
    done_vals, done = 0, 0
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(threads) as ex:
        futs = [ex.submit(t) for t in tasks]
        for f in futs:
            done_vals += f.result()
            done += 1
            if time.perf_counter() - t0 > budget_s:
                for g in futs:
                    g.cancel()
                break
    dt = time.perf_counter() - t0
    return done_vals / dt, done, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    pool, ops, a, b = make_workload(args=args)
    sample = OracleSample(pool, ops, a, b)
    steps = []
    res = None
    for s in range(args.warmup + args.steps):
        res = sample.time(args.ref_budget)
        if s >= args.warmup:
            steps.append(res["value"])
    sample.close()
    value = statistics.median(steps)
    line = {"impl": "reference", "metric": "batched Roaring AND/OR Gints/s", "value": value, "unit": "Gints/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u16/u64 integer", "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD, "global_batch": N_PAIRS},
            "cpu_baseline": dict(res, value=value),
            "e2e": {"value": value, "unit": "Gints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import paper_1709_07821_gb300 as rb

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rb.build()
    rb.lib()

    pool, ops, a, b = make_workload(seed_offset=rank, args=args)
    n_pairs = len(ops)
    if args.schedule:
        rb.set_schedule(*[int(x) for x in args.schedule.split(",")])
    sizes = pool.sizes().astype(np.float64)
    units = float((sizes[a] + sizes[b]).sum())      # input values per step (pairs counted once)

    t0 = time.time()
    G = []
    for i in range(pool.n):
        G.append(rb.Bitmap.from_sorted(pool.values(i)))
    torch.cuda.synchronize()
    pool_bytes = sum(g.payload_bytes() + 10 * g.n_containers for g in G)
    log(f"rank {rank}: built {len(G)} device bitmaps ({pool_bytes / 1e9:.2f} GB) in {time.time() - t0:.1f}s")

    if args.subsets_only:
        # the bitset-dominated legs alone (profiling k_heavy)
        names = tuple(args.subset.split(",")) if args.subset else None
        print(json.dumps({"bitset_and_or": bitset_subset_legs(rb, G, pool, sizes, only=names)}))
        return 0

    if args.serving_only:
        # the serving leg alone (profiling the multi-way kernels)
        rates = tuple(float(x) for x in args.serving_rates.split(","))
        print(json.dumps({"serving": serving_on_index(rb, args, rates=rates, max_queries=args.serving_queries)}))
        return 0

    plan_m = rb.Plan(G, ops, a, b)
    jflags = np.full(n_pairs, rb.Q_COUNT_ONLY, np.uint32)
    plan_j = rb.Plan(G, np.zeros(n_pairs, np.uint32), a, b, jflags)

    sched_info = tuned_schedule(rb, plan_m, args)

    stream = torch.cuda.current_stream()

    def step():
        # both batches are enqueued before either is collected, so the device
        # runs them back to back while the host turns the first one's results
        # into handles; results stay raw handles, released in one call
        plan_m.launch()
        plan_j.launch()
        outs, counts = plan_m.collect(raw=True)
        _, inter = plan_j.collect(want_bitmaps=False)
        return outs, counts, inter

    for _ in range(args.warmup):
        outs, _, _ = step()
        plan_m.free_raw(outs)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = Clocks(local) if rank == 0 else None
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kms, jst, alg, outb, step_ms = [], [], [], [], []
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        outs, counts, inter = step()
        st = plan_m.stats()
        kms.append(st)
        jst.append(plan_j.stats())
        alg.append(st["alg_bytes"])
        outb.append(st["out_bytes"])
        plan_m.free_raw(outs)
        s1.record(stream)
        s1.synchronize()
        step_ms.append(s0.elapsed_time(s1))
    ev1.record(stream)
    torch.cuda.synchronize()
    total_ms = ev0.elapsed_time(ev1)
    clk = clocks.stop() if clocks else None
    total_ms = reduce_max(total_ms)
    ms_per_step = total_ms / args.steps
    units_total = reduce_sum(units)
    value = job_value(units_total, ms_per_step)

    # end to end through the public API: queries from host memory, counts back
    # to host, one rb_batch_op + rb_batch_jaccard per step (no plan reuse)
    e2e_steps = max(1, min(args.steps, 3))
    t1 = time.perf_counter()
    for _ in range(e2e_steps):
        bms, cnt = rb.batch_op(G, ops, a, b, raw=True)
        jj, ii, uu = rb.batch_jaccard(G, a, b)
        rb.free_handles(bms, n_pairs)
    torch.cuda.synchronize()
    e2e_s = reduce_max((time.perf_counter() - t1) / e2e_steps)

    bitset_legs = {} if args.no_subsets else bitset_subset_legs(rb, G, pool, sizes)
    h2d = 2 * (32 * len(G) + 32 * n_pairs + 8 * (n_pairs + 1) + 128) + 2 * 16 * n_pairs
    d2h = 2 * (40 * n_pairs + 128) + 8 * n_pairs * 4
    e2e = {"value": units_total / e2e_s / 1e9, "unit": "Gints/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "what": "rb_batch_op + rb_batch_jaccard from host query arrays, counts/Jaccard to host, results kept "
                   "on the device as library handles and released in one call; index resident on the device"}

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    peak, peak_kind = measured_peaks()
    mean = lambda xs, k: statistics.mean(x[k] for x in xs)
    kern = {k: (mean(kms, k + "_ms"), mean(kms, k + "_bytes")) for k in ("lean", "small", "heavy")}
    dom = max(kern, key=lambda k: kern[k][0])
    kernel_ms, alg_bytes = kern[dom]
    achieved = alg_bytes / (kernel_ms / 1e3) / 1e9
    stage_ms = sum(v[0] for v in kern.values())
    stage_gbs = sum(v[1] for v in kern.values()) / (stage_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": args.traffic if args.traffic is not None else kernel_traffic("k_" + dom, alg_bytes),
                "kernel": f"k_{dom} (materialising batch)", "kernel_ms": kernel_ms,
                "alg_bytes_per_launch": alg_bytes, "peak_kind": peak_kind,
                "pair_stage": {**{f"{k}_ms": v[0] for k, v in kern.items()}, **{f"{k}_bytes": v[1] for k, v in kern.items()},
                               "achieved_gbs": stage_gbs, "frac": stage_gbs / peak,
                               "deferred_pairs": mean(kms, "deferred"), "small_pairs": mean(kms, "small_pairs")},
                "jaccard_stage": {"lean_ms": mean(jst, "lean_ms"), "small_ms": mean(jst, "small_ms"),
                                  "heavy_ms": mean(jst, "heavy_ms"),
                                  "alg_bytes": statistics.mean(x["lean_bytes"] + x["small_bytes"] + x["heavy_bytes"]
                                                               for x in jst)}}

    # per-pair baseline on the same GPU: rb_apply one pair at a time
    per = per_pair_leg(rb, G, ops, a, b, sizes, n=args.per_pair_sample)
    cfg_legs = None if args.no_configs else config_legs(rb, args)
    serving = None if args.no_serving else serving_on_index(rb, args)
    cpu = cpu_oracle_leg(pool, ops, a, b, budget_s=args.cpu_budget) if not args.no_cpu else None

    line = {"metric": "batched Roaring AND/OR Gints/s", "value": value, "unit": "Gints/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u16/u64 integer", "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD, "global_batch": n_pairs * ws,
                       "pool_bytes": pool_bytes, "units_per_step": units_total,
                       "l2": "inputs larger than L2 (pool and outputs are GBs), no flush",
                       "parallelism": f"replicas x{ws}", "schedule": rb.get_schedule(),
                       "schedule_source": sched_info},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            # per step: k_lean + k_small + k_heavy + k_compact (materialising batch), k_lean + k_small +
            # k_heavy (Jaccard batch)
            "gpu_launches": 7 * args.steps,
            "clocks": clk,
            "step_ms_p50": statistics.median(step_ms), "step_ms_p99": float(np.percentile(step_ms, 99)),
            "per_pair": per, "bitset_and_or": bitset_legs, "configs": cfg_legs, "serving": serving}
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def bitset_subset_legs(rb, G, pool, sizes, n_pairs=16384, reps=5, only=None):
    """Bitset-dominated AND/OR: pairs of dense-clustered pool bitmaps (ops AND
    and OR, 50/50), (1) drawn uniformly, (2) drawn among pairs whose key
    ranges overlap, so that bitset x bitset pairs are actually combined."""
    peak, _ = measured_peaks()
    rng = np.random.default_rng(44)
    dense = np.array([i for i in range(pool.n) if pool.klass(i) == 1])
    kmin = np.array([int(pool.values(i)[0]) >> 16 for i in dense])
    kmax = np.array([int(pool.values(i)[-1]) >> 16 for i in dense])
    order = np.argsort(kmin)
    over = []
    for x in range(len(order)):
        i = order[x]
        for y in range(x + 1, len(order)):
            j = order[y]
            if kmin[j] > kmax[i]:
                break
            over.append((dense[i], dense[j]))
    over = np.array(over, dtype=np.uint32).reshape(-1, 2)
    out = {}
    sets = {"uniform": (rng.choice(dense, n_pairs), rng.choice(dense, n_pairs))}
    if len(over):
        pick = over[rng.choice(len(over), n_pairs)]
        sets["overlapping"] = (pick[:, 0], pick[:, 1])
    for name, (a, b) in sets.items():
        if only and name not in only:
            continue
        keep = a != b
        a, b = a[keep].astype(np.uint32), b[keep].astype(np.uint32)
        ops = rng.integers(0, 2, len(a)).astype(np.uint32)
        plan = rb.Plan(G, ops, a, b)
        stats = []
        for r in range(3 + reps):
            outs, _ = plan.run()
            st = plan.stats()
            for o in outs:
                if o is not None:
                    o.free()
            if r >= 3:
                stats.append(st)
        plan.free()
        hms = statistics.mean(s["heavy_ms"] for s in stats)
        lms = statistics.mean(s["lean_ms"] + s["small_ms"] for s in stats)
        hb = statistics.mean(s["heavy_bytes"] for s in stats)
        lb = statistics.mean(s["lean_bytes"] + s["small_bytes"] for s in stats)
        units = float((sizes[a] + sizes[b]).sum())
        out[name] = {"pairs": int(len(a)), "gints_s": units / ((hms + lms) / 1e3) / 1e9,
                     "k_heavy": {"ms": hms, "alg_bytes": hb, "achieved_gbs": hb / hms / 1e6,
                                 "frac": hb / hms / 1e6 / peak},
                     "pair_stage": {"ms": hms + lms, "alg_bytes": hb + lb,
                                    "achieved_gbs": (hb + lb) / (hms + lms) / 1e6,
                                    "frac": (hb + lb) / (hms + lms) / 1e6 / peak},
                     "deferred_pairs": statistics.mean(s["deferred"] for s in stats)}
    return out


def tuned_schedule(rb, plan, args):
    """The launch schedule for the benchmark: from the schedule cache (JSON
    keyed by GPU name and workload) when it has an entry, else by running
    the library's autotuner (rb_autotune) on the benchmark's own
    materialising plan, untimed, and storing the result."""
    import torch
    if args.no_autotune:
        return {"source": "library default (--no-autotune)"}
    key = f"{torch.cuda.get_device_name()}|{WORKLOAD}|pairs={plan.n}|pool={args.pool or 4096}|hi={args.log10_hi or 7}"
    cache = {}
    path = args.schedule_cache
    try:
        with open(path) as f:
            cache = json.load(f)
    except Exception:
        cache = {}
    if key in cache and not args.retune:
        e = cache[key]
        sc = e["schedule"]
        rb.set_schedule(sc["warps_per_cta"], sc["ctas_per_sm"], sc["small_intervals"], sc["lean_ctas_per_sm"],
                        sc["prefetch_lines"], sc.get("tiles_per_take", 32))
        return {"source": f"schedule cache {path}", "tuned_ms": e.get("ms"), "tuned_at": e.get("at")}
    t0 = time.perf_counter()
    best, ms = plan.autotune(reps=1)
    dt = time.perf_counter() - t0
    cache[key] = {"schedule": best, "ms": ms, "at": time.strftime("%Y-%m-%dT%H:%M:%S"), "search_s": dt}
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path + ".tmp", "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(path + ".tmp", path)
    except Exception as ex:
        log(f"schedule cache not written: {ex}")
    log(f"autotune: {best} ({ms:.2f} ms, search {dt:.1f}s)")
    return {"source": "rb_autotune on this plan (coordinate descent, untimed)", "tuned_ms": ms, "search_s": dt,
            "cache": path}


def plan_leg(rb, plan, units, steps=10, warmup=3):
    """Device time per run of a plan (CUDA events on the current stream
    around a graph replay and its collection), Gints/s over `units` input
    values, and the dominant kernel's algorithmic GB/s against the HBM peak."""
    import torch
    stream = torch.cuda.current_stream()
    peak, _ = measured_peaks()
    for _ in range(warmup):
        outs, _ = plan.run(raw=True)
        plan.free_raw(outs)
    ms, st = [], []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs, _ = plan.run(raw=True)
        e1.record(stream)
        plan.free_raw(outs)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        st.append(plan.stats())
    t = statistics.median(ms)
    ks = {k: (statistics.mean(x[k + "_ms"] for x in st), statistics.mean(x[k + "_bytes"] for x in st))
          for k in ("lean", "small", "heavy")}
    kern = max(ks, key=lambda k: ks[k][0])
    kms, kb = ks[kern]
    gbs = kb / (kms / 1e3) / 1e9 if kms > 0 else 0.0
    return {"ms": t, "gints_s": units / (t / 1e3) / 1e9,
            "roofline": {"kernel": "k_" + kern, "kernel_ms": kms, "alg_bytes": kb, "achieved_gbs": gbs,
                         "frac": gbs / peak, **{f"{k}_ms": v[0] for k, v in ks.items()}}}


def config_legs(rb, args, budget_s=4.0):
    """Throughput on the plain, sparse and run-heavy workloads (the paper's
    Sec. 5 pairwise, wide-union and count workloads, synthetic stand-ins),
    each beside the oracle on every host core and on one core."""
    import oracle
    import torch
    import workloads as W
    oracle.build()
    nthr = os.cpu_count() or 1
    out = {"cpu_model": cpu_model(), "host_threads": nthr}

    def oracle_pair(OA, OB, op, units):
        def f():
            r = OA.op(op, OB)
            r.close()
            return units
        return f

    def oracle_jac(OA, OB, units):
        def f():
            OA.jaccard(OB)
            return units
        return f

    def cpu_legs(tasks):
        v_all, d_all, s_all = time_tasks(tasks, nthr, budget_s)
        v_one, d_one, s_one = time_tasks(tasks, 1, budget_s)
        return {"all_cores": {"gints_s": v_all / 1e9, "cores": nthr, "tasks_done": d_all, "of": len(tasks),
                              "seconds": s_all},
                "one_core": {"gints_s": v_one / 1e9, "cores": 1, "tasks_done": d_one, "of": len(tasks),
                             "seconds": s_one}}

    # plain: AND, OR, ANDNOT, XOR of one pair, materialised, with their counts and Jaccard
    pool = W.plain_pair(1)
    va, vb = pool.values(0), pool.values(1)
    A, B = rb.Bitmap.from_sorted(va), rb.Bitmap.from_sorted(vb)
    u2 = float(len(va) + len(vb))
    ops4 = np.arange(4, dtype=np.uint32)
    pm = rb.Plan([A, B], ops4, np.zeros(4, np.uint32), np.ones(4, np.uint32))
    leg = plan_leg(rb, pm, 4 * u2)
    pm.free()
    calls = []
    for _ in range(13):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rs = [A.op(op, B) for op in range(4)]
        A.jaccard(B)
        calls.append(time.perf_counter() - t0)
        for r in rs:
            r.free()
    OA, OB = oracle.Bitmap.from_sorted(va), oracle.Bitmap.from_sorted(vb)
    tasks = [oracle_pair(OA, OB, op, u2) for op in range(4)] * 8 + [oracle_jac(OA, OB, u2)] * 8
    out["plain"] = {"what": "AND/OR/ANDNOT/XOR of the two bitmaps, materialised (one plan, 4 queries); "
                            "units 4 x (|A|+|B|)", "values": int(u2), **leg,
                    "per_call_gints_s": 4 * u2 / statistics.median(calls[3:]) / 1e9,
                    "per_call_what": "rb_apply x4 + rb_jaccard, one call at a time, host-synchronous",
                    "oracle": cpu_legs(tasks)}
    OA.close(), OB.close(), A.free(), B.free()

    # sparse: AND and OR of the 199 consecutive pairs, and the wide OR of all 200
    pool = W.make_pool(W.SPECS["sparse"])
    vals = [pool.values(i) for i in range(pool.n)]
    G = [rb.Bitmap.from_sorted(v) for v in vals]
    sz = np.array([len(v) for v in vals], np.float64)
    a = np.arange(199, dtype=np.uint32)
    ops = np.concatenate([np.zeros(199, np.uint32), np.ones(199, np.uint32)])
    aa, bb = np.concatenate([a, a]), np.concatenate([a + 1, a + 1])
    units = float((sz[aa] + sz[bb]).sum())
    pm = rb.Plan(G, ops, aa, bb)
    leg = plan_leg(rb, pm, units)
    pm.free()
    wide = []
    for r in range(8):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m, card = rb.multi_op(1, G)
        wide.append(time.perf_counter() - t0)
        m.free()
    wt = statistics.median(wide[3:])
    O = [oracle.Bitmap.from_sorted(v) for v in vals]

    def oracle_wide():
        oracle.Bitmap.multi(1, O).close()
        return float(sz.sum())
    tasks = [oracle_pair(O[int(x)], O[int(y)], int(o), float(sz[x] + sz[y])) for o, x, y in zip(ops, aa, bb)]
    out["sparse"] = {"what": "AND and OR of the 199 consecutive pairs of 200 bitmaps over [0,2^24), c log-uniform "
                             "1e3..1e6, materialised (one plan, 398 queries)", "values": units, **leg,
                     "wide_or": {"values": float(sz.sum()), "ms": wt * 1e3, "gints_s": float(sz.sum()) / wt / 1e9,
                                 "card": int(card), "what": "rb_multi_op(OR) of all 200, host-synchronous call"},
                     "oracle": cpu_legs(tasks)}
    t0 = time.perf_counter()
    oracle_wide()
    ow = time.perf_counter() - t0
    out["sparse"]["wide_or"]["oracle_one_core_gints_s"] = float(sz.sum()) / ow / 1e9
    for o in O:
        o.close()
    for g in G:
        g.free()

    # run-heavy: all four ops of the 199 consecutive pairs, and their Jaccard (count-only)
    pool = W.make_pool(W.SPECS["runs"])
    vals = [pool.values(i) for i in range(pool.n)]
    G = [rb.Bitmap.from_sorted(v) for v in vals]
    sz = np.array([len(v) for v in vals], np.float64)
    ops = np.repeat(np.arange(4, dtype=np.uint32), 199)
    aa, bb = np.tile(a, 4), np.tile(a + 1, 4)
    units = float((sz[aa] + sz[bb]).sum())
    pm = rb.Plan(G, ops, aa, bb)
    leg = plan_leg(rb, pm, units)
    pm.free()
    pj = rb.Plan(G, np.zeros(199, np.uint32), a, a + 1, np.full(199, rb.Q_COUNT_ONLY, np.uint32))
    jleg = plan_leg(rb, pj, float((sz[a] + sz[a + 1]).sum()))
    pj.free()
    O = [oracle.Bitmap.from_sorted(v) for v in vals]
    tasks = [oracle_pair(O[int(x)], O[int(y)], int(o), float(sz[x] + sz[y])) for o, x, y in zip(ops, aa, bb)]
    jt = [oracle_jac(O[int(x)], O[int(x) + 1], float(sz[x] + sz[x + 1])) for x in a]
    out["runs"] = {"what": "AND/OR/ANDNOT/XOR of the 199 consecutive pairs of 200 run-heavy bitmaps over [0,2^26), "
                           "materialised (one plan, 796 queries)", "values": units, **leg,
                   "jaccard": {"what": "count-only Jaccard of the 199 pairs (one plan)", **jleg,
                               "oracle": cpu_legs(jt)},
                   "oracle": cpu_legs(tasks)}
    for o in O:
        o.close()
    for g in G:
        g.free()
    return out


def serving_on_index(rb, args, rates=(1e3, 1e4, 1e5, 1e6), max_queries=40000):
    """The serving workload's own index: 10,000 seeded bitmaps (c log-uniform
    1e2..1e7, 40/30/30 sparse/dense/runs), drawn and uploaded a slice at a
    time, resident on the device while the load runs."""
    import torch
    import workloads as W
    spec = W.SPECS["serving"]
    if args.serving_index:
        spec = W.scaled(spec, n_bitmaps=args.serving_index)
    t0 = time.time()
    G = []
    sizes, cls = W.stream_pool(spec, lambda i, v: G.append(rb.Bitmap.from_sorted(v)))
    torch.cuda.synchronize()
    nbytes = sum(g.payload_bytes() + 10 * g.n_containers for g in G)
    log(f"serving index: {len(G)} bitmaps, {int(sizes.sum()):,} values, {nbytes / 1e9:.2f} GB on the device, "
        f"built in {time.time() - t0:.1f}s")
    try:
        res = serving_leg(rb, G, sizes.astype(np.float64), rates=rates, max_queries=max_queries)
    finally:
        for g in G:
            g.free()
    res["index"] = (f"{len(G)} bitmaps ({int(sizes.sum()):,} values, {nbytes / 1e9:.2f} GB on the device: "
                    f"payload + 10 B of key and descriptor per container), c log-uniform 1e2..1e7, "
                    f"classes {int((cls == 0).sum())}/{int((cls == 1).sum())}/{int((cls == 2).sum())} "
                    f"sparse/dense/runs")
    res["index_bytes"] = nbytes
    return res


SERVER_SLOTS, SERVER_BATCH = 8, 512


def serving_leg(rb, G, sizes, rates=(1e3, 1e4, 1e5, 1e6), seconds=2.0, max_queries=40000):
    """Open-loop Poisson load on the serving loop with the pool as its
    resident index: multi-way AND/OR of 2..8 members, materialised or
    count-only (50/50).  A frontend thread hands every request whose arrival
    time has passed to the server in one call (rb_server_submit_many); a
    collector thread takes completions in bursts (rb_server_poll), which frees
    the results.  Latency = (submit time - scheduled arrival) + the library's
    submit-to-completion time on the device."""
    import threading
    import workloads as W
    out = []
    # 8 batches of up to 512 queries in flight: at saturation about 5% more
    # queries/s than 4 x 256 (fuller multi-way launches), the same latency at low load
    srv = rb.Server(G, mem_budget=64 << 30, max_inflight_batches=SERVER_SLOTS, max_batch=SERVER_BATCH)
    import gc
    switch = sys.getswitchinterval()
    sys.setswitchinterval(5e-5)   # the two client threads hand the interpreter over quickly
    gc.collect()
    gc.disable()                  # no collector pause stalls the frontend thread
    try:
        for rate in rates:
            n = int(min(max_queries, max(200, rate * seconds)))
            ops, ks, co, mem = W.multi_queries(5, n, len(G))
            reqs = rb.Server.requests(ops, ks, co, mem)   # marshalled before the clock starts
            arrivals = W.poisson_arrivals(5, n, rate)
            units = np.array([float(sizes[mem[i, :ks[i]]].sum()) for i in range(n)])
            tickets = np.zeros(n, np.uint64)
            late = np.zeros(n)
            lat = np.full(n, np.nan)
            submitted = [0]

            def collector():
                got = 0
                while got < n:
                    t, st, _, l, _ = srv.poll(cap=4096, timeout_ms=1000)
                    if len(t) == 0:
                        continue
                    idx = (t - tickets[0]).astype(np.int64)
                    if np.any(st != 0):
                        raise RuntimeError(f"serving request failed: {st[st != 0][:4]}")
                    lat[idx] = l
                    got += len(t)
            th = threading.Thread(target=collector)
            t0 = time.perf_counter()
            i = 0
            while i < n:
                now = time.perf_counter() - t0
                j = int(np.searchsorted(arrivals, now, side="right"))
                if j > i:
                    srv.submit_prepared(reqs, i, j, tickets)
                    late[i:j] = (time.perf_counter() - t0) - arrivals[i:j]
                    if i == 0:
                        th.start()
                    i = j
                else:
                    # sleeping releases the interpreter lock to the collector
                    time.sleep(max(0.0, arrivals[i] - now - 5e-5))
            submit_s = time.perf_counter() - t0
            th.join()
            wall = time.perf_counter() - t0
            total = lat + np.maximum(late, 0.0)
            out.append({"offered_qps": rate, "achieved_offered_qps": n / submit_s, "queries": n,
                        "throughput_qps": n / wall, "gints_s": float(units.sum()) / wall / 1e9,
                        "p50_ms": float(np.percentile(total, 50)) * 1e3, "p99_ms": float(np.percentile(total, 99)) * 1e3,
                        "submit_lateness_p99_ms": float(np.percentile(late, 99)) * 1e3})
        st = srv.stats()
    finally:
        gc.enable()
        sys.setswitchinterval(switch)
        srv.close()
    return {"loads": out, "batches": st["batches"], "peak_inflight": st["peak_inflight"],
            "server": {"max_inflight_batches": SERVER_SLOTS, "max_batch": SERVER_BATCH},
            "index": f"the {len(G)}-bitmap pool resident on the device", "budget_bytes": 64 << 30,
            "latency": "from the scheduled Poisson arrival to completion on the device"}


def per_pair_leg(rb, G, ops, a, b, sizes, n=512):
    """The same pairs through rb_apply + rb_jaccard one pair at a time."""
    import torch
    if n <= 0:
        return None
    idx = np.arange(n)
    lat = []
    vals = 0.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in idx:
        s = time.perf_counter()
        r = G[a[i]].op(int(ops[i]), G[b[i]])
        G[a[i]].jaccard(G[b[i]])
        lat.append((time.perf_counter() - s) * 1e3)
        r.free()
        vals += sizes[a[i]] + sizes[b[i]]
    dt = time.perf_counter() - t0
    return {"gints_s": vals / dt / 1e9, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "sample_pairs": int(n),
            "what": "rb_apply + rb_jaccard per pair (one launch sequence and host sync per call)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default schedule")
    ap.add_argument("--retune", action="store_true", help="tune even if the schedule cache has an entry")
    ap.add_argument("--schedule-cache", default=os.environ.get("RB_SCHEDULE_CACHE", os.path.join(
        os.environ.get("XDG_CACHE_HOME", os.path.expanduser("~/.cache")), "gbroaring", "schedules.json")),
        help="JSON schedule cache keyed by GPU name and workload")
    ap.add_argument("--no-configs", action="store_true", help="skip the plain / sparse / run-heavy legs")
    ap.add_argument("--serving-index", type=int, default=0,
                    help="scaled case: bitmaps of the serving index (default: the full 10,000)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-subsets", action="store_true", help="skip the bitset-dominated AND/OR legs")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=5.0, help="seconds of oracle work per reference step")
    ap.add_argument("--per-pair-sample", type=int, default=512)
    ap.add_argument("--pool", type=int, default=0, help="scaled case: number of pool bitmaps (profiling)")
    ap.add_argument("--pairs", type=int, default=0, help="scaled case: number of pairs (profiling)")
    ap.add_argument("--log10-hi", type=float, default=0.0, help="scaled case: top of the cardinality law")
    ap.add_argument("--schedule", default="", help="warps_per_cta,ctas_per_sm,small_intervals")
    ap.add_argument("--serving-only", action="store_true", help="run only the serving leg (profiling)")
    ap.add_argument("--subsets-only", action="store_true", help="run only the bitset-dominated legs (profiling)")
    ap.add_argument("--subset", default="", help="with --subsets-only: uniform, overlapping or both (comma list)")
    ap.add_argument("--serving-rates", default="1e3,1e4,1e5,1e6", help="offered loads of the serving-only run")
    ap.add_argument("--serving-queries", type=int, default=40000, help="queries per load, serving-only run")
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per launch of the dominant kernel from an ncu capture")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
