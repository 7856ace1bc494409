"""Benchmark: exact range search by adaptive group testing on GB300.

One step = one pass of the whole query path (query preparation, dense cutover
when enabled, every frontier level, the leaf tests, the FP64 recheck and the
CSR assembly) over one batch of queries against a resident tree.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is whole-job queries/s with inputs resident in
HBM; `e2e` is the same metric through the C ABI with pinned host inputs and
host results (copies inside the timed region); `roofline` reports the
dominant kernel against the measured HBM copy bandwidth; `cpu_baseline` is
the FP64 oracle (Algorithm 1) timed on the host cores on a bounded sample.
Under torchrun every rank serves its own batch against its own replica of
the tree (queries are independent: weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "queries/s at exact recall (N=1M, d=1000)"
UNIT = "queries/s"
L2_FLUSH_BYTES = 512 << 20


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="softmax_n1m_d1000")
    p.add_argument("--rho", type=float, default=0.8)
    p.add_argument("--dtype", default="bf16", choices=["f32", "bf16", "fp8"])
    p.add_argument("--cutover", type=int, default=-1)
    p.add_argument("--tile", type=int, default=0,
                   help="GEMM tile code (128, 256, 512, 1024); with --cutover, else autotuned")
    p.add_argument("--subtract", type=int, default=0, help="1 / -1: force the subtraction path on / off")
    p.add_argument("--inflight", type=int, default=0,
                   help="tests-in-flight code (1, 2, 4, +8, or 16: ring); with --cutover, else autotuned")
    p.add_argument("--queries", type=int, default=0, help="queries per step (0: the workload's)")
    p.add_argument("--tune-sample", type=int, default=0,
                   help="queries the autotuner times (0: the whole step's batch)")
    p.add_argument("--max-batch", type=int, default=0,
                   help="queries per micro-batch (0: sized by the frontier budget)")
    p.add_argument("--items", type=int, default=0, help="database size (0: the workload's)")
    p.add_argument("--scratch-gb", type=float, default=0.0,
                   help="device scratch budget of a query call in GB (0: the library's default)")
    p.add_argument("--sweep-cutover", default="", help="comma list of cutover levels to time too")
    p.add_argument("--cpu-sample", type=int, default=0, help="oracle sample size (0: auto)")
    p.add_argument("--parity-sample", type=int, default=256,
                   help="queries checked against the oracle's FP64 brute force")
    p.add_argument("--layout", default="tree", choices=["tree", "prefix"],
                   help="tree: a row per pool; prefix: Eq. 1's cumulative sums restarted per "
                        "block of 2^c items (--prefix-level c), the blocks scored by the GEMM")
    p.add_argument("--prefix-level", type=int, default=3)
    p.add_argument("--no-comparators", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-stream", action="store_true", help="skip the streaming-setting run")
    p.add_argument("--no-e2e", action="store_true",
                   help="skip the end-to-end calls (small profiling runs)")
    p.add_argument("--no-large", action="store_true",
                   help="skip the large form (N = 10M, FP8 rows, 100,000 queries)")
    p.add_argument("--serve-rates", default="50000,400000,0",
                   help="offered request rates for the serving run (0: all at once)")
    p.add_argument("--serve-groups", type=int, default=0,
                   help="also time server steps that each answer a fixed group of this many "
                        "queries (no arrival clock: for profiling one served step)")
    return p.parse_args()


def _note(msg: str):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    print(f"bench: {time.strftime('%H:%M:%S')} {msg}", file=sys.stderr, flush=True)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
            "fallback"


class Clocks:
    """nvidia-smi samples every 20 ms.  The sampler is started ahead of the
    warm-up (nvidia-smi takes a while to start); only the samples stamped
    inside the timed region (mark()/stop() wall-clock times) are kept."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.t0 = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def wait_ready(self):
        """Wait, at most 3 s, for the first sample: the sampler is running."""
        end = time.time() + 3.0
        while self.p is not None and time.time() < end:
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.01)

    def mark(self):
        """Start of the timed region."""
        self.t0 = time.time()

    def stop(self, gpu_index: int = 0):
        t1 = time.time()
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.05)        # let the sampler flush its last line
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(", ") for r in self.f.read().splitlines() if r.strip()]
        os.unlink(self.f.name)
        rows = [r for r in rows if len(r) >= 10]
        idx = {r[1] for r in rows}
        if len(idx) > 1:
            rows = [r for r in rows if r[1] == str(gpu_index)] or rows

        def stamp(x):
            try:
                import datetime
                return datetime.datetime.strptime(x.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except Exception:
                return None
        t0 = self.t0 if self.t0 is not None else t1
        inside = [r for r in rows if stamp(r[0]) is not None and t0 <= stamp(r[0]) <= t1]
        rows = [r[1:] for r in (inside or rows[-1:])]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.strip() == "Active"})
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_median": statistics.median(pw) if pw else None,
                "samples": len(rows), "in_timed_region": bool(inside), "reasons": reasons}


def _cpu_model() -> str:
    """The host CPU's model name (lscpu), else the machine type."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return f"{line.split(':', 1)[1].strip()} ({platform.machine()}, {os.cpu_count()} cpus)"
    except Exception:
        pass
    return f"{platform.processor() or platform.machine()} ({os.cpu_count()} cpus)"


def _traffic_record(kernel: str, run_config: dict):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source and on this run's configuration (workload,
    size, rho, row format, cutover: the mix of levels and the L2 reuse depend
    on them), else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kernel)
    except Exception:
        return None
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2311_02573_gb300", "csrc", rec["source"])
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if sha != rec.get("source_sha"):
        return None
    if any(run_config.get(k) != v for k, v in (rec.get("config") or {}).items()):
        return None
    return rec


def reduce_max(value: float, dist=None) -> float:
    """The largest of the ranks' values (the job is as slow as its slowest
    rank); a host-side reduction over the process group, no data-path
    collective."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def serve_run(gt, tree, Q, rhos, rate, n_req, dtype, inserts=None, insert_frac=0.01, seed=0,
              schedule="auto", rho_per_query=None, cutover=-1):
    """Poisson request stream through the continuous-batching server.

    Returns achieved queries/s (completed / span from first arrival to last
    completion) and per-request latency (completion - arrival) percentiles."""
    rng = np.random.default_rng(seed)
    B = Q.shape[0]
    if rate > 0:
        arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    else:
        arrivals = np.zeros(n_req)
    qi = rng.integers(0, B, n_req)
    Qreq = np.ascontiguousarray(Q[qi])   # the requests' vectors, made before the clock starts
    rho = (rho_per_query[qi] if rho_per_query is not None
           else rhos[rng.integers(0, len(rhos), n_req)]).astype(np.float32)
    is_ins = rng.random(n_req) < insert_frac if inserts is not None else np.zeros(n_req, bool)
    srv = gt.Server(tree, dtype=dtype, queue_capacity=n_req, schedule=schedule, cutover=cutover)
    lat = np.full(n_req, np.nan)
    sub = 0
    n_done = 0
    n_q = int((~is_ins).sum())
    ins_i = 0
    t0 = time.perf_counter()
    while n_done < n_q:
        now = time.perf_counter() - t0
        k = int(np.searchsorted(arrivals, now, side="right"))
        if k > sub:
            # the arrivals in order: runs of queries (submitted as views, no
            # copy on the client's side) between inserts
            a0 = sub
            for e in list(np.flatnonzero(is_ins[sub:k]) + sub) + [k]:
                if e > a0:
                    srv.submit(Qreq[a0:e], rho[a0:e], np.arange(a0, e))
                if e < k:
                    srv.insert(inserts[ins_i % inserts.shape[0]][None])
                    ins_i += 1
                a0 = e + 1
            sub = k
        in_flight = srv.step()
        tnow = time.perf_counter() - t0
        tags, _, _, _ = srv.poll_arrays()
        if tags.size:
            lat[tags] = tnow - arrivals[tags]
            n_done += int(tags.size)
        if n_done < n_q and sub < n_req and in_flight == 0 and \
                arrivals[sub] > time.perf_counter() - t0 + 1e-4 and srv.stats()["pending"] == 0:
            time.sleep(max(0.0, arrivals[sub] - (time.perf_counter() - t0) - 5e-5))
    span = (time.perf_counter() - t0) - float(arrivals[0])
    st = srv.stats()
    srv.close()
    l = lat[~np.isnan(lat)] * 1e3
    return {"offered_qps": rate if rate > 0 else "all at t=0", "requests": int(n_q),
            "inserts": int(is_ins.sum()), "achieved_qps": round(n_q / span, 1),
            "p50_ms": round(float(np.percentile(l, 50)), 3),
            "p99_ms": round(float(np.percentile(l, 99)), 3),
            "steps": st["steps"], "mean_group": round(st["admitted"] / max(1, st["steps"]), 1),
            "cutover": st["cutover"], "launches": st["launches"],
            "schedule": {1: "levels", 2: "drain", 3: "immediate"}.get(st["schedule"], st["schedule"])}



def serve_fixed_groups(gt, tree, Q, rho, group, dtype, steps=60, warm=10):
    """Server steps that each admit and answer one group of `group` queries
    (the default schedule), with no arrival clock: the host wall time of a
    step (gt_server_step, synchronize included), median over the steps after
    the first `warm`."""
    srv = gt.Server(tree, dtype=dtype)
    B = Q.shape[0]
    times = []
    for i in range(steps):
        lo = (i * group) % max(1, B - group)
        srv.submit(Q[lo:lo + group], rho, np.arange(lo, lo + group))
        t0 = time.perf_counter()
        srv.step()
        times.append(time.perf_counter() - t0)
        srv.poll_arrays()
    st = srv.stats()
    srv.close()
    return {"group": group, "steps": steps, "step_ms_median": round(1e3 * float(np.median(times[warm:])), 4),
            "schedule": {1: "levels", 2: "drain", 3: "immediate"}.get(st["schedule"], st["schedule"]),
            "launches_per_step": round(st["launches"] / max(1, st["steps"]), 2)}


def side_by_side(gt, tree, Fd, Qd, rd, B, dtype, tune, flush, capacity, reps=3):
    """The batch split in two halves answered at the same time by two trees
    over the same rows, each call's kernels sized for part of the SMs
    (gt_set_sm_limit) and issued from its own host thread and stream, so one
    half's dense GEMM (tensor-bound) can overlap the other's gathers
    (memory-bound).  Host wall-clock seconds per batch, against the same
    batch in one call on every SM, timed the same way."""
    import threading
    import torch
    sub = 1 if tune.get("subtract") else -1
    kw = dict(dtype=dtype, cutover=tune["cutover"], subtract=sub, results_on_device=True)
    tree2 = gt.Tree(Fd, capacity=capacity)
    tree2.set_tuning(dtype, cutover=tune["cutover"], inflight=tune["inflight"], tile=tune["tile_n"])
    trees = (tree, tree2)
    streams = (torch.cuda.Stream(), torch.cuda.Stream())
    halves = ((0, B // 2), (B // 2, B))

    def wall(fn):
        best = None
        for rep in range(reps + 1):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if rep > 0:
                best = dt if best is None else min(best, dt)
        return best

    def one_call():
        tree.query(Qd, rd, stream=streams[0], **kw).free()

    def two_calls():
        res = [None, None]

        def run(i):
            lo, hi = halves[i]
            res[i] = trees[i].query(Qd[lo:hi], rd[lo:hi], stream=streams[i], **kw)
        ths = [threading.Thread(target=run, args=(i,)) for i in (0, 1)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        for r in res:
            r.free()

    out = {"call": "gt_query, two trees, two host threads and streams, halves of the batch",
           "one_call_all_sms_ms": round(1e3 * wall(one_call), 3)}
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    for split in (n_sm * 5 // 12, n_sm // 2, n_sm * 7 // 12):
        tree.set_sm_limit(split)
        tree2.set_sm_limit(n_sm - split)
        out[f"two_calls_{split}_{n_sm - split}_sms_ms"] = round(1e3 * wall(two_calls), 3)
    tree.set_sm_limit(0)
    tree2.close()
    best = min(v for k, v in out.items() if k.startswith("two_calls"))
    out["speedup_best_split"] = round(out["one_call_all_sms_ms"] / best, 3)
    return out


def served_d512_run(gt, flush, rates=(5000.0, 20000.0, 50000.0)):
    """The served form at N = 1M, d = 512: BF16 rows, per-query rho ~ U[0.8,
    0.97], 1% of requests inserts; the batch path's queries/s (CUDA events)
    and the server's p50/p99 at the offered rates."""
    import torch
    import synth
    ds = synth.generate("softmax_n1m_d512_served")
    B = ds.Q.shape[0]
    Fd = torch.from_numpy(ds.F).cuda()
    t = gt.Tree(Fd, capacity=ds.F.shape[0] + 65536)
    del Fd
    Qd, rd = torch.from_numpy(ds.Q).cuda(), torch.from_numpy(ds.rho).cuda()
    stream = torch.cuda.current_stream()
    tune = t.autotune(Qd, rd, dtype="bf16", stream=stream)
    t.query(Qd, rd, results_on_device=True, stream=stream).free()
    ts = []
    for _ in range(3):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = t.query(Qd, rd, results_on_device=True, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
        r.free()
    extra = ds.F[np.random.default_rng(9).choice(ds.F.shape[0], 4096, replace=False)]
    served = [serve_run(gt, t, ds.Q, None, r_, int(min(20000, max(8000, r_ * 0.4))), "bf16",
                        inserts=extra, seed=13, rho_per_query=ds.rho) for r_ in rates]
    t.close()
    return {"workload": "softmax_n1m_d512_served", "N": int(ds.F.shape[0]), "d": int(ds.F.shape[1]),
            "queries": int(B), "rho": "per query, U[0.8, 0.97]",
            "batch_qps": round(B / (statistics.mean(ts) / 1e3), 1), "unit": UNIT,
            "autotune": {k: tune[k] for k in ("cutover", "inflight", "tile_n", "subtract")},
            "serving": served}


def large_run(gt, flush, check, max_batch=4096, rho=0.9):
    """The large form: N = 10M, d = 1000, FP8 rows with per-row scales (FP32
    masters for the rechecks), 100,000 queries in micro-batches of 4096,
    heavy-tailed planted duplicates; the margin screen and the oracle's
    check on a sample of the queries (including the most planted ones)."""
    import torch
    import synth
    free, _ = torch.cuda.mem_get_info()
    if free < 200e9:
        return {"skipped": f"needs ~200 GB of free device memory, {free / 1e9:.0f} GB free"}
    w = synth.WORKLOADS["softmax_n10m_d1000"]
    rng = np.random.default_rng(5)
    counts = synth._plant_counts(w, w.n_queries)
    sample = np.union1d(np.sort(rng.choice(w.n_queries, 12, replace=False)), np.argsort(counts)[-4:])
    t0 = time.time()
    ds = synth.generate(w, screen=sample)
    gen_s = time.time() - t0
    Fd = torch.from_numpy(ds.F).cuda()
    t = gt.Tree(Fd, formats=("bf16", "fp8"))
    del Fd
    torch.cuda.empty_cache()
    r = ds.rho_for(rho)
    Qd, rd = torch.from_numpy(ds.Q).cuda(), torch.from_numpy(r).cuda()
    stream = torch.cuda.current_stream()
    B = ds.Q.shape[0]
    # the tree's cutover level, subtraction path and tests in flight chosen
    # on one micro-batch (setup, outside the timed calls)
    t0 = time.time()
    tune = t.autotune(Qd[:max_batch], rd[:max_batch], dtype="fp8", stream=stream)
    tune_s = time.time() - t0
    t.query(Qd, rd, dtype="fp8", max_batch=max_batch, results_on_device=True, stream=stream).free()
    ts = []
    for _ in range(2):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = t.query(Qd, rd, dtype="fp8", max_batch=max_batch, results_on_device=True,
                      stream=stream, timing=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
        st = res.stats
        res.free()
    out = {"workload": "softmax_n10m_d1000", "N": int(ds.F.shape[0]), "d": int(ds.F.shape[1]),
           "queries": int(B), "rho": rho, "row_format": "fp8", "micro_batch": max_batch,
           "value": round(B / (statistics.mean(ts) / 1e3), 1), "unit": UNIT,
           "ms_per_batch": round(statistics.mean(ts), 2), "micro_batches": st["micro_batches"],
           "cutover": st["cutover"], "kernel_ms": st["kernel_ms"],
           "gathered_tests_per_query": st["gathered_tests"] / B, "generate_s": round(gen_s, 1),
           "autotune": {"cutover": tune["cutover"], "subtract": tune["subtract"],
                        "inflight": tune["inflight"], "tile_n": tune["tile_n"],
                        "sample": max_batch, "seconds": round(tune_s, 1), "ms": tune["ms"]}}
    if check:
        import oracle
        got = t.query(ds.Q[sample], r[sample], dtype="fp8")
        ref = oracle.brute_force(ds.F, ds.Q[sample], r[sample])
        out["parity_sample"] = {"queries": int(len(sample)), "oracle": "brute_force (FP64)",
                                "identical": bool(np.array_equal(got.offsets, ref.offsets)
                                                  and np.array_equal(got.ids, ref.ids)),
                                "oracle_ambiguous": int(ref.ambiguous.sum())}
    t.close()
    del ds
    return out


def signed_run(gt, flush, check, N=262144, d=256, B=2000, rho=0.8, n_check=64):
    """Descriptors with negative entries (Sec. 2: pools by element-wise
    maximum and minimum; the paper runs no experiment on them): seeded
    Gaussian unit vectors, queries a random item plus noise (cosine about
    0.94 to it), a GT_POOL_MAXMIN tree, autotuned.  Queries/s with inputs on
    the device, CUDA events; beside it a dense FP32 library product (cuBLAS
    through torch) with the threshold applied, for context; the sets checked
    against the oracle's FP64 brute force on a sample of the queries."""
    import torch
    import synth
    F, Q = synth.signed_workload(N, d, B, noise=0.35 / np.sqrt(d), seed=11)
    Fd, Qd = torch.from_numpy(F).cuda(), torch.from_numpy(Q).cuda()
    rd = torch.full((B,), rho, dtype=torch.float32, device="cuda")
    t = gt.Tree(Fd, pooling="maxmin")
    tune = t.autotune(Qd, rd, dtype="bf16")
    stream = torch.cuda.current_stream()

    def timed(fn, n=3):
        warm = fn()
        if hasattr(warm, "free"):
            warm.free()
        ts, stats = [], None
        for _ in range(n):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            if hasattr(r, "free"):
                stats = r.stats
                r.free()
        return B / (statistics.mean(ts) / 1e3), stats
    qps, st = timed(lambda: t.query(Qd, rd, dtype="bf16", results_on_device=True, stream=stream))

    def library():
        hits = 0
        for lo in range(0, N, 65536):
            hits += int((Qd @ Fd[lo:lo + 65536].T >= rho).sum())
        return hits
    torch.backends.cuda.matmul.allow_tf32 = False
    lib_qps, _ = timed(library)
    out = {"workload": f"signed Gaussian unit vectors, N={N}, d={d}, {B} queries, rho={rho}",
           "value": round(qps, 1), "unit": "queries/s", "cutover": tune["cutover"],
           "inflight": tune["inflight"], "tests_per_query": st["tests"] / B,
           "gathered_tests_per_query": st["gathered_tests"] / B,
           "rechecks_per_query": st["rechecks"] / B, "results_per_query": st["results"] / B,
           "fp32_library_product_qps": round(lib_qps, 1)}
    if check:
        import oracle
        res = t.query(Q[:n_check], np.full(n_check, rho, np.float32), dtype="bf16")
        ref = oracle.brute_force(F, Q[:n_check], np.full(n_check, rho, np.float32))
        out["parity_sample"] = {"queries": n_check, "oracle": "brute_force (FP64)",
                                "identical": bool(np.array_equal(res.offsets, ref.offsets)
                                                  and np.array_equal(res.ids, ref.ids)),
                                "oracle_ambiguous": int(ref.ambiguous.sum())}
    t.close()
    return out


def streaming_run(gt, ds, dtype, rho, chunk=100, n_check=256, seed=0):
    """The paper's streaming setting (Sec. 4): build on 80% of the database,
    then add the rest `chunk` points at a time, firing one query after each
    chunk, until the whole database is in.  Reports the index build time, the
    mean insertion time per point, the mean query time, and precision and
    recall on a sample of the queries, each against the exhaustive scan
    (gt_exhaustive_tree, the paper's Exh over the tree's items) restricted to
    the items present when the query ran."""
    import torch
    N = ds.F.shape[0]
    n0 = int(0.8 * N)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tree = gt.Tree(ds.F[:n0], capacity=N)      # from host memory, as a user would
    torch.cuda.synchronize()
    ibt = time.perf_counter() - t0
    Fd = torch.from_numpy(ds.F[:n0]).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tree2 = gt.Tree(Fd, capacity=N)            # rows already on the device
    torch.cuda.synchronize()
    ibt_dev = time.perf_counter() - t0
    tree2.close()
    del Fd
    rng = np.random.default_rng(seed)
    n_chunks = (N - n0 + chunk - 1) // chunk
    qid = rng.integers(0, ds.Q.shape[0], n_chunks)
    rho_h = np.full(1, rho, dtype=np.float32)
    check = set(rng.choice(n_chunks, min(n_check, n_chunks), replace=False).tolist())
    t_ins, t_q, got = [], [], {}
    n = n0
    for k in range(n_chunks):
        rows = np.ascontiguousarray(ds.F[n:n + chunk])
        t0 = time.perf_counter()
        tree.insert(rows)
        torch.cuda.synchronize()
        t_ins.append((time.perf_counter() - t0) / rows.shape[0])
        n += rows.shape[0]
        q = np.ascontiguousarray(ds.Q[qid[k]:qid[k] + 1])
        t0 = time.perf_counter()
        res = tree.query(q, rho_h, dtype=dtype)
        t_q.append(time.perf_counter() - t0)
        if k in check:
            got[k] = (n, res.neighbours(0))
    # the answer at snapshot n is {i < n : q.f_i >= rho}: one exhaustive pass
    # over the full database, filtered per query
    ks = sorted(got)
    ref = tree.exhaustive(np.ascontiguousarray(ds.Q[qid[ks]]), np.full(len(ks), rho, dtype=np.float32))
    tree.close()
    tp = fp = fn = 0
    for i, k in enumerate(ks):
        n_snap, ids = got[k]
        want = ref.neighbours(i)
        want = set(want[want < n_snap].tolist())
        have = set(ids.tolist())
        tp += len(want & have)
        fp += len(have - want)
        fn += len(want - have)
    t_q = np.array(t_q) * 1e3
    return {"initial_items": n0, "inserted": N - n0, "chunk": chunk, "queries": n_chunks, "rho": rho,
            "ibt_s": round(ibt, 3), "ibt_device_rows_s": round(ibt_dev, 4),
            "mit_ms_per_point": round(float(np.mean(t_ins)) * 1e3, 5),
            "mqt_ms": round(float(np.mean(t_q)), 3), "mqt_p99_ms": round(float(np.percentile(t_q, 99)), 3),
            "checked_queries": len(ks), "mp": 1.0 if tp + fp == 0 else round(tp / (tp + fp), 6),
            "mr": 1.0 if tp + fn == 0 else round(tp / (tp + fn), 6),
            "reference": "gt_exhaustive_tree on the final database, ids filtered to the snapshot",
            "timing": "host wall clock per public-API call (gt_insert of a host chunk; gt_query of one "
                      "host query with a host CSR result)"}


def _e2e_calls(a, tree, Q, rho, B, stream, flush):
    """End to end through the C ABI: pinned host inputs, CSR written into
    caller-owned pinned host buffers (gt_query_into), every step's copies
    inside the timed region; and gt_query with a library-allocated host CSR."""
    import torch
    _note("end-to-end calls")
    Qh = torch.from_numpy(Q).pin_memory()
    rh = torch.from_numpy(rho).pin_memory()
    r = tree.query(Qh, rh, dtype=a.dtype, cutover=a.cutover, stream=stream)
    offs_h = torch.empty(B + 1, dtype=torch.int64).pin_memory()
    ids_h = torch.empty(max(1, int(r.ids.size * 1.5)), dtype=torch.int32).pin_memory()
    offs_np, ids_np = offs_h.numpy(), ids_h.numpy()
    torch.cuda.synchronize()
    e2e_t, e2e_lib_t, d2h = [], [], 0
    for _ in range(max(2, a.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        n_res = tree.query_into(Qh, rh, offs_np, ids_np, dtype=a.dtype, cutover=a.cutover,
                                stream=stream)
        e2e_t.append(time.perf_counter() - t1)
        d2h = offs_np.nbytes + n_res * 4
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        r = tree.query(Qh, rh, dtype=a.dtype, cutover=a.cutover, stream=stream)
        e2e_lib_t.append(time.perf_counter() - t1)
    e2e = {"value": round(B / statistics.mean(e2e_t), 1), "unit": UNIT,
           "h2d_bytes_per_step": int(Qh.numel() * 4 + rh.numel() * 4),
           "d2h_bytes_per_step": int(d2h),
           "call": "gt_query_into, pinned host inputs and caller-owned pinned host CSR"}
    e2e_library_csr = {"value": round(B / statistics.mean(e2e_lib_t), 1), "unit": UNIT,
                       "call": "gt_query with a library-allocated (pageable) host CSR"}
    assert np.array_equal(r.offsets, offs_np) and np.array_equal(r.ids, ids_np[:n_res])
    host_result = r
    return e2e, e2e_library_csr, host_result


def run_reference(a):
    """The oracle (Algorithm 1, FP64 cumulative sums) on the host cores."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    import synth
    ds = synth.generate(a.workload)          # the margin screen may use the GPU: inputs only
    B = ds.Q.shape[0]
    per_step = a.cpu_sample or 64
    rho = ds.rho_for(a.rho if ds.rho is None else None)
    rng = np.random.default_rng(1)
    threads = oracle.max_threads()
    # the cumulative sums are the offline index (Eq. 1): built once, untimed;
    # only the query loop is timed
    index = oracle.Index(ds.F, threads=threads)
    times = []
    for step in range(a.warmup + a.steps):
        qs = rng.choice(B, per_step, replace=False)
        res = index.query(ds.Q[qs], rho[qs], threads=threads)
        if step >= a.warmup:
            times.append(res.seconds)
    index.close()
    total = sum(times)
    value = per_step * a.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * total / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic softmax features (seeded)",
            "config": {"workload": a.workload, "N": int(ds.F.shape[0]), "d": int(ds.F.shape[1]),
                       "queries_per_step": per_step, "rho": a.rho},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "cpu_model": _cpu_model(),
                             "sample": f"Algorithm 1 (FP64 cumulative sums) on {per_step} random "
                                       f"queries per step, rho={a.rho}; cumulative-sum build "
                                       "not timed"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
        return
    import torch

    import synth
    from paper_2311_02573_gb300 import gt
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    t_gen = time.time()
    ds = synth.generate(a.workload, N=a.items or None)
    t_gen = time.time() - t_gen
    _note(f"generated {a.workload} in {t_gen:.1f} s")
    B = a.queries or ds.Q.shape[0]
    Q = ds.Q[:B]
    rho = ds.rho_for(a.rho if ds.rho is None else None)[:B]
    N, d = ds.F.shape
    Fd = torch.from_numpy(ds.F).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    # spare capacity for the serving run's inserts (no storage growth mid-stream)
    _note("building the tree")
    pre = a.layout == "prefix"
    if pre:
        # no comparators or streaming run for this layout (they run the tree);
        # its GEMM level is fixed by the build, the autotuner picks the tile
        a.no_comparators = a.no_stream = True
        tree = gt.Tree(Fd, capacity=N + 65536, layout="prefix", prefix_level=a.prefix_level,
                       formats=("bf16", "f32") if a.dtype == "f32" else None)
    else:
        tree = gt.Tree(Fd, capacity=N + 65536)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    Qd = torch.from_numpy(Q).to(dev)
    rd = torch.from_numpy(rho).to(dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    tune = None
    if a.tile and not pre:
        tree.set_tuning(a.dtype, tile=a.tile)
    if a.inflight and not pre:
        tree.set_tuning(a.dtype, inflight=a.inflight)
    if a.cutover == -1:
        # the autotuner picks the cutover level and tests in flight per warp on
        # a sample batch (setup, outside the timed region)
        ns = a.tune_sample or B
        _note(f"autotuning on {ns} queries")
        tune = tree.autotune(Qd[:ns], rd[:ns], dtype=a.dtype, stream=stream)

    scratch = int(a.scratch_gb * 1e9)

    def step(**kw):
        return tree.query(Qd, rd, dtype=a.dtype, cutover=a.cutover, results_on_device=True,
                          stream=stream, subtract=a.subtract, max_batch=a.max_batch,
                          scratch_bytes=scratch, **kw)

    _note("timed steps")
    clocks = Clocks()
    clocks.start()
    clocks.wait_ready()
    # (the warm-up calls take the timed calls' options, so the CUDA graph the
    # timed steps replay is captured here, not inside the first timed step)
    for _ in range(a.warmup):
        step(timing=True).free()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    stats = []
    torch.cuda.synchronize()
    clocks.mark()
    # (Python's cyclic collector is paused over the timed steps, as timeit
    # does: a collection inside a step would time the interpreter, not the
    # library)
    gc.collect()
    gc.disable()
    try:
        for i in range(a.steps):
            flush.zero_()                       # L2 flush, outside the timed events
            ev[i][0].record(stream)
            r = step(timing=True)
            ev[i][1].record(stream)
            stats.append(r.stats)
            r.free()
        torch.cuda.synchronize()
    finally:
        gc.enable()
    clk = clocks.stop(local)
    step_ms = [s.elapsed_time(e) for s, e in ev]
    total_ms = reduce_max(sum(step_ms), dist)
    value = ws * B * a.steps / (total_ms / 1e3)

    # dominant kernel and its roofline; the other hot kernel reported beside it
    st0 = stats[-1]
    km = {k: sum(s["kernel_ms"][k] for s in stats) / len(stats) for k in st0["kernel_ms"]}
    peaks, peaks_src = _peaks()
    gather_ms = km["levels"] + km["leaf"]
    g_launches = max(1, st0["level_launches"] + st0["micro_batches"])
    gb = st0["gathered_bytes"]
    g_ach = gb / (gather_ms * 1e-3) / 1e9 if gather_ms > 0 else 0.0
    run_cfg = {"workload": a.workload, "N": int(N), "queries": int(B), "rho": a.rho,
               "dtype": a.dtype, "cutover": st0["cutover"]}
    tr = _traffic_record("gather_prefix" if pre else "gather", run_cfg)
    # Rows of popular pools are read by many queries and partly served from L2,
    # so the algorithmic row bytes per second can exceed the copy peak.  The
    # fraction is therefore taken on DRAM bytes (the algorithmic bytes times
    # the DRAM/algorithmic ratio of a one-pass ncu capture of the same kernels
    # on the same configuration, recorded with its command in
    # profiles/traffic.json); the algorithmic rate is reported beside it.
    ratio = tr["dram_bytes_per_algorithmic_byte"] if tr else None
    traffic = ratio * gb / g_launches if ratio else None
    g_dram = g_ach * ratio if ratio else None
    roof_gather = {"kernel": "gather (k_ring modes 5, 6: the prefix splits below the GEMM level)" if pre
                   else "gather (k_ring / k_level: the levels below the cutover and the items)",
                   "bound": "hbm",
                   "achieved": round(g_dram if ratio else g_ach, 1), "peak": peaks["hbm_gbs"],
                   "unit": "GB/s",
                   "frac": round((g_dram if ratio else g_ach) / peaks["hbm_gbs"], 4),
                   "basis": "DRAM bytes (algorithmic bytes x the DRAM/algorithmic ratio of "
                            f"{tr.get('case', 'an ncu capture')}) per CUDA-event second" if ratio else
                            "algorithmic bytes (no DRAM record for the current kernel source "
                            "and this configuration)",
                   "achieved_algorithmic": round(g_ach, 1),
                   "frac_algorithmic": round(g_ach / peaks["hbm_gbs"], 4),
                   "dram_per_algorithmic_byte": ratio,
                   "peak_source": f"hbm_gbs of {peaks_src}",
                   "algorithmic_bytes_per_launch": gb / g_launches,
                   "avg_launch_ms": gather_ms / g_launches,
                   "traffic": traffic}
    roof_dense = None
    if km["dense"] > 0 and st0["cutover"] >= 0:
        # algorithmic: 2 d FLOP per (query, pool) score (the kernel's K is d
        # padded to a multiple of 64, not counted)
        flops = 2.0 * st0["dense_tests"] * d               # per step (one launch per micro-batch)
        n_l = max(1, st0["micro_batches"])
        ach = flops / (km["dense"] * 1e-3) / 1e12
        # The step is a few milliseconds with idle gaps (the L2 flush) between
        # steps, and the SM clock stays at its maximum through the timed
        # region (the clock record), so the GEMM is compared with the burst
        # figure; the seconds-long power-capped figure is reported beside it.
        peak = peaks["bf16_tflops"]
        sus = peaks.get("bf16_tflops_sustained")
        trd = _traffic_record("k_dense", run_cfg)
        roof_dense = {"kernel": "k_dense (tcgen05 cutover GEMM)", "bound": "tensor",
                      "achieved": round(ach, 1), "peak": peak, "unit": "TFLOP/s",
                      "frac": round(ach / peak, 4),
                      "frac_of_sustained": round(ach / sus, 4) if sus else None,
                      "peak_source": f"bf16_tflops (burst) of {peaks_src}; frac_of_sustained "
                                     f"against bf16_tflops_sustained (seconds-long, power-capped)",
                      "algorithmic_flops_per_launch": flops / n_l,
                      "avg_launch_ms": km["dense"] / n_l,
                      "traffic": (trd["dram_bytes_per_flop"] * flops / n_l) if trd else None,
                      "traffic_source": trd.get("case") if trd else None}
    if roof_dense and km["dense"] > gather_ms:
        roof, roof_other = roof_dense, roof_gather
    else:
        roof, roof_other = roof_gather, roof_dense

    comparators = {}
    if not a.no_comparators:
        def timed(fn, n=2):
            fn().free()
            torch.cuda.synchronize()
            ts = []
            for _ in range(n):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
                s = r.stats
                r.free()
            return B / (statistics.mean(ts) / 1e3), s
        for name, kw in (("plain_f32_traversal", dict(dtype="f32", cutover=-2)),
                         ("bf16_traversal", dict(dtype="bf16", cutover=-2)),
                         ("fp8_traversal", dict(dtype="fp8", cutover=-2))):
            if kw["dtype"] == a.dtype and kw["cutover"] == a.cutover:
                continue
            qps, s = timed(lambda: tree.query(Qd, rd, results_on_device=True, stream=stream, **kw))
            comparators[name] = {"value": round(qps, 1), "unit": UNIT,
                                 "tests_per_query": s["tests"] / B,
                                 "gathered_bytes_per_query": s["gathered_bytes"] / B}
        if a.dtype != "fp8" and tune is not None:
            # FP8 rows at the same cutover: where the extra time goes (tests per
            # level, leaf re-scores from the BF16 and FP32 rows, FP64 rechecks)
            qps, s = timed(lambda: tree.query(Qd, rd, dtype="fp8", results_on_device=True,
                                              stream=stream, timing=True))
            comparators["fp8_rows"] = {
                "value": round(qps, 1), "unit": UNIT, "cutover": s["cutover"],
                "gathered_tests_per_query": s["gathered_tests"] / B,
                "level_tests_per_query": [round(x / B, 1) for x in
                                          s["level_tests"][:max(0, s["cutover"]) + 1]],
                "refines_per_query": s["refines"] / B, "rechecks_per_query": s["rechecks"] / B,
                "gathered_bytes_per_query": s["gathered_bytes"] / B, "kernel_ms": s["kernel_ms"],
                "bf16_rows": {"gathered_tests_per_query": st0["gathered_tests"] / B,
                              "level_tests_per_query": [round(x / B, 1) for x in
                                                        st0["level_tests"][:max(0, st0["cutover"]) + 1]],
                              "refines_per_query": st0["refines"] / B,
                              "rechecks_per_query": st0["rechecks"] / B,
                              "gathered_bytes_per_query": st0["gathered_bytes"] / B}}
        for c in [int(x) for x in a.sweep_cutover.split(",") if x.strip()]:
            qps, s = timed(lambda: tree.query(Qd, rd, dtype=a.dtype, cutover=c,
                                              results_on_device=True, stream=stream, timing=True))
            comparators[f"cutover_{c}"] = {"value": round(qps, 1), "unit": UNIT,
                                           "tests_per_query": s["tests"] / B,
                                           "gathered_tests_per_query": s["gathered_tests"] / B,
                                           "kernel_ms": s["kernel_ms"]}
        try:
            # the paper's Exh: every (query, item) pair, over the database's rows
            # as the caller holds them (gt_exhaustive: the rows are quantised to
            # BF16 inside each call, then one tcgen05 GEMM with the bound-checked
            # threshold and the FP64 recheck; no tree)
            qps, s = timed(lambda: gt.exhaustive(Fd, Qd, rd, results_on_device=True, stream=stream))
            comparators["exhaustive_gemm_bf16"] = {
                "value": round(qps, 1), "unit": UNIT, "call": "gt_exhaustive over the FP32 rows "
                "on the device (BF16 copy made inside the call)", "rechecks": s["rechecks"],
                "results": s["results"]}
        except gt.GTError as e:
            comparators["exhaustive_gemm_bf16"] = {"unavailable": str(e)}
        # the paper's Our-Max: pools by element-wise maximum (Sec. 2), tuned the
        # same way; its answers are the same exact sets
        mtree = gt.Tree(torch.from_numpy(ds.F).to(dev), pooling="max")
        mtune = mtree.autotune(Qd, rd, dtype=a.dtype, stream=stream)
        qps, s = timed(lambda: mtree.query(Qd, rd, dtype=a.dtype, results_on_device=True,
                                           stream=stream), n=3)
        mres = mtree.query(Qd, rd, dtype=a.dtype, stream=stream)
        ref_res = tree.query(Qd, rd, dtype=a.dtype, stream=stream)
        comparators["max_pooling"] = {
            "value": round(qps, 1), "unit": UNIT, "tests_per_query": s["tests"] / B,
            "gathered_tests_per_query": s["gathered_tests"] / B,
            "cutover": mtune["cutover"], "inflight": mtune["inflight"],
            "same_sets_as_sum_pooling": bool(np.array_equal(mres.offsets, ref_res.offsets)
                                             and np.array_equal(mres.ids, ref_res.ids))}
        mres.free()
        ref_res.free()
        mtree.close()
        torch.cuda.empty_cache()
        if tune is not None:
            comparators["side_by_side"] = side_by_side(gt, tree, Fd, Qd, rd, B, a.dtype, tune, flush,
                                                       N + 65536)
            torch.cuda.empty_cache()
        comparators["signed_maxmin"] = signed_run(gt, flush, rank == 0 and not a.no_cpu)
        torch.cuda.empty_cache()
        # the paper's prefix-sum layout (Eq. 1), with the sums restarted per
        # block of 2^3 items: N prefix rows instead of a row per pool
        N_, stride_ = ds.F.shape[0], (ds.F.shape[1] + 63) // 64 * 64
        rows_tree = sum((N_ + (1 << h) - 1) >> h for h in range(0, 64) if (1 << h) < 2 * N_)
        ptree = gt.Tree(torch.from_numpy(ds.F).to(dev), layout="prefix", prefix_level=3,
                        formats=("bf16", "f32"), capacity=N_ + 65536)
        pres = {}
        for pdt in ("bf16", "f32"):
            qps, s = timed(lambda: ptree.query(Qd, rd, dtype=pdt, results_on_device=True,
                                               stream=stream, timing=True), n=3)
            r_ = ptree.query(Qd, rd, dtype=pdt, stream=stream)
            ref_res = tree.query(Qd, rd, dtype=a.dtype, stream=stream)
            pres[pdt] = {"value": round(qps, 1), "unit": UNIT, "tests_per_query": s["tests"] / B,
                         "gathered_tests_per_query": s["gathered_tests"] / B,
                         "rechecks_per_query": s["rechecks"] / B, "kernel_ms": s["kernel_ms"],
                         "same_sets_as_tree": bool(np.array_equal(r_.offsets, ref_res.offsets)
                                                   and np.array_equal(r_.ids, ref_res.ids))}
            r_.free()
            ref_res.free()
        comparators["prefix_layout"] = {
            "prefix_level": 3, "bf16": pres["bf16"], "f32": pres["f32"],
            # device bytes: FP32 items + BF16 prefix rows + BF16 block totals
            # (+ FP32 prefix rows when kept) against the tree's FP32 + BF16 + FP8
            # rows of every pool
            "device_gb_bf16_rows": round((N_ * 4 + N_ * 2 + ((N_ + 7) >> 3) * 2) * stride_ / 1e9, 2),
            "device_gb_with_f32_rows": round((N_ * 8 + N_ * 2 + ((N_ + 7) >> 3) * 2) * stride_ / 1e9, 2),
            "tree_device_gb": round(rows_tree * stride_ * 7 / 1e9, 2)}
        if not a.no_serve:
            # the same continuous-batching server over the prefix layout (its
            # GEMM tile tuned first), 50k q/s offered, 1% of requests inserts
            ptree.autotune(Qd, rd, dtype="bf16", stream=stream)
            rhos = np.array(ds.workload.rhos or (a.rho,), dtype=np.float32)
            extra = ds.F[np.random.default_rng(8).choice(N, 4096, replace=False)]
            comparators["prefix_layout"]["serving"] = serve_run(gt, ptree, Q, rhos, 50000.0, 20000,
                                                                "bf16", inserts=extra)
        ptree.close()
        torch.cuda.empty_cache()
    del Fd

    e2e = e2e_library_csr = host_result = None
    if a.no_e2e:
        a.no_cpu = True       # the oracle checks the end-to-end call's result
    else:
        e2e, e2e_library_csr, host_result = _e2e_calls(a, tree, Q, rho, B, stream, flush)

    cpu = None
    parity = None
    if rank == 0 and not a.no_cpu:
        import oracle
        threads = oracle.max_threads()
        n = a.cpu_sample or 1024
        qs = np.random.default_rng(2).choice(B, min(n, B), replace=False)
        qs.sort()
        index = oracle.Index(ds.F, threads=threads)
        ref = index.query(Q[qs], rho[qs], threads=threads)
        # the same oracle on one thread (the paper does not state its threads)
        q1 = qs[: min(len(qs), 64)]
        ref1 = index.query(Q[q1], rho[q1], threads=1)
        index.close()
        cpu = {"value": round(len(qs) / ref.seconds, 2), "unit": UNIT, "cores": threads,
               "kind": "oracle", "cpu_model": _cpu_model(),
               "sample": f"Algorithm 1 (FP64 cumulative sums) on {len(qs)} of the {B} queries, "
                         f"rho={a.rho}; cumulative-sum build not timed",
               "one_thread": {"value": round(len(q1) / ref1.seconds, 2), "unit": UNIT, "cores": 1,
                              "sample": f"the first {len(q1)} of those queries"}}
        # parity against the definition: the oracle's FP64 brute force on a
        # bounded sample (every item of the database against each query)
        qb = np.random.default_rng(3).choice(B, min(a.parity_sample, B), replace=False)
        qb.sort()
        bf = oracle.brute_force(ds.F, Q[qb], rho[qb], threads=threads)
        ok = all(np.array_equal(bf.neighbours(i), host_result.neighbours(int(q)))
                 for i, q in enumerate(qb))
        ok_alg1 = all(np.array_equal(ref.neighbours(i), host_result.neighbours(int(q)))
                      for i, q in enumerate(qs))
        parity = {"queries": int(len(qb)), "identical": bool(ok), "oracle": "brute_force (FP64)",
                  "oracle_ambiguous": int(bf.ambiguous.sum()),
                  "brute_force_seconds": round(bf.seconds, 2),
                  "algorithm1": {"queries": int(len(qs)), "identical": bool(ok_alg1),
                                 # decisions inside its FP64 rounding bound
                                 "ambiguous_decisions": int(ref.ambiguous.sum())}}

    # the serving run inserts rows, so it comes after every exactness check
    served_fixed = None
    if a.serve_groups > 0 and rank == 0:
        served_fixed = serve_fixed_groups(gt, tree, Q, float(a.rho), a.serve_groups, a.dtype)
    serving = None
    if not a.no_serve and rank == 0:
        rhos = np.array(ds.workload.rhos or (a.rho,), dtype=np.float32)
        extra = ds.F[np.random.default_rng(7).choice(N, 4096, replace=False)]
        serving = []
        for r in [float(x) for x in a.serve_rates.split(",") if x.strip()]:
            n_req = int(min(200_000, max(20_000, r * 0.4))) if r > 0 else 100_000
            serving.append(serve_run(gt, tree, Q, rhos, r, n_req, a.dtype, inserts=extra))
        if not pre and a.cutover == -1 and tune is not None:
            # the server's three schedules at 50k q/s offered, back to back:
            # one launch per level per step; each step draining the previous
            # step's group in one persistent launch; or each step answering
            # the group it admits (GEMM, then that launch)
            serving_schedules = {}
            for sched in ("levels", "drain", "immediate"):
                serving_schedules[sched] = serve_run(gt, tree, Q, rhos, 50000.0, 20000, a.dtype,
                                                     inserts=extra, seed=5, schedule=sched)
            serving.append({"schedules_at_50k": serving_schedules})

    # the paper's streaming setting, on a tree of its own (after the main tree is freed)
    tree.close()
    tree = None
    served_d512 = None
    if not a.no_serve and not pre and rank == 0 and a.workload == "softmax_n1m_d1000":
        torch.cuda.empty_cache()
        served_d512 = served_d512_run(gt, flush)
    large = None
    if not a.no_large and not pre and rank == 0 and a.workload == "softmax_n1m_d1000":
        torch.cuda.empty_cache()
        large = large_run(gt, flush, not a.no_cpu)
    streaming = None
    if not a.no_stream and rank == 0:
        streaming = streaming_run(gt, ds, a.dtype, 0.9 if 0.9 in (ds.workload.rhos or ()) else a.rho)

    if rank == 0:
        lat = sorted(step_ms)
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(total_ms / a.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": a.dtype, "data": "synthetic softmax features (seeded)",
            "config": {"workload": a.workload, "N": int(N), "d": int(d), "queries_per_step": B,
                       "rho": a.rho, "row_format": a.dtype, "layout": a.layout,
                       "prefix_level": a.prefix_level if pre else None,
                       "cutover": st0["cutover"], "l2": f"flushed between steps "
                       f"({L2_FLUSH_BYTES >> 20} MiB write, outside the timed events)",
                       "parallelism": f"replicas x{ws}",
                       "autotune": None if tune is None else
                       {"cutover": tune["cutover"], "inflight": tune["inflight"],
                        "tile_n": tune["tile_n"], "sample": a.tune_sample or B,
                        "ms": {k: round(v, 3) for k, v in tune["ms"].items()}}},
            "roofline": roof,
            "roofline_other": roof_other,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "e2e_library_csr": e2e_library_csr,
            "gpu_launches": int(sum(s["launches"] for s in stats)),
            "clocks": clk,
            "latency_ms": {"p50": round(lat[len(lat) // 2], 3),
                           "p99": round(lat[min(len(lat) - 1, int(0.99 * len(lat)))], 3),
                           "unit": "per step (one batch)"},
            "stats_per_step": {"tests_per_query": st0["tests"] / B,
                               "gathered_tests_per_query": st0["gathered_tests"] / B,
                               "dense_tests_per_query": st0["dense_tests"] / B,
                               "level_tests_per_query": [round(x / B, 1) for x in
                                                         st0["level_tests"][:st0["cutover"] + 1]]
                               if st0["cutover"] >= 0 else None,
                               "rechecks": st0["rechecks"], "refines": st0["refines"],
                               "results": st0["results"],
                               "micro_batches": st0["micro_batches"], "kernel_ms": km},
            "comparators": comparators,
            "serving": serving,
            "served_n1m_d512": served_d512,
            "served_fixed_groups": served_fixed,
            "large_n10m_fp8": large,
            "streaming": streaming,
            "parity_sample": parity,
            "build_s": round(build_s, 3), "generate_s": round(t_gen, 1),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
