#!/usr/bin/env python
"""Benchmark: RREF via block-iterative PLE of a dense random GF(2) matrix.

One step = one gf2_rref (PLE followed by RREF recovery, every step of the
hot path) of the 65536 x 65536 Bernoulli(1/2) matrix (512 MiB packed), the
paper's Table 2 workload at the size the project targets.  The throughput is
bit-operations per second with the LINPACK-style count
W(m, n, r) = m n r - (m + n) r^2 / 2 + r^3 / 3 (= n^3/3 for a full-rank
square matrix).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (eager elimination, all host cores) on
a bounded sample of the same workload: the first pivot steps of the same
matrix over its full width.  Under torchrun (N > 1) every rank runs an
independent replica on its own GPU (the single-matrix path has no exchange
step); the reference arm runs on rank 0 only.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PLE seconds & Gbitop/s at 32768²/65536² GF(2); batched mats/s; served p99 ms"
UNIT = "Gbitop/s"
N_MAIN = 65536
N_SIDE = 32768
L2_BYTES = 126 * 2**20


def work_bits(m: int, n: int, r: int) -> float:
    return m * n * r - (m + n) * r * r / 2.0 + r ** 3 / 3.0


def bf16_peak(sustained: bool = False):
    """Measured dense bf16 TFLOP/s of this machine's GB300 for the GEMM's roofline:
    the burst figure (a kernel timed alone) or the sustained one (a kernel
    timed inside a long step)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["bf16_tflops_sustained" if sustained else "bf16_tflops"]), "measured"
    except Exception:
        return (1700.0 if sustained else 1900.0), "fallback"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


UPDATE_SOURCES = ("kernels_update.cu", "tables_dev.cuh", "common.cuh")


def update_kernel_digest() -> str:
    h = hashlib.sha256()
    for name in UPDATE_SOURCES:
        with open(os.path.join(ROOT, "paper_1111_6549_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def update_kernel_traffic():
    """DRAM bytes per algorithmic byte of the update kernel, from the committed
    ncu summary, if it was taken on the current kernel sources (else None)."""
    digest = update_kernel_digest()
    for path in glob.glob(os.path.join(ROOT, "profiles", "update_kernel*.md")):
        text = open(path).read()
        mh = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
        mt = re.search(r"dram_bytes_per_algorithmic_byte:\s*([0-9.eE+]+)", text)
        if mh and mt and mh.group(1) == digest:
            return float(mt.group(1)), os.path.relpath(path, ROOT)
    return None, None


def batched_alu_counters():
    """ALU-pipe instructions of one batched_ple_kernel launch on the 4096-matrix
    batch and the pipe's peak per cycle, from the committed ncu summary, if it
    was taken on the current kernel sources (else None)."""
    h = hashlib.sha256()
    for name in ("kernels_batched.cu", "panel_dev.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1111_6549_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    digest = h.hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", "batched_ple_kernel.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    mh = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    mi = re.search(r"alu_inst_per_launch:\s*([0-9.eE+]+)", text)
    mp = re.search(r"alu_peak_inst_per_cycle:\s*([0-9.eE+]+)", text)
    if not (mh and mi and mp) or mh.group(1) != digest:
        return None
    return float(mi.group(1)), float(mp.group(1)), os.path.relpath(path, ROOT)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"gf2_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                maxs.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sms) if sms else None,
                "sm_max_mhz": max(maxs) if maxs else None, "reasons": sorted(reasons),
                "samples": len(sms)}


def dist_setup(n_gpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    return world, rank, local, pg


def max_over_ranks(value: float, pg) -> float:
    """The step time every rank reports is the slowest rank's (gloo all-reduce MAX)."""
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t[0])


def oracle_sample(A: np.ndarray, m: int, n: int, pivots: int, threads: int):
    """Time the oracle's first `pivots` elimination steps over the full width."""
    import oracle
    B = A.copy()
    t0 = time.perf_counter()
    k, _, _ = oracle.ple(B, m, n, max_pivots=pivots, threads=threads)
    dt = time.perf_counter() - t0
    w = sum((m - p) * (n - p) for p in range(k))
    return w, dt, k


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baseline(A: np.ndarray, m: int, n: int, target_s: float = 12.0):
    """The CPU oracle on the bench's host: a bounded sample of the same
    workload on every core, plus single-threaded timings -- the full 2048^2
    RREF (median of 3) and the first pivot steps of the 32768^2 elimination
    over its full width, extrapolated by the work count to the whole
    elimination."""
    import gf2inputs as gi
    import oracle
    threads = os.cpu_count() or 1
    w1, dt1, k1 = oracle_sample(A, m, n, 32, threads)
    per = dt1 / max(k1, 1)
    piv = int(max(64, min(8192, target_s / max(per, 1e-6))))
    w, dt, k = oracle_sample(A, m, n, piv, threads)
    # single thread: 2048^2 RREF via PLE, three runs
    A2 = gi.dense_square(2048)
    t2 = []
    for _ in range(3):
        B = A2.copy()
        t0 = time.perf_counter()
        r2, _ = oracle.rref(B, 2048, 2048, threads=1)
        t2.append(time.perf_counter() - t0)
    ms2 = statistics.median(t2) * 1e3
    # single thread: 32768^2, first pivot steps for about 4 s
    A3 = gi.dense_square(32768)
    wa, da, ka = oracle_sample(A3, 32768, 32768, 8, 1)
    pv = int(max(16, min(4096, 4.0 / max(da / max(ka, 1), 1e-6))))
    ws_, ds_, ks_ = oracle_sample(A3, 32768, 32768, pv, 1)
    rate1 = ws_ / ds_
    full = sum((32768 - p) * (32768 - p) for p in range(32768))
    return {"value": w / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {k} pivot steps of the eager oracle elimination of the same "
                      f"{m}x{n} matrix over its full width ({dt:.1f} s); W = sum_p (m-p)(n-p)",
            "seconds": dt, "cpu_model": cpu_model(), "nproc": threads,
            "single_thread": {
                "rref_2048_ms_median_of_3": ms2, "rank_2048": int(r2),
                "rref_2048_gbitops": work_bits(2048, 2048, int(r2)) / (ms2 / 1e3) / 1e9,
                "elim_32768_sample": f"first {ks_} pivot steps of the 32768x32768 elimination ({ds_:.1f} s)",
                "elim_32768_gbitops": rate1 / 1e9,
                "elim_32768_estimated_s": full / rate1}}


def run_reference(args):
    world, rank, local, pg = dist_setup(args.gpus)
    if rank != 0:
        return 0                      # the CPU reference runs on rank 0 only
    import gf2inputs as gi
    m = n = args.n
    A = gi.dense_square(n)
    threads = os.cpu_count() or 1
    _, dt1, k1 = oracle_sample(A, m, n, 16, threads)
    piv = int(max(32, min(4096, 1.5 / max(dt1 / max(k1, 1), 1e-6))))   # about 1.5 s per step
    for _ in range(args.warmup):
        oracle_sample(A, m, n, piv, threads)
    tw, tt = 0.0, 0.0
    for _ in range(args.steps):
        w, dt, k = oracle_sample(A, m, n, piv, threads)
        tw += w
        tt += dt
    value = tw / tt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": f"rref_via_ple dense Bernoulli(1/2) {m}x{n} GF(2)", "m": m, "n": n,
                       "sample_pivots_per_step": piv},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"first {piv} pivot steps of the eager oracle elimination of "
                                       f"the {m}x{n} matrix over its full width, per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def bench_batched(h, torch, dev, stream, reps: int = 5):
    """The batched workload: 4096 matrices with sides uniform in 64..1024 (25%
    with 10% of rows zeroed) in one gf2_ple_batched call, against the plain
    path (one gf2_ple_async per matrix) on the same GPU."""
    import gf2inputs as gi
    import paper_1111_6549_gb300 as g
    specs = gi.batch_recipe(count=4096)
    mats = [gi.batch_matrix(sp) for sp in specs]
    offs, tot = [], 0
    for A in mats:
        offs.append(tot)
        tot += A.size
    host = np.zeros(tot, dtype=np.uint64)
    for A, o in zip(mats, offs):
        host[o:o + A.size] = A.ravel()
    pristine = torch.from_numpy(host.view(np.int64)).to(dev)
    work = torch.empty_like(pristine)
    maxm = max(sp["m"] for sp in specs)
    P = torch.empty((len(specs), maxm), dtype=torch.int64, device=dev)
    Q = torch.empty((len(specs), maxm), dtype=torch.int64, device=dev)
    R = torch.zeros(len(specs), dtype=torch.int64, device=dev)
    items = []
    for b, (sp, o, A) in enumerate(zip(specs, offs, mats)):
        items.append((work[o:o + A.size].view(A.shape[0], A.shape[1]), sp["m"], sp["n"], P[b], Q[b],
                      R[b:b + 1]))
    def timed(fn):
        work.copy_(pristine)
        fn()                                              # warm-up
        times = []
        for _ in range(reps):
            work.copy_(pristine)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        return statistics.median(times)

    # the C-ABI call with its descriptor array built once (building 4096
    # ctypes descriptors in Python would otherwise dominate the timed region)
    lib, descs = g.load(), h._descs(items)
    h._bind_stream()

    def direct():
        rc = lib.gf2_ple_batched(h._h, descs, len(items))
        assert rc == 0, rc

    t_default = timed(direct)                             # default configuration in every class
    chosen, tune_ms = h.batched_autotune(reps=3)          # per size class, on separate seeded batches
    t = timed(direct)
    plan = h.batched_plan(items)                          # the same launch captured as a CUDA graph
    t_graph = timed(plan.launch)
    plan.close()
    ranks = R.cpu().numpy()
    wsum = sum(work_bits(sp["m"], sp["n"], int(rk)) for sp, rk in zip(specs, ranks))
    nbytes = 2 * 8 * tot
    # plain path: one single-matrix call per matrix
    work.copy_(pristine)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for (A_, m_, n_, P_, Q_, R_) in items:
        h.ple_async(A_, m_, n_, P_, Q_, R_)
    b.record(stream)
    torch.cuda.synchronize()
    t_plain = a.elapsed_time(b)
    hbm, _ = peaks()
    # roofline against the ALU pipe (the batched kernel keeps every matrix in
    # shared memory and L2; its bound is integer logic, not HBM)
    alu = batched_alu_counters()
    clk_mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            clk_mhz = float(json.load(fh).get("sm_max_mhz", clk_mhz))
    except Exception:
        pass
    broof = None
    if alu:
        inst, peak_pc, src = alu
        ach = inst / (t_default / 1e3)          # the counters were taken in the default configuration
        pk = peak_pc * clk_mhz * 1e6
        broof = {"kernel": "batched_ple_kernel", "bound": "alu", "achieved": ach, "peak": pk,
                 "unit": "ALU-pipe warp instructions/s", "frac": ach / pk,
                 "source": f"{src}: ALU-pipe instructions of one launch on this batch and the pipe's peak per "
                           f"cycle (ncu, default configuration), over this run's default-configuration time; "
                           f"peak at {clk_mhz:.0f} MHz"}
    return {"workload": "4096 matrices, m,n ~ U{64..1024}, Bernoulli(1/2), 25% with 10% rows zeroed",
            "roofline": broof,
            "ms": t, "mats_per_s": len(specs) / (t / 1e3), "gbitops": wsum / (t / 1e3) / 1e9,
            "hbm_gbs_algorithmic": nbytes / (t / 1e3) / 1e9,
            "hbm_frac": nbytes / (t / 1e3) / 1e9 / hbm,
            "plain_ms": t_plain, "speedup_vs_plain": t_plain / t, "launches": 1,
            "graph_replay_ms": t_graph, "default_config_ms": t_default,
            "autotune": {"classes": "max(m,n) <= 128, 256, 512, 1024, 2048, 4096",
                         "configs": "0: k=8 x8 tables, 2-word tiles; 1: k=8, 1 word; 2: k=4 x16, 1 word; "
                                    "3: k=4, 2 words; 4: k=4, 4 words",
                         "chosen": chosen, "ms_per_class_and_config": tune_ms}}


def bench_sparse(h, torch, dev, stream, weights=(1, 10, 40, 200), n=10000):
    """The sparse workloads of Section 4's Figure: n x n with exactly w ones per
    row at random columns; RREF via PLE (the paper's "PLE" times include the
    RREF), CUDA-event median of 5 after 2 warm-ups."""
    import gf2inputs as gi
    out = {"workload": f"{n}x{n} GF(2), w nonzeros per row at uniform random distinct columns",
           "paper_context": "Xeon E5345, one core (Figure): 0.97 s at w=1, peak ~1.32 s near w=33-41, "
                            "0.72-0.75 s for w >= 120",
           "points": []}
    for w in weights:
        A = gi.row_weight_matrix(n, n, w)
        pristine = torch.from_numpy(A.view(np.int64)).to(dev)
        work = torch.empty_like(pristine)
        Q = torch.empty(n, dtype=torch.int64, device=dev)
        rk = torch.zeros(1, dtype=torch.int64, device=dev)
        times = []
        for i in range(7):
            work.copy_(pristine)
            if i == 2:
                h.reset_stats()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.rref_async(work, n, n, Q, rk)
            b.record(stream)
            torch.cuda.synchronize()
            if i >= 2:
                times.append(a.elapsed_time(b))
        st = h.stats()
        r = int(rk.cpu()[0])
        t = statistics.median(times)
        out["points"].append({"w": w, "rank": r, "ms": t, "gbitops": work_bits(n, n, r) / (t / 1e3) / 1e9,
                              "block_panel_stripes_per_step": st["panel_fallbacks"] / 5})
    return out


class BusySampler:
    """nvidia-smi utilization.gpu (percent of time a kernel ran) sampled every
    100 ms while active; median and mean of the samples."""

    def __init__(self, index: int):
        self.index = index
        self.path = os.path.join("/tmp", f"gf2_util_{os.getpid()}.csv")
        self.proc = None

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", "--query-gpu=utilization.gpu",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        vals = []
        for line in open(self.path):
            try:
                vals.append(float(line.strip()))
            except ValueError:
                pass
        os.unlink(self.path)
        return {"median_pct": statistics.median(vals), "mean_pct": sum(vals) / len(vals),
                "samples": len(vals)} if vals else None


def bench_served(h, torch, dev, rates=(100, 300, 1000, 3000, 10000, 20000), seconds=2.0, max_jobs=2000,
                 plain_jobs=300, pool_size=48, slots=6):
    """The served solve workload: Poisson arrivals of gf2_solve jobs (n
    log-uniform in 128..16384, 1..64 right-hand sides) through the
    continuous-batching server at each offered rate, `seconds` of arrivals
    (at least 200 and at most max_jobs jobs), against the plain path (one job
    at a time through one handle) on the first plain_jobs arrivals.  Inputs
    come from a pool of pre-generated jobs reused in arrival order.  The GPU's
    busy fraction is sampled during each served run; the knee is the highest
    offered rate the server still keeps up with (jobs/s >= 90 % of it)."""
    import gf2inputs as gi
    import paper_1111_6549_gb300 as g
    pool = []
    for jb in gi.solve_stream_recipe(pool_size, rate=1.0):
        A, B = gi.solve_job_inputs(jb)
        n, nrhs = jb["n"], jb["nrhs"]
        Ap = torch.from_numpy(A.view(np.int64)).pin_memory()
        Bp = torch.from_numpy(B.view(np.int64)).pin_memory()
        Xp = torch.zeros_like(Bp).pin_memory()
        pool.append((n, nrhs, Ap, Bp, Xp))
    max_n = max(p[0] for p in pool)
    out = {"workload": "Poisson arrivals of solve jobs, n log-uniform 128..16384, nrhs U{1..64}",
           "slots": slots, "pool": pool_size, "seconds_per_rate": seconds, "rates": []}
    srv = g.Server(slots=slots, max_n=max_n, max_nrhs=64)
    dA = torch.empty((max_n, gi.words_for(max_n)), dtype=torch.int64, device=dev)
    dB = torch.empty((max_n, 1), dtype=torch.int64, device=dev)
    q = lambda v, f: v[min(len(v) - 1, int(f * len(v)))]
    for rate in rates:
        jobs = int(min(max_jobs, max(200, rate * seconds)))
        arr = gi.solve_stream_recipe(jobs, rate=float(rate), seed=gi.BASE_SEED + 4 + rate)
        with BusySampler(dev.index or 0) as busy:
            t0 = g.Server.clock() + 0.01
            for k, jb in enumerate(arr):
                n, nrhs, Ap, Bp, Xp = pool[k % pool_size]
                while g.Server.clock() < t0 + jb["t"]:
                    pass
                srv.submit(k, Ap, n, Bp, nrhs, Xp)
            srv.drain()
        res = srv.poll(jobs + 8)
        lat = sorted((r[5] - r[3]) * 1e3 for r in res)
        span = max(r[5] for r in res) - min(r[3] for r in res)
        # plain path: one job at a time, same arrivals, the first plain_jobs of them
        lat_p, t_first, t_last = [], None, None
        t0 = g.Server.clock() + 0.01
        for k, jb in enumerate(arr[:plain_jobs]):
            n, nrhs, Ap, Bp, Xp = pool[k % pool_size]
            ta = t0 + jb["t"]
            while g.Server.clock() < ta:
                pass
            now = g.Server.clock()
            t_first = now if t_first is None else t_first
            a = dA[:n, :gi.words_for(n)]
            b = dB[:n, :1]
            a.copy_(Ap, non_blocking=True)
            b.copy_(Bp, non_blocking=True)
            h.solve(a, b, n, nrhs)
            Xp.copy_(b.cpu())
            t_last = g.Server.clock()
            lat_p.append((t_last - ta) * 1e3)
        lat_p.sort()
        out["rates"].append({"rate_per_s": rate, "jobs": len(res),
                             "served": {"p50_ms": q(lat, 0.5), "p99_ms": q(lat, 0.99),
                                        "jobs_per_s": len(res) / span, "gpu_busy": busy.summary()},
                             "plain": {"jobs": len(lat_p), "p50_ms": q(lat_p, 0.5), "p99_ms": q(lat_p, 0.99),
                                       "jobs_per_s": len(lat_p) / (t_last - t_first)}})
    srv.close()
    keep = [r["rate_per_s"] for r in out["rates"] if r["served"]["jobs_per_s"] >= 0.9 * r["rate_per_s"]]
    out["knee_rate_per_s"] = max(keep) if keep else None
    out["capacity_jobs_per_s"] = max(r["served"]["jobs_per_s"] for r in out["rates"])
    out["plain_capacity_jobs_per_s"] = max(r["plain"]["jobs_per_s"] for r in out["rates"])
    return out


def tc_compare(args):
    """Tensor-core (tcgen05) versus table forms of the product and of the PLE
    trailing update, same inputs, CUDA-event medians; prints one JSON line."""
    import torch
    import gf2inputs as gi
    import paper_1111_6549_gb300 as g
    dev = torch.device("cuda", 0)
    h = g.Handle(0)
    stream = torch.cuda.current_stream(dev)
    try:
        h.set_option(g.OPT_MUL_GEMM_FORMAT, 4)
        lib_gemm = True
    except g.GF2Error:
        lib_gemm = False
    h.set_option(g.OPT_MUL_GEMM_FORMAT, 0)

    def timeit(fn, reps=5, pre=None):
        ts = []
        for i in range(reps + 2):
            if pre:
                pre()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            if i >= 2:
                ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    out = {"mode": "tc_compare", "mul": [], "ple": []}
    for (m, k, n) in [(16384, 64, 16384), (16384, 256, 16384), (16384, 512, 16384), (16384, 1024, 16384),
                      (16384, 2048, 16384), (16384, 4096, 16384), (16384, 16384, 16384), (32768, 32768, 32768)]:
        A = torch.from_numpy(gi.bernoulli_matrix(m, k, 1).view(np.int64)).to(dev)
        B = torch.from_numpy(gi.bernoulli_matrix(k, n, 2).view(np.int64)).to(dev)
        C = torch.zeros((m, gi.words_for(n)), dtype=torch.int64, device=dev)
        res, outs = {"m": m, "k": k, "n": n}, {}
        forms = [("table", 0, 0, 0), ("tcgen05_smem_expand", 1, 0, 0), ("own_fp4_gemm", 0, 1, 0)]
        if lib_gemm:
            forms += [("library_fp8_gemm", 0, 1, 8), ("library_fp4_gemm", 0, 1, 4)]
        for name, tc, gk, fmt in forms:
            h.set_option(g.OPT_TC_MUL, tc)
            h.set_option(g.OPT_MUL_GEMM_MIN_K, gk)
            h.set_option(g.OPT_MUL_GEMM_FORMAT, fmt)
            res[name + "_ms"] = timeit(lambda: h.mul(C, A, B, m, k, n))
            res[name + "_tera_and_xor_per_s"] = m * k * n / (res[name + "_ms"] / 1e3) / 1e12
            outs[name] = C.clone()
        res["identical"] = all(bool(torch.equal(outs["table"], v)) for v in outs.values())
        out["mul"].append(res)
    h.set_option(g.OPT_TC_MUL, 0)
    h.set_option(g.OPT_MUL_GEMM_MIN_K, 1024)
    h.set_option(g.OPT_MUL_GEMM_FORMAT, 0)
    for nn in (16384, 32768):
        A = torch.from_numpy(gi.dense_square(nn).view(np.int64)).to(dev)
        Wk = torch.empty_like(A)
        P = torch.empty(nn, dtype=torch.int64, device=dev)
        Q = torch.empty_like(P)
        R = torch.zeros(1, dtype=torch.int64, device=dev)
        res, outs = {"n": nn}, {}
        for tc in (0, 1):
            h.set_option(g.OPT_TC_UPDATE, tc)
            key = "tc" if tc else "table"
            res[key + "_ms"] = timeit(lambda: h.ple_async(Wk, nn, nn, P, Q, R), reps=3, pre=lambda: Wk.copy_(A))
            outs[tc] = Wk.clone()
            h.reset_stats()
            h.set_profiling(1)
            Wk.copy_(A)
            h.ple_async(Wk, nn, nn, P, Q, R)
            torch.cuda.synchronize()
            res[key + "_update_ms"] = h.stats()["update_ms"]
            h.set_profiling(0)
        res["identical"] = bool(torch.equal(outs[0], outs[1]))
        out["ple"].append(res)
    h.set_option(g.OPT_TC_UPDATE, 0)
    # the carriers alone: one CTA per SM issuing back-to-back MMAs of each
    # form on operands already in place (AND-population counts per second;
    # each launch's count is checked against the exact value)
    out["carriers"] = {}
    for name, c, per in (("fp4_tcgen05_mxf4", g.CARRIER_FP4, 64), ("fp4_tcgen05_mxf4nvf4_4x", g.CARRIER_NVF4, 64),
                         ("fp8_tcgen05_f8f6f4", g.CARRIER_FP8, 64), ("b1_mma_sync_and_popc", g.CARRIER_B1, 256)):
        t0 = time.time()
        g.carrier_rate(c, 1024)
        est_ms = (time.time() - t0) * 1e3 / 1024
        lim = (2 ** 31 // 256 - 1) if c == g.CARRIER_B1 else (2 ** 24 // 64 - 1)
        iters = int(min(lim, max(1024, 40.0 / max(est_ms, 1e-6))))
        rates = []
        for _ in range(3):
            rate, cnt = g.carrier_rate(c, iters)
            assert cnt == iters * per, (name, cnt, iters * per)
            rates.append(rate)
        out["carriers"][name] = {"iters": iters, "and_popc_per_s": max(rates)}
    h.close()
    print(json.dumps(out), flush=True)
    return 0


def run_ours(args):
    import torch
    import gf2inputs as gi
    import paper_1111_6549_gb300 as g

    world, rank, local, pg = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    h = g.Handle(local)
    if args.tma:
        h.set_option(g.OPT_TMA_UPDATE, 1)
    if args.paired:
        h.set_option(g.OPT_WIDE_UPDATE, 0)
    if args.ple_block is not None:
        h.set_option(g.OPT_PLE_BLOCK, args.ple_block)
    if args.gemm_format is not None:
        h.set_option(g.OPT_MUL_GEMM_FORMAT, args.gemm_format)
    if args.rref_block is not None:
        h.set_option(g.OPT_RREF_BLOCK, args.rref_block)
    stream = torch.cuda.current_stream(dev)

    m = n = args.n
    A = gi.dense_square(n)
    W = gi.words_for(n)
    pristine = torch.from_numpy(A.view(np.int64)).to(dev)
    work = torch.empty_like(pristine)
    Q = torch.empty(n, dtype=torch.int64, device=dev)

    def step():
        return h.rref_async(work, m, n, Q, rank_dev)

    rank_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    for _ in range(args.warmup):
        work.copy_(pristine)
        step()
    torch.cuda.synchronize()

    # ---- timed region (device time of exactly K steps)
    h.reset_stats()
    h.set_profiling(3)          # every 7th update launch bracketed by events on its stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for i in range(args.steps):
            work.copy_(pristine)
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if pg:
        pg.barrier()
    st = h.stats()
    h.set_profiling(0)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    # one more step, right after the timed ones and not counted in them, with
    # every GEMM launch (and nothing else) bracketed by events: the dominant
    # kernel's live roofline (bracketing them inside the timed steps cost the
    # step about 3 ms of lost overlap)
    h.reset_stats()
    h.set_profiling(5)
    work.copy_(pristine)
    step()
    torch.cuda.synchronize()
    sg = h.stats()
    h.set_profiling(0)
    r = int(rank_dev.cpu()[0])
    # diagnostic pass (not part of the timed steps): every kernel timed
    h.reset_stats()
    h.set_profiling(2)
    diag_steps = 2
    for _ in range(diag_steps):
        work.copy_(pristine)
        step()
    torch.cuda.synchronize()
    sd = h.stats()
    h.set_profiling(0)
    per_step_ms = ms / args.steps
    max_ms = max_over_ranks(ms, pg)
    W_bits = work_bits(m, n, r)
    value = world * args.steps * W_bits / (max_ms / 1e3) / 1e9

    # ---- rooflines, measured live.  The update kernel's object comes first;
    # the dominant kernel (the largest share of the step's launch time: the
    # own FP4 GEMM) becomes `roofline` below.
    hbm, hbm_kind = peaks()
    upd_gbs = st["update_bytes"] / (st["update_ms"] / 1e3) / 1e9 if st["update_ms"] > 0 else None
    upd_per_launch_bytes = st["update_bytes"] / max(st["update_timed_launches"], 1)
    ratio, ratio_src = update_kernel_traffic()
    traffic = ratio * upd_per_launch_bytes if ratio is not None else None
    rp_gbs = ((st["rref_pass_bytes"] / (st["rref_pass_ms"] / 1e3) / 1e9)
              if st["rref_pass_ms"] > 0 and st["rref_pass_bytes"] > 0 else None)
    upd_roof = {"kernel": "update_pipe_kernel (tabulated trailing update of the PLE stripes; "
                          + ("paired 64-byte tiles)" if args.paired else "wide 128-byte tiles)"),
                "bound": "hbm", "achieved": upd_gbs, "peak": hbm, "unit": "GB/s",
                "frac": (upd_gbs / hbm) if upd_gbs else None, "peak_kind": hbm_kind,
                "frac_of_nominal_8000": (upd_gbs / 8000.0) if upd_gbs else None,
                "traffic": traffic, "algorithmic_bytes_per_launch": upd_per_launch_bytes,
                "traffic_source": (f"{ratio_src}: ncu dram__bytes_read.sum + dram__bytes_write.sum of "
                                   f"update_pipe_kernel launches of a 32768^2 PLE, {ratio:.4f} DRAM bytes per "
                                   f"algorithmic byte, times this run's algorithmic bytes per launch")
                                  if ratio else None,
                "launches_per_step": st["update_launches"] / args.steps,
                "timed_launches": st["update_timed_launches"],
                "update_share_of_step_diagnostic": None,
                "kernel_ms_per_step_diagnostic": {k: sd[k + "_ms"] / diag_steps
                                                  for k in ("update", "panel", "prep", "rref_prep", "rref_pass",
                                                            "gemm", "other")},
                "algorithmic_bytes_per_step_diagnostic": sd["update_bytes"] / diag_steps,
                "rref_backsub_kernel": {"kernel": "rref_leaf_kernel (fused back-substitution leaves of the "
                                                  "compact RREF recovery); rref_pass_kernel when the "
                                                  "stripe-wise recovery runs",
                                        "ms_per_step_diagnostic": sd["rref_pass_ms"] / diag_steps,
                                        "launches_per_step": st["rref_pass_launches"] / args.steps,
                                        "achieved_gbs": rp_gbs, "frac": (rp_gbs / hbm) if rp_gbs else None,
                                        "algorithmic_bytes_per_step": st["rref_pass_bytes"] /
                                        max(st["rref_pass_timed_launches"], 1) * st["rref_pass_launches"] /
                                        args.steps},
                "note": "achieved = algorithmic bytes / CUDA-event time of every 7th update launch "
                        "of the timed steps (events on the launching stream); the per-kind breakdown "
                        "comes from a separate pass with every launch bracketed by events (the update "
                        "runs on a side stream beside the panels); the RREF back-substitution kernels "
                        "are counted apart (rref_backsub_kernel: the compact recovery's leaves are bound by "
                        "shared-memory lookups, not HBM, so they report no byte rate)"}
    upd_roof["update_share_of_step_diagnostic"] = (upd_roof["kernel_ms_per_step_diagnostic"]["update"] /
                                                   per_step_ms) if per_step_ms > 0 else None
    g_ms, g_fl = sg["gemm_ms"], sg["gemm_flops"]
    g_tf = g_fl / (g_ms / 1e3) / 1e12 if g_ms > 0 and g_fl > 0 else None
    bf16s, bf16s_kind = bf16_peak(sustained=True)
    fp4s = 6.0 * bf16s
    roofline = {"kernel": "gemm_f4_kernel (own tcgen05 FP4 GEMM: the blocked PLE's trailing products and "
                          "TRSM halves, the compact RREF recovery's joins)",
                "bound": "tensor", "achieved": g_tf, "peak": fp4s, "unit": "TFLOP/s",
                "frac": (g_tf / fp4s) if g_tf else None,
                "peak_kind": f"{bf16s_kind} bf16 sustained x 6 (nominal FP4 13.5 / bf16 2.25 PFLOP/s)",
                "traffic": None,
                "traffic_source": "none for the step's launches (their DRAM bytes depend on each product's "
                                  "shape); a 16384^3 capture is summarised in profiles/gemm_f4_kernel_16384.md",
                "flops_per_launch": g_fl / max(sg["gemm_timed_launches"], 1),
                "flops_per_step": sg["gemm_flops_all"],
                "launches_per_step": sg["gemm_launches"],
                "timed_launches": sg["gemm_timed_launches"],
                "ms_per_step": g_ms,
                "dominance": "largest share of the step's serialised launch time (ncu launch list, "
                             "profiles/launches_rref_65536.md)",
                "note": "achieved = 2 m k n / summed CUDA-event time (events on the launching stream) of "
                        "every GEMM launch of one step of the same workload run right after the timed steps "
                        "with only those launches bracketed (bracketing them inside the timed steps cost "
                        "the step about 3 ms of lost overlap); the update kernel's HBM roofline is "
                        "update_roofline"}

    # ---- the plain paths: (a) the same kernels one stripe after another, no
    # look-ahead; (b) the naive baseline -- one panel per launch and the
    # trailing updates as one-by-one row additions (no tables, no blocked
    # products, no look-ahead)
    plain_ms = naive_ms = None
    if rank == 0 and args.side:
        def once():
            work.copy_(pristine)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b)
        h.set_option(g.OPT_LOOKAHEAD, 0)
        plain_ms = min(once() for _ in range(2))
        h.set_option(g.OPT_NAIVE_UPDATE, 1)
        h.set_option(g.OPT_PLE_BLOCK, 0)
        h.set_option(g.OPT_RREF_BLOCK, 0)
        naive_ms = once()
        h.set_option(g.OPT_NAIVE_UPDATE, 0)
        h.set_option(g.OPT_PLE_BLOCK, -1 if args.ple_block is None else args.ple_block)
        h.set_option(g.OPT_RREF_BLOCK, -1 if args.rref_block is None else args.rref_block)
        h.set_option(g.OPT_LOOKAHEAD, 1)

    # ---- 32768^2 side measurement (same path, a few steps)
    side = {}
    if args.side and rank == 0:
        ns = N_SIDE
        As = gi.dense_square(ns)
        ps = torch.from_numpy(As.view(np.int64)).to(dev)
        ws = torch.empty_like(ps)
        Qs = torch.empty(ns, dtype=torch.int64, device=dev)
        rk = torch.zeros(1, dtype=torch.int64, device=dev)
        for _ in range(3):
            ws.copy_(ps)
            h.rref_async(ws, ns, ns, Qs, rk)
        times = []
        for _ in range(5):
            ws.copy_(ps)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.rref_async(ws, ns, ns, Qs, rk)
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        rs = int(rk.cpu()[0])
        tmed = statistics.median(times)
        # PLE alone at 32768^2
        pt = []
        Ps = torch.empty(ns, dtype=torch.int64, device=dev)
        for _ in range(5):
            ws.copy_(ps)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.ple_async(ws, ns, ns, Ps, Qs, rk)
            b.record(stream)
            torch.cuda.synchronize()
            pt.append(a.elapsed_time(b))
        mt = []
        for _ in range(4):
            ws.copy_(ps)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.rref_m4ri_async(ws, ns, ns, Qs, rk)
            b.record(stream)
            torch.cuda.synchronize()
            mt.append(a.elapsed_time(b))
        side = {"n": ns, "rank": rs, "rref_ms": tmed, "rref_gbitops": work_bits(ns, ns, rs) / tmed / 1e6,
                "m4ri_rref_ms": statistics.median(mt[1:]),
                "ple_ms": statistics.median(pt), "ple_gbitops": work_bits(ns, ns, rs) / statistics.median(pt) / 1e6}
        del ps, ws
    # ---- the own tensor-core GEMM alone: the 32768^3 GF(2) product, against
    # the FP4 peak (the measured bf16 peak times the nominal FP4 / bf16 ratio)
    gemm = None
    if args.side and rank == 0:
        ng = 32768
        Ag = torch.from_numpy(gi.bernoulli_matrix(ng, ng, gi.BASE_SEED + 7).view(np.int64)).to(dev)
        Bg = torch.from_numpy(gi.bernoulli_matrix(ng, ng, gi.BASE_SEED + 8).view(np.int64)).to(dev)
        Cg = torch.empty_like(Ag)
        h.mul(Cg, Ag, Bg, ng, ng, ng)
        gt = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.mul(Cg, Ag, Bg, ng, ng, ng)
            b.record(stream)
            torch.cuda.synchronize()
            gt.append(a.elapsed_time(b))
        gms = statistics.median(gt)
        bf16, bf16_kind = bf16_peak()
        fp4_peak = bf16 * 6.0 if bf16 else None
        tf = 2.0 * ng ** 3 / (gms / 1e3) / 1e12
        gemm = {"kernel": "gemm_f4_kernel (tcgen05 kind::mxf4, TMA-fed, parities from tensor memory)",
                "workload": f"C = A B over GF(2), {ng}^3, Bernoulli(1/2); bit expansion included",
                "ms": gms, "bound": "tensor", "achieved": tf, "unit": "TFLOP/s (2 m k n, exact 0/1 FP4)",
                "peak": fp4_peak, "frac": (tf / fp4_peak) if fp4_peak else None,
                "peak_kind": f"{bf16_kind} bf16 x 6 (nominal FP4 13.5 / bf16 2.25 PFLOP/s)"}
        del Ag, Bg, Cg
    # PLE alone at the main size
    ple_ms = m4ri_ms = None
    if rank == 0 and args.side:
        P = torch.empty(n, dtype=torch.int64, device=dev)
        pt = []
        for _ in range(3):
            work.copy_(pristine)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.ple_async(work, m, n, P, Q, rank_dev)
            b.record(stream)
            torch.cuda.synchronize()
            pt.append(a.elapsed_time(b))
        ple_ms = statistics.median(pt)
        mt = []
        for _ in range(2):
            work.copy_(pristine)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.rref_m4ri_async(work, m, n, Q, rank_dev)
            b.record(stream)
            torch.cuda.synchronize()
            mt.append(a.elapsed_time(b))
        m4ri_ms = min(mt)

    # ---- end to end through the host-buffer C ABI call (pinned buffers)
    e2e = None
    if not args.no_e2e:
        pin = torch.empty((m, W), dtype=torch.int64, pin_memory=True)
        pin_src = torch.from_numpy(A.view(np.int64))
        Qh = torch.empty(n, dtype=torch.int64, pin_memory=True)
        pin.copy_(pin_src)
        h.rref_host(pin, m, n, Qh)          # warm-up
        tt = 0.0
        steps_e2e = max(1, min(args.steps, 5))
        for _ in range(steps_e2e):
            pin.copy_(pin_src)
            t0 = time.perf_counter()
            h.rref_host(pin, m, n, Qh)
            tt += time.perf_counter() - t0
        e2e = {"value": steps_e2e * W_bits / tt / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": m * W * 8, "d2h_bytes_per_step": m * W * 8 + n * 8 + 8,
               "steps": steps_e2e, "ms_per_step": tt / steps_e2e * 1e3,
               "call": "gf2_rref_host (pinned host buffers; H2D, PLE, RREF, D2H, synchronous)"}

    batched = None
    if rank == 0 and not args.no_batch:
        batched = bench_batched(h, torch, dev, stream)
    sparse = None
    if rank == 0 and not args.no_sparse:
        sparse = bench_sparse(h, torch, dev, stream)
    served = None
    if rank == 0 and not args.no_serve:
        served = bench_served(h, torch, dev, seconds=args.served_seconds, slots=args.served_slots,
                              max_jobs=int(1000 * args.served_seconds))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(A, m, n)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": f"rref_via_ple dense Bernoulli(1/2) {m}x{n} GF(2), "
                                       f"{m * W * 8 / 2**20:.0f} MiB packed",
                           "m": m, "n": n, "rank": r, "stripe_columns": 64,
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "l2": f"inputs ({m * W * 8 / 2**20:.0f} MiB) larger than L2; fresh copy restored "
                                 "before each step",
                           "seconds_per_step": max_ms / args.steps / 1e3,
                           "ple_only_ms": ple_ms, "m4ri_rref_ms": m4ri_ms, "side_32768": side,
                           "plain_path_ms": naive_ms,
                           "speedup_vs_plain_path": (naive_ms / (max_ms / args.steps)) if naive_ms else None,
                           "plain_path": "naive baseline: one panel per launch per 64-column stripe, trailing "
                                         "updates as one-by-one row additions (no tables, no blocked products, "
                                         "no look-ahead)",
                           "no_lookahead_ms": plain_ms},
                "roofline": roofline, "update_roofline": upd_roof, "gemm_roofline": gemm, "cpu_baseline": cpu, "e2e": e2e, "batched": batched,
                "served": served,
                "sparse": sparse,
                "rref_65536_ms": max_ms / args.steps if n == 65536 else None,
                "ple_65536_ms": ple_ms if n == 65536 else None,
                "rref_32768_ms": side.get("rref_ms"), "ple_32768_ms": side.get("ple_ms"),
                "m4ri_32768_ms": side.get("m4ri_rref_ms"),
                "gpu_launches": st["kernel_launches"], "clocks": clk.summary(),
                "panel_fallbacks": st["panel_fallbacks"], "wall_s_timed": t_wall}
        print(json.dumps(line), flush=True)
    h.close()
    return 0


def run_only(args):
    """One call of one workload at --size (default 32768), for profilers: ple /
    rref (dense Bernoulli(1/2) square), mul (--size^3 product), batched (the
    4096-matrix batch, two calls).  Prints one line, no timing claims."""
    import torch
    import gf2inputs as gi
    import paper_1111_6549_gb300 as g
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    h = g.Handle(0)
    n = args.n if args.n is not None else N_SIDE
    if args.only in ("ple", "rref"):
        A = torch.from_numpy(gi.dense_square(n).view(np.int64)).to(dev)
        Q = torch.empty(n, dtype=torch.int64, device=dev)
        if args.only == "ple":
            P = torch.empty(n, dtype=torch.int64, device=dev)
            r = h.ple(A, n, n, P, Q)
        else:
            r = h.rref(A, n, n, Q)
        print(f"{args.only} {n}x{n} rank {r}")
    elif args.only == "mul":
        Ag = torch.from_numpy(gi.bernoulli_matrix(n, n, gi.BASE_SEED + 7).view(np.int64)).to(dev)
        Bg = torch.from_numpy(gi.bernoulli_matrix(n, n, gi.BASE_SEED + 8).view(np.int64)).to(dev)
        Cg = torch.empty_like(Ag)
        for _ in range(2):
            h.mul(Cg, Ag, Bg, n, n, n)
        torch.cuda.synchronize()
        print(f"mul {n}^3 done")
    else:
        specs = gi.batch_recipe(count=4096)
        mats = [gi.batch_matrix(sp) for sp in specs]
        offs, tot = [], 0
        for A in mats:
            offs.append(tot)
            tot += A.size
        host = np.zeros(tot, dtype=np.uint64)
        for A, o in zip(mats, offs):
            host[o:o + A.size] = A.ravel()
        work = torch.from_numpy(host.view(np.int64)).to(dev)
        maxm = max(sp["m"] for sp in specs)
        P = torch.empty((len(specs), maxm), dtype=torch.int64, device=dev)
        Q = torch.empty((len(specs), maxm), dtype=torch.int64, device=dev)
        R = torch.zeros(len(specs), dtype=torch.int64, device=dev)
        items = [(work[o:o + A.size].view(A.shape[0], A.shape[1]), sp["m"], sp["n"], P[b], Q[b], R[b:b + 1])
                 for b, (sp, o, A) in enumerate(zip(specs, offs, mats))]
        for _ in range(2):
            h.ple_batched(items)
        torch.cuda.synchronize()
        print(f"batched 4096 matrices, rank sum {int(R.sum())}")
    h.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", dest="n", type=int, default=None)
    ap.add_argument("--no-side", dest="side", action="store_false")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-sparse", action="store_true")
    ap.add_argument("--only", choices=("ple", "rref", "mul", "batched"), default=None,
                    help="one call of one workload at --size (default 32768) for a profiler; no timing")
    ap.add_argument("--served-seconds", type=float, default=2.0,
                    help="seconds of Poisson arrivals per offered rate in the served sweep (30: the full sweep)")
    ap.add_argument("--served-slots", type=int, default=6, help="execution slots of the solve server")
    ap.add_argument("--gemm-format", type=int, default=None, choices=(0, 8, 4),
                    help="GF(2) product form in the blocked steps: 0 the own tcgen05 FP4 GEMM (default), "
                         "4 / 8 the library GEMM (builds with GF2_WITH_CUBLASLT=1 only)")
    ap.add_argument("--rref-block", type=int, default=None,
                    help="base block width of the recursive RREF recovery (0: flat; default: the library's)")
    ap.add_argument("--ple-block", type=int, default=None,
                    help="PLE column block for the blocked trailing update (GF2_OPT_PLE_BLOCK)")
    ap.add_argument("--paired", action="store_true",
                    help="table updates in the paired 64-byte-tile form (GF2_OPT_WIDE_UPDATE = 0)")
    ap.add_argument("--tma", action="store_true",
                    help="run the update in its TMA-staged form (GF2_OPT_TMA_UPDATE)")
    ap.add_argument("--tc-compare", action="store_true",
                    help="only compare the tensor-core and table forms (product, PLE update)")
    args = ap.parse_args()
    if args.only:
        return run_only(args)
    if args.n is None:
        args.n = N_MAIN
    if args.impl == "reference":
        return run_reference(args)
    if args.tc_compare:
        return tc_compare(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
