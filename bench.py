"""Benchmark of the sketch-and-solve least-squares path on GB300.

Workload (the configuration the headline metric is quoted on): dense
A = G diag(sigma) Q of 1,048,576 x 256 FP32 with kappa = 1e6, b = A x_true +
1e-4 noise, CountSketch with d = 1024.  One step = one complete solve through
the C ABI: sketch [A | b] -> FP64 Householder QR -> back-solve ->
R-preconditioned refinement until eta(x) = ||A^T r|| / (||A||_F ||r||) <= 1e-6.

Reported: LS solves/s (value), p50/p99 solve latency, the sketch-apply HBM
bandwidth and the dominant kernel's roofline fraction (per-kernel CUDA-event
times measured on the launch stream inside the timed region), an end-to-end
figure with host-resident inputs copied in every step, and the CPU oracle timed
on a bounded sample of the same workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): each rank solves its own independent problem (replicas,
weak scaling); timing is the max over ranks.
"""
import argparse
import ctypes as C
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sketch-apply HBM GB/s vs peak; LS solves/s + p99 latency at rel-res ≤1e-6"
M, N, D, KAPPA, NOISE, TOL = 1 << 20, 256, 1024, 1e6, 1e-4, 1e-6
DATA_SEED, SKETCH_SEED = 1002, 1
FP64_PEAK_TFLOPS = 1.25      # GB300 nominal FP64 (vector and tensor), for ALU-bound kernels
WORKLOAD = ("dense FP32 A = G diag(sigma) Q, 1048576 x 256, kappa 1e6, noise 1e-4; CountSketch d=1024; "
            "sketch-and-solve then R-preconditioned refinement to eta <= 1e-6")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), float(j["bf16_tflops"]), "measured"
    return 6800.0, 1900.0, "fallback"


def read_stream_gbs(dev):
    """Read-only HBM stream on this GPU (torch sum over 4 GiB of FP32, best of 5),
    reported beside the copy-bandwidth peak: the passes only read A."""
    import torch
    x = torch.ones(1 << 30, dtype=torch.float32, device=dev)
    best = float("inf")
    for _ in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        x.sum()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del x
    torch.cuda.empty_cache()
    return (1 << 32) / (best / 1e3) / 1e9


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """SM clock, its maximum, power and the clock event reasons of one GPU, from
    an nvidia-smi subprocess polling every 40 ms (a separate process, so the
    benchmark's own host thread is not slowed).  Each sample carries
    nvidia-smi's timestamp; the timed region's samples are those between mark()
    and stop().  Output is line-buffered (stdbuf) and nvidia-smi is stopped with
    SIGINT so that no sample is lost.  The samples are kept in
    $SNSOLVE_BENCH_OUT/clocks_rankN.csv (default: bench_out/ beside bench.py)."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.t_mark = None
        out = os.environ.get("SNSOLVE_BENCH_OUT", os.path.join(ROOT, "bench_out"))
        self.path = os.path.join(out, f"clocks_rank{device_index}.csv")

    def start(self):
        """Starts sampling and returns once the first sample is written, so
        nvidia-smi's start-up (driver queries) stays outside the timed region."""
        import shutil
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            cmd = ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                   "-lms", "40"]
            if shutil.which("stdbuf"):
                cmd = ["stdbuf", "-oL"] + cmd
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 3.0 and self._lines() < 1:
            time.sleep(0.01)

    def _lines(self):
        try:
            with open(self.path) as f:
                return sum(1 for _ in f)
        except OSError:
            return 0

    def mark(self):
        """Marks the start of the timed region."""
        self.t_mark = time.time()

    def stop(self):
        if self.proc is None:
            return None
        t_end = time.time()
        time.sleep(0.05)                       # the sample that covers the region's end
        import signal
        try:
            self.proc.send_signal(signal.SIGINT)
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            return clock_summary(f.read().splitlines(), self.t_mark if self.t_mark is not None else t_end, t_end)


def clock_summary(lines, t0, t1):
    """Summary of nvidia-smi sample lines (ClockSampler.Q order, csv, no units)
    taken in the wall-clock interval [t0, t1]: median SM clock, maximum clock,
    the slowdown reasons seen, sample counts.  Falls back to the last sample
    when none lies in the interval."""
    import datetime
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 10:
            continue
        try:
            ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            continue
        rows.append((ts, parts))
    if not rows:
        return None
    region = [p for ts, p in rows if t0 <= ts <= t1]
    use = region if region else [rows[-1][1]]
    sm = [float(r[2]) for r in use if re.match(r"^[0-9.]+$", r[2])]
    mx = [float(r[3]) for r in use if re.match(r"^[0-9.]+$", r[3])]
    pw = [float(r[4]) for r in use if re.match(r"^[0-9.]+$", r[4])]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in use for i in range(4) if r[6 + i].lower().startswith("active")})
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(use), "samples_in_region": len(region),
            "power_w_median": float(np.median(pw)) if pw else None, "source": "nvidia-smi, 40 ms period"}


# ------------------------------------------------------------------ workload
def make_inputs(rank, device):
    import torch
    from synth import ill_conditioned_problem
    A, b, _ = ill_conditioned_problem(M, N, seed=DATA_SEED + 1000 * rank, kappa=KAPPA, noise=NOISE)
    return A, b


def max_over_ranks(ms, device, world):
    """The slowest rank's time (the step is done when every replica is done)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(steps, world, max_ms):
    """Solves per second of the whole job: every rank solved `steps` problems."""
    return steps * world / (max_ms / 1e3)


def kernel_profile(L):
    nk = L.snsolve_profile_num_kernels()
    ms = (C.c_double * nk)()
    cnt = (C.c_uint64 * nk)()
    L.snsolve_profile_read(ms, cnt, nk)
    return {L.snsolve_profile_kernel_name(i).decode(): (ms[i], cnt[i]) for i in range(nk) if cnt[i]}


def algorithmic(name, m, n, d):
    """(bound, algorithmic bytes or flops per launch) of a kernel class."""
    if name in ("normal_pass",):
        return "hbm", m * n * 4.0
    if name in ("resid_pass",):
        return "hbm", m * (n + 1) * 4.0
    if name in ("cs_gather_dense", "cs_stream_dense", "cs_sort_blocks", "cs_apply"):
        return "hbm", m * (n + 1) * 4.0
    if name in ("qr_house",):
        q = n + 1
        return "alu", 2.0 * d * q * q - 2.0 / 3.0 * q ** 3
    return None, None


TRAFFIC_JSON = os.path.join(ROOT, "profiles", "traffic.json")
_UNIT = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12,
         "KB": 1e3, "MB": 1e6, "GB": 1e9, "B": 1.0}


def traffic_table():
    """Per-launch DRAM bytes (read + write) of kernel classes from ncu captures,
    as recorded by `bench.py --record-traffic` in profiles/traffic.json, with the
    library source hash each was taken at: {name: (bytes, source hash)}."""
    if not os.path.exists(TRAFFIC_JSON):
        return {}
    with open(TRAFFIC_JSON) as f:
        j = json.load(f)
    return {k: (float(v["dram_bytes_per_full_launch"]), v["source"]) for k, v in j.items()}


def record_traffic(raw_csv, name, kernel_regex, read_scale, write_scale, case, command):
    """Reads the raw page of an ncu capture (`ncu -i X.ncu-rep --page raw --csv`),
    takes the launches whose kernel name matches kernel_regex, and records their
    mean dram__bytes_read.sum * read_scale + dram__bytes_write.sum * write_scale
    (the scales carry a small captured case to a full-size launch) under `name`
    in profiles/traffic.json, with the current source hash."""
    import csv
    with open(raw_csv) as f:
        rows = list(csv.reader(f))
    hdr = rows[0]
    ki = hdr.index("Kernel Name")
    ri, wi = hdr.index("dram__bytes_read.sum"), hdr.index("dram__bytes_write.sum")
    units = rows[1] if rows[1][ri] in _UNIT or rows[1][ri] == "" else None
    body = rows[2:] if units else rows[1:]

    def val(row, i):
        return float(row[i].replace(",", "")) * (_UNIT.get(units[i], 1.0) if units else 1.0)

    sel = [r for r in body if len(r) > max(ki, ri, wi) and re.search(kernel_regex, r[ki])]
    if not sel:
        raise SystemExit(f"no launch of {kernel_regex} in {raw_csv}")
    rd = float(np.mean([val(r, ri) for r in sel]))
    wr = float(np.mean([val(r, wi) for r in sel]))
    j = {}
    if os.path.exists(TRAFFIC_JSON):
        with open(TRAFFIC_JSON) as f:
            j = json.load(f)
    j[name] = {"dram_bytes_per_full_launch": rd * read_scale + wr * write_scale, "source": source_hash(),
               "captured_read_bytes": rd, "captured_write_bytes": wr, "read_scale": read_scale,
               "write_scale": write_scale, "launches_averaged": len(sel), "captured_case": case,
               "command": command}
    with open(TRAFFIC_JSON, "w") as f:
        json.dump(j, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps({name: j[name]}))


def source_hash():
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2409_14309_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:12]


# ------------------------------------------------------------------ CPU oracle
def oracle_solve_sample(A, b, rows):
    """The oracle's sketch-and-solve + SAP on the first `rows` rows; returns the
    seconds of (sketch, qr+solve, iterations), the iteration count and the
    oracle's sketch (SA, Sb)."""
    from oracle import sketch as OS
    from oracle import solve as OL
    As = A[:rows].astype(np.float64)
    bs = b[:rows].astype(np.float64)
    t0 = time.perf_counter()
    SA = OS.countsketch_apply(As, D, SKETCH_SEED)
    Sb = OS.countsketch_apply(bs, D, SKETCH_SEED)
    t1 = time.perf_counter()
    xhat, R, _ = OL.sketch_and_solve(SA, Sb)
    t2 = time.perf_counter()
    x, it, _ = OL.lsqr_preconditioned(As, bs, R, xhat, tol=TOL, max_iter=500)
    t3 = time.perf_counter()
    return t1 - t0, t2 - t1, t3 - t2, it, SA, Sb


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_errors(A, b, SA, Sb, x_gpu, eta_gpu):
    """The GPU solution's errors against the FP64 oracle, outside any timed
    region: the oracle's eta(x) over the whole matrix, and the forward error and
    residual excess against x* from the oracle's FP64 sketch-and-precondition run
    to 1e-14 (its fixed point is x*, pinned by the oracle's tests)."""
    from oracle import solve as OL
    A64, b64 = A.astype(np.float64), b.astype(np.float64)
    t0 = time.perf_counter()
    x_star, it, est, _ = OL.sketch_and_precondition(A64, b64, SA, Sb, tol=1e-14, max_iter=500)
    r_star = np.linalg.norm(b64 - A64 @ x_star)
    r_gpu = np.linalg.norm(b64 - A64 @ x_gpu)
    return {"eta_oracle_fp64": float(OL.eta(A64, b64, x_gpu)), "eta_reported_by_solver": float(eta_gpu),
            "forward_error_vs_x_star": float(np.linalg.norm(x_gpu - x_star) / np.linalg.norm(x_star)),
            "residual_excess": float(r_gpu / r_star - 1.0),
            "x_star": f"oracle FP64 sketch-and-precondition (LSQR on A R^-1) to {est:.1e} in {it} iterations",
            "seconds": time.perf_counter() - t0}


def cpu_baseline(A, b, steps=2, x_gpu=None, eta_gpu=None):
    """The oracle as it stands on the host cores: full-size solves of the
    workload (about 10-20 s of CPU work in total).  With x_gpu, also the GPU
    solution's errors against the oracle (untimed)."""
    ts = []
    its = 0
    SA = Sb = None
    for _ in range(max(1, steps)):
        t_sk, t_qr, t_it, its, SA, Sb = oracle_solve_sample(A, b, M)
        ts.append(t_sk + t_qr + t_it)
    t = float(np.median(ts))
    out = {"value": 1.0 / t, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
           "sample": f"{len(ts)} complete solves of the workload by the oracle (numpy FP64: row-scatter "
                     f"CountSketch, Householder QR, R-preconditioned LSQR to eta<=1e-6, {its} iterations); "
                     f"median time"}
    if x_gpu is not None:
        out["oracle_check"] = oracle_errors(A, b, SA, Sb, x_gpu, eta_gpu)
    return out


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cs-variant", default="auto", choices=["auto", "sorted", "stream"])
    ap.add_argument("--workload", default="solve",
                    choices=["solve", "batched", "served", "sketches", "latency", "csr", "profile-case", "paper"])
    ap.add_argument("--paper-m", default="5000,20000,100000,250000,500000,1000000",
                    help="paper workload: rows of A to sweep")
    ap.add_argument("--paper-passes", type=int, default=64, help="paper workload: passes budget per solve")
    ap.add_argument("--requests", type=int, default=20000)
    ap.add_argument("--rates", default="0.5,0.8,1.0,1.5",
                    help="served workload: arrival rates as multiples of the one-slot capacity")
    ap.add_argument("--sweep-requests", type=int, default=4000,
                    help="served workload: requests at the rates below the highest one")
    ap.add_argument("--gauss-terms", default="auto", choices=["auto", "1", "2", "3"],
                    help="profile-case gaussian: BF16 terms of [A | b]")
    ap.add_argument("--case", default="solve", choices=["solve", "countsketch", "srht", "gaussian", "csr", "batched"],
                    help="profile-case: which small case to run")
    ap.add_argument("--latency-solves", type=int, default=200,
                    help="solves of the separate latency pass (p50/p99)")
    ap.add_argument("--record-traffic", nargs=7,
                    metavar=("RAW_CSV", "NAME", "KERNEL_REGEX", "READ_SCALE", "WRITE_SCALE", "CASE", "COMMAND"),
                    help="record an ncu capture's DRAM bytes per launch in profiles/traffic.json and exit")
    args = ap.parse_args()
    if args.record_traffic:
        r = args.record_traffic
        return record_traffic(r[0], r[1], r[2], float(r[3]), float(r[4]), r[5], r[6])
    warm = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "sketches":
        return run_sketches(args)
    if args.workload == "latency":
        return run_latency(args)
    if args.workload == "csr":
        return run_csr(args)
    if args.workload == "profile-case":
        return run_profile_case(args)
    if args.workload == "paper":
        return run_paper(args)

    import torch
    import torch.distributed as dist
    import paper_2409_14309_gb300 as sns
    from paper_2409_14309_gb300 import abi

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    ctx = sns.Context(local)
    L = abi.lib()

    A_h, b_h = make_inputs(rank, dev)
    A = torch.from_numpy(A_h).to(dev)
    b = torch.from_numpy(b_h).to(dev)
    prob = sns.dense_problem(A, b)
    op = sns.opts(D, "countsketch", SKETCH_SEED, args.cs_variant, tol=TOL)
    ws = torch.empty(ctx.lstsq_workspace(prob, op), dtype=torch.uint8, device=dev)
    x = torch.empty(N, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up
    for _ in range(warm):
        _, info = ctx.lstsq_problem(prob, op, x=x, ws=ws)
    torch.cuda.synchronize()

    # timed region: K solves, no instrumentation; clocks sampled
    clk = ClockSampler(local)
    launches0 = L.snsolve_launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    infos = []
    clk.start()
    barrier()
    torch.cuda.synchronize()
    clk.mark()
    ev[0].record(stream)
    for k in range(args.steps):
        _, info = ctx.lstsq_problem(prob, op, x=x, ws=ws)
        infos.append((info.status, info.iters, info.outer, info.eta))
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    launches = L.snsolve_launch_count() - launches0
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = max_over_ranks(ev[0].elapsed_time(ev[-1]), dev, world)
    value = whole_job_rate(args.steps, world, total_ms)

    # latency: a separate pass of single solves, one event pair around each,
    # no clock sampling and no per-kernel events
    nlat = max(args.latency_solves, 1)
    lev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nlat)]
    for k in range(nlat):
        lev[k][0].record(stream)
        ctx.lstsq_problem(prob, op, x=x, ws=ws)
        lev[k][1].record(stream)
    torch.cuda.synchronize()
    lat_ms = sorted(e0.elapsed_time(e1) for e0, e1 in lev)

    # the same K solves again with a CUDA event pair around every launch (on
    # the launching stream): per-kernel durations for the roofline.  Kept out
    # of the region above because ~200 event records per solve add gaps.
    L.snsolve_profile(1)
    kernel_profile(L)                              # clear
    torch.cuda.synchronize()
    passes_run = 0
    for k in range(args.steps):
        _, info2 = ctx.lstsq_problem(prob, op, x=x, ws=ws)
        passes_run += info2.iters
    torch.cuda.synchronize()
    prof = kernel_profile(L)
    L.snsolve_profile(0)
    if "normal_pass" in prof:
        # a refinement cycle that has converged leaves its remaining pass
        # launches empty: count the passes that ran (their time includes the
        # empty launches, so the rate is if anything understated)
        prof["normal_pass"] = (prof["normal_pass"][0], passes_run)

    # roofline of the dominant kernel and of the sketch apply
    hbm_peak, bf16_peak, peak_kind = peaks()
    read_gbs = read_stream_gbs(dev) if rank == 0 else None
    traffic = traffic_table()
    src = source_hash()
    dom = max(prof.items(), key=lambda kv: kv[1][0])[0] if prof else None

    def roof(name):
        ms, cnt = prof[name]
        bound, amount = algorithmic(name, M, N, D)
        if bound is None:
            return None
        avg_s = ms / cnt / 1e3
        tr = traffic.get(name)
        tval = tr[0] if tr and tr[1] == src else None
        if bound == "hbm":
            ach = amount / avg_s / 1e9
            return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                    "frac": ach / hbm_peak, "traffic": tval, "peak_kind": f"{peak_kind} copy bandwidth",
                    "read_stream_GBps": read_gbs, "frac_of_read_stream": ach / read_gbs if read_gbs else None,
                    "algorithmic_bytes_per_launch": amount, "avg_launch_ms": avg_s * 1e3,
                    "launches_per_step": cnt / args.steps}
        ach = amount / avg_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": tval, "peak_kind": "GB300 nominal FP64",
                "algorithmic_flops_per_launch": amount, "avg_launch_ms": avg_s * 1e3,
                "launches_per_step": cnt / args.steps}

    # the single-launch plan and its dependent gather are timed as one span
    # ("cs_apply": one event pair, so no event separates the pair); other
    # variants as the sum of their kernels
    if "cs_apply" in prof:
        sk_names = ["cs_apply"]
        sk_ms, sk_n = prof["cs_apply"]
    else:
        sk_names = [k for k in ("cs_sort_blocks", "cs_gather_dense", "cs_stream_dense") if k in prof]
        sk_ms = sum(prof[k][0] for k in sk_names)
        sk_n = max([prof[k][1] for k in ("cs_gather_dense", "cs_stream_dense") if k in prof] or [0])
    sketch = None
    if sk_n:
        gbs = M * (N + 1) * 4.0 / (sk_ms / sk_n / 1e3) / 1e9
        sketch = {"kernels": sk_names, "variant": args.cs_variant, "bound": "hbm", "achieved": gbs,
                  "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak, "avg_apply_ms": sk_ms / sk_n,
                  "algorithmic_bytes": M * (N + 1) * 4.0}

    # end to end: host-resident inputs (pinned), copied in every step and solved
    # through the public API, the solution read back every step.  Two device
    # buffers and a copy stream: step k+1's inputs are copied while step k is
    # solved, as a serving loop would do (the host-to-device link, ~210 GB/s
    # here, otherwise serialises with the solve).  The timed region starts
    # with the first step's copy, which nothing overlaps (pipeline fill).
    e2e = None
    if not args.no_e2e:
        Ah = torch.from_numpy(A_h).pin_memory()
        bh = torch.from_numpy(b_h).pin_memory()
        xh = torch.empty(N, dtype=torch.float64).pin_memory()
        bufs = [(torch.empty_like(A), torch.empty_like(b)) for _ in range(2)]
        copy_st = torch.cuda.Stream(device=dev)
        done_copy = [torch.cuda.Event() for _ in range(2)]
        free_buf = [torch.cuda.Event() for _ in range(2)]

        def issue_copy(k):
            Ad, bd = bufs[k % 2]
            with torch.cuda.stream(copy_st):
                copy_st.wait_event(free_buf[k % 2])
                Ad.copy_(Ah, non_blocking=True)
                bd.copy_(bh, non_blocking=True)
                done_copy[k % 2].record(copy_st)

        def solve(k):
            Ad, bd = bufs[k % 2]
            stream.wait_event(done_copy[k % 2])
            xx, _ = ctx.lstsq(Ad, bd, D, seed=SKETCH_SEED, tol=TOL, ws=ws)
            free_buf[k % 2].record(stream)
            xh.copy_(xx, non_blocking=True)

        for k in range(2):                       # warm-up of the whole loop
            issue_copy(k)
            solve(k)
        torch.cuda.synchronize()
        ke = max(3, args.steps)                  # the same step count as the device-timed loop
        barrier()
        t0 = time.perf_counter()
        issue_copy(0)
        for k in range(ke):
            if k + 1 < ke:
                issue_copy(k + 1)
            solve(k)
        torch.cuda.synchronize()
        ems = (time.perf_counter() - t0) * 1e3
        barrier()
        ems = max_over_ranks(ems, dev, world)
        e2e = {"value": whole_job_rate(ke, world, ems), "unit": "solves/s",
               "h2d_bytes_per_step": int(A.numel() * 4 + b.numel() * 4), "d2h_bytes_per_step": int(N * 8),
               "pipelined": "step k+1's host-to-device copy overlaps step k's solve (two device buffers, a copy "
                            "stream); every step copies its inputs and reads back its solution",
               "timer": "host wall clock around the loop, after a device synchronize on both sides"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        _, info = ctx.lstsq_problem(prob, op, x=x, ws=ws)
        cpu = cpu_baseline(A_h, b_h, x_gpu=x.cpu().numpy(), eta_gpu=info.eta)

    if rank == 0:
        def pct(v, q):
            return v[min(len(v) - 1, int(math.ceil(q * len(v))) - 1)]
        st = sorted(step_ms)
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": warm, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 passes + f64 QR/solves", "data": "synthetic",
            "config": {"workload": WORKLOAD, "m": M, "n": N, "d": D, "kappa": KAPPA, "tol_eta": TOL,
                       "sketch": "countsketch", "parallelism": f"replicas x{world}",
                       "l2": "A is 1.08 GB > 129 MB L2 and is streamed every pass; no flush needed"},
            "p50_ms": pct(lat_ms, 0.50), "p99_ms": pct(lat_ms, 0.99),
            "latency": {"solves": nlat, "p50_ms": pct(lat_ms, 0.50), "p99_ms": pct(lat_ms, 0.99),
                        "max_ms": lat_ms[-1],
                        "pass": "separate pass after the timed region: one CUDA event pair around each solve, no "
                                "clock sampling, no per-kernel events"},
            "p50_ms_timed_region": pct(st, 0.50), "p99_ms_timed_region": pct(st, 0.99),
            "step_ms": [round(t, 4) for t in step_ms],
            "kernel_timing": "per-launch CUDA events on the launching stream, in a second pass of the same "
                             "K solves; value and latencies come from the uninstrumented pass",
            "roofline": roof(dom) if dom else None,
            "sketch_apply": sketch,
            "kernels": {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
                        for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])},
            "solve": {"status": [i[0] for i in infos][-1], "iters": infos[-1][1], "outer": infos[-1][2],
                      "eta": infos[-1][3]},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
            "source": src,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()

# ------------------------------------------------------------------ paper workload
def _paper_device(m, n, kappa, beta, gen, dev):
    """The paper's benchmark problem generated on the device (FP64): A = U diag(sigma)
    V^T, x* = w / ||w||, r* = beta P z / ||P z|| with P = I - U U^T, b = A x* + r*."""
    import torch
    G = torch.randn(m, n, generator=gen, device=dev, dtype=torch.float64)
    U, Rr = torch.linalg.qr(G)
    U = U * torch.sign(torch.diagonal(Rr))[None, :]
    del G, Rr
    V = _haar(n, gen, dev)
    sig = kappa ** (-torch.arange(n, device=dev, dtype=torch.float64) / max(n - 1, 1))
    A = (U * sig[None, :]) @ V.T
    w = torch.randn(n, generator=gen, device=dev, dtype=torch.float64)
    x_star = w / torch.linalg.norm(w)
    z = torch.randn(m, generator=gen, device=dev, dtype=torch.float64)
    for _ in range(2):
        z -= U @ (U.T @ z)
    del U
    b = A @ x_star + beta * z / torch.linalg.norm(z)
    return A.contiguous(), b, x_star


def run_paper(args):
    """The paper's benchmark setup (Sec. 3.1, after Epperly et al. 2024) on one GPU:
    FP64 A of m x 1000, kappa 1e10, beta 1e-10, m swept from 5e3 to 1e6.  Per m:
    sketch-and-precondition (SAP), sketch-and-apply (SAA) and the unpreconditioned
    iteration (R = I; the role of the paper's LSQR baseline), each with the same
    budget of passes over the matrix, timed with CUDA events; forward error
    ||x - x*|| / ||x*|| and residual error ||A (x - x*)|| / beta against the known
    x* (the paper's Figs. 3-5 quantities).  CountSketch d = 4n."""
    import torch
    import paper_2409_14309_gb300 as sns
    dev = torch.device("cuda", 0)
    ctx = sns.Context(0)
    n, kappa, beta = 1000, 1e10, 1e-10
    budget = args.paper_passes
    ms = [int(v) for v in args.paper_m.split(",")]
    rows = []
    for m in ms:
        gen = torch.Generator(device=dev)
        gen.manual_seed(4000 + m)
        A, b, x_star = _paper_device(m, n, kappa, beta, gen, dev)
        torch.cuda.synchronize()
        prob = sns.dense_problem(A, b)
        row = {"m": m}
        for label, meth, pre in (("sap", "sap", True), ("saa", "saa", True), ("unpreconditioned", "sap", False)):
            op = sns.opts(4 * n, "countsketch", 1, tol=1e-300, max_iter=budget, precondition=pre, method=meth)
            ws = torch.empty(ctx.lstsq_workspace(prob, op), dtype=torch.uint8, device=dev)
            x = torch.empty(n, dtype=torch.float64, device=dev)
            ctx.lstsq_problem(prob, op, x=x, ws=ws)                   # warm-up
            torch.cuda.synchronize()
            reps = 2
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                _, info = ctx.lstsq_problem(prob, op, x=x, ws=ws)
            e1.record()
            torch.cuda.synchronize()
            d = x - x_star
            row[label] = {"ms": e0.elapsed_time(e1) / reps, "passes": info.iters, "residual_passes": info.outer,
                          "forward_error": float(torch.linalg.norm(d) / torch.linalg.norm(x_star)),
                          "residual_error": float(torch.linalg.norm(A @ d) / beta), "eta": info.eta,
                          "status": sns.status_name(info.status)}
            del ws
        rows.append(row)
        del A, b, x_star, prob
        torch.cuda.empty_cache()
    print(json.dumps({"workload": "paper", "config": {"n": n, "kappa": kappa, "beta": beta, "d": 4 * n,
                                                      "dtype": "f64", "sketch": "countsketch",
                                                      "passes_budget": budget,
                                                      "stop": "fixed budget of passes (eta floors near 1e-7 "
                                                              "in FP64 at this beta)"},
                      "data": "synthetic (U diag(sigma) V^T, known x*)", "rows": rows}))


# ------------------------------------------------------------------ batched workload
def _haar(n, gen, dev):
    import torch
    Z = torch.randn(n, n, generator=gen, device=dev, dtype=torch.float64)
    Q, R = torch.linalg.qr(Z)
    return Q * torch.sign(torch.diagonal(R))[None, :]


def _ill_dense(m, n, kappa, noise, gen, dev):
    """A = G diag(sigma) Q (FP32) and b = A x_true + noise, generated on the device."""
    import torch
    sig = kappa ** (-torch.arange(n, device=dev, dtype=torch.float64) / max(n - 1, 1))
    Mx = (sig[:, None] * _haar(n, gen, dev)).float()
    A = torch.randn(m, n, generator=gen, device=dev) @ Mx
    xt = torch.randn(n, generator=gen, device=dev, dtype=torch.float64)
    b = (A.double() @ xt + noise * torch.randn(m, generator=gen, device=dev, dtype=torch.float64)).float()
    return A.contiguous(), b


def run_batched(args):
    """4096 problems, m ~ U[4096, 65536], n ~ U{16,32,64,128}, d = 4n, kappa 1e3: one
    snsolve_lstsq_batched call per step (graph replay) vs one snsolve_lstsq call per
    problem."""
    import torch
    import paper_2409_14309_gb300 as sns
    from synth import batched_shapes
    dev = torch.device("cuda", 0)
    ctx = sns.Context(0)
    shapes = batched_shapes(4096, seed=1004)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1004)
    As, bs = [], []
    for (m, n, d) in shapes:
        A, b = _ill_dense(m, n, 1e3, 1e-3, gen, dev)
        As.append(A)
        bs.append(b)
    ds = [d for (_, _, d) in shapes]
    seeds = list(range(len(shapes)))
    torch.cuda.synchronize()
    ws = None
    xs, infos = ctx.lstsq_batched(As, bs, ds, seeds)          # tunes on first call
    for _ in range(max(1, args.warmup - 1)):
        xs, infos = ctx.lstsq_batched(As, bs, ds, seeds)
    torch.cuda.synchronize()
    t = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        xs, infos = ctx.lstsq_batched(As, bs, ds, seeds)
        e1.record()
        torch.cuda.synchronize()
        t.append(e0.elapsed_time(e1))
    batched_ms = float(np.median(t))
    # plain form: one solve per launch sequence
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat = []
    e0.record()
    for A, b, d, sd in zip(As, bs, ds, seeds):
        t0 = time.perf_counter()
        ctx.lstsq(A, b, d, seed=sd)
        lat.append((time.perf_counter() - t0) * 1e3)
    e1.record()
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    tot_bytes = sum(A.numel() * 4 + b.numel() * 4 for A, b in zip(As, bs))
    q = [n + 1 for (_, n, _) in shapes]
    flops = sum(2.0 * d * qq * qq - 2.0 / 3.0 * qq ** 3 for d, qq in zip(ds, q))
    line = {"metric": METRIC, "workload": "batched", "value": len(shapes) / (batched_ms / 1e3), "unit": "solves/s",
            "n_gpus": 1, "steps": args.steps, "ms_per_step": batched_ms, "higher_is_better": True,
            "config": {"workload": "4096 dense FP32 problems, m~U[4096,65536], n~U{16,32,64,128}, d=4n, kappa 1e3, "
                                   "sketch-and-solve (CountSketch + FP64 QR + back-solve) in one persistent launch",
                       "input_bytes": tot_bytes, "qr_flops": flops},
            "batch_latency_ms": batched_ms,
            "plain": {"value": len(shapes) / (plain_ms / 1e3), "unit": "solves/s",
                      "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                      "form": "one snsolve_lstsq call per problem, in order"},
            "achieved": {"input_GBps": tot_bytes / (batched_ms / 1e3) / 1e9,
                         "fp64_TFLOPs": flops / (batched_ms / 1e3) / 1e12},
            "status_ok": int(sum(1 for i in infos if i.status == 0))}
    print(json.dumps(line))


# ------------------------------------------------------------------ served workload
def _csr_device(m, n, dens, gen, dev):
    """CSR with round(dens*n) (>= 1) uniformly random columns per row (duplicates
    allowed, they add) and N(0,1) values, built on the device."""
    import torch
    k = max(1, int(round(dens * n)))
    col = torch.randint(0, n, (m, k), generator=gen, device=dev, dtype=torch.int32)
    col, _ = torch.sort(col, dim=1)
    val = torch.randn(m, k, generator=gen, device=dev)
    rowptr = torch.arange(0, (m + 1) * k, k, device=dev, dtype=torch.int64)
    xt = torch.randn(n, generator=gen, device=dev)
    b = (val * xt[col.long()]).sum(1) + 1e-3 * torch.randn(m, generator=gen, device=dev)
    return rowptr, col.reshape(-1).contiguous(), val.reshape(-1).contiguous(), b.contiguous()


def _dense_request(m, n, gen, dev):
    """Dense FP32 N(0,1) A and b = A x_true + 1e-3 noise, built on the device."""
    import torch
    A = torch.randn(m, n, generator=gen, device=dev)
    xt = torch.randn(n, generator=gen, device=dev)
    b = torch.mv(A, xt) + 1e-3 * torch.randn(m, generator=gen, device=dev)
    return A, b


def run_served(args):
    """Poisson stream of --requests requests (default 20,000) with the served
    workload's shape mix (m log-uniform in [2^14, 2^22], n in {32..1024}, half
    dense FP32 N(0,1) / half CSR at 0.5-5% density, b = A x_true + 1e-3 noise,
    tolerance 1e-3 or 1e-10).  Each request's data is generated on the device at
    its arrival, on a client stream; latency runs from data-ready to result, and
    the generation time is reported beside it.  An 8-slot server against one
    slot (the plain form) at arrival rates --rates x the plain form's measured
    capacity (one rate above it); the highest rate runs --requests requests, the
    others --sweep-requests.  The client holds at most 100 GB of request
    data: beyond that, arrivals wait (the wait is reported)."""
    import torch
    import paper_2409_14309_gb300 as sns
    from synth import served_requests
    dev = torch.device("cuda", 0)
    ctx = sns.Context(0)
    client = torch.cuda.Stream(device=dev)
    R = args.requests
    rates = [float(x) for x in args.rates.split(",")]
    specs = served_requests(R, seed=1005, rate_per_s=1.0)
    client_cap = 100 << 30

    def req_bytes(sp):
        m, n = sp["m"], sp["n"]
        if sp["sparse"]:
            k = max(1, int(round(sp["density"] * n)))
            return m * k * 8 + (m + 1) * 8 + m * 4
        return m * n * 4 + m * 4

    def run(slots, rate, nreq, seed):
        srv = sns.Server(ctx, hbm_budget_bytes=150 << 30, max_slots=slots)
        gen = torch.Generator(device=dev)
        gen.manual_seed(seed)
        rng = np.random.default_rng(seed)
        gaps = rng.exponential(1.0 / rate, size=nreq) if rate else np.zeros(nreq)
        arrive = np.cumsum(gaps)
        made, held = [], 0                       # generated, not yet submitted: (i, event, data)
        out = {}                                 # rid -> (i, data, t_ready)
        lat, gen_ms, hold_ms = [], [], []
        bad, nxt, done = 0, 0, 0
        t0 = time.perf_counter()
        while done < nreq:
            progressed = False
            for rid in list(out):
                code, info = srv.poll(rid, timeout_us=0)
                if code == 0:
                    i, data, t_ready, nb = out.pop(rid)
                    lat.append((time.perf_counter() - t_ready) * 1e3)
                    bad += int(info.status != 0)
                    held -= nb
                    done += 1
                    progressed = True
            still = []
            for i, ev, data, t_arr, nb in made:
                if ev.query():
                    t_ready = time.perf_counter()
                    gen_ms.append((t_ready - t_arr) * 1e3)
                    sp = specs[i]
                    n, d = sp["n"], 4 * sp["n"]
                    if sp["sparse"]:
                        rid, _ = srv.submit_csr(*data, n, d, seed=i, tol=sp["tol"], max_iter=2000)
                    else:
                        rid, _ = srv.submit(data[0], data[1], d, seed=i, tol=sp["tol"], max_iter=1000)
                    out[rid] = (i, data, t_ready, nb)
                    progressed = True
                else:
                    still.append((i, ev, data, t_arr, nb))
            made = still
            now = time.perf_counter() - t0
            while nxt < nreq and arrive[nxt] <= now:
                sp = specs[nxt]
                nb = req_bytes(sp)
                if held + nb > client_cap and held > 0:
                    break                        # client memory full: the arrival waits
                hold_ms.append((now - arrive[nxt]) * 1e3)
                with torch.cuda.stream(client):
                    if sp["sparse"]:
                        data = _csr_device(sp["m"], sp["n"], sp["density"], gen, dev)
                    else:
                        data = _dense_request(sp["m"], sp["n"], gen, dev)
                    ev = torch.cuda.Event()
                    ev.record(client)
                made.append((nxt, ev, data, t0 + now, nb))
                held += nb
                nxt += 1
                progressed = True
            if not progressed:
                time.sleep(0.0001)
        wall = time.perf_counter() - t0
        srv.close()
        return {"requests": nreq, "solves_per_s": nreq / wall, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "gen_p50_ms": float(np.percentile(gen_ms, 50)),
                "arrival_wait_p99_ms": float(np.percentile(hold_ms, 99)), "failed": bad, "wall_s": wall}

    run(8, None, min(64, R), 7)                                # warm-up (library caches, allocator)
    cap_n = min(R, 2000)
    plain_cap = run(1, None, cap_n, 11)["solves_per_s"]        # closed loop: one slot's capacity
    sweep = []
    for fr in rates:
        rate = fr * plain_cap
        nreq = R if fr == max(rates) else min(R, args.sweep_requests)
        served = run(8, rate, nreq, 1005)
        plain = run(1, rate, nreq, 1005)
        sweep.append({"rate_x_plain_capacity": fr, "rate_per_s": rate, "served_8_slots": served,
                      "plain_one_slot": plain})
    head = max(sweep, key=lambda e: e["rate_x_plain_capacity"])
    line = {"metric": METRIC, "workload": "served", "value": head["served_8_slots"]["solves_per_s"],
            "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
            "config": {"requests": R, "sweep_requests": min(R, args.sweep_requests),
                       "arrival": f"Poisson, rates {rates} x the one-slot capacity "
                                                 f"({plain_cap:.1f}/s); headline at the highest rate",
                       "requests_shape": "m log-uniform [2^14,2^22], n in {32..1024}, half dense FP32 N(0,1) / "
                                         "half CSR 0.5-5%, b = A x_true + 1e-3 noise, generated on the device "
                                         "per request at arrival (client stream)",
                       "tol": "1e-3 or 1e-10 (50/50)", "budget_bytes": 150 << 30, "slots": 8,
                       "client_data_cap_bytes": client_cap},
            "served": head["served_8_slots"], "plain_one_slot": head["plain_one_slot"],
            "plain_capacity_solves_per_s": plain_cap, "sweep": sweep}
    print(json.dumps(line))


# ------------------------------------------------------------------ sketch kinds
def run_sketches(args):
    """snsolve_sketch alone on the 1048576 x 256 workload for every sketch kind:
    HBM GB/s (A and b read once) and, for the Gaussian GEMM, tensor TFLOP/s.
    Outside the timed loops, the quality of each sketch as a preconditioner:
    kappa(A R^-1) with R from a QR of the sketch (FP64, from the eigenvalues of
    R^-T (A^T A) R^-1; torch's linear algebra as a measuring tool)."""
    import torch
    import paper_2409_14309_gb300 as sns
    from paper_2409_14309_gb300 import abi
    dev = torch.device("cuda", 0)
    ctx = sns.Context(0)
    L = abi.lib()
    A_h, b_h = make_inputs(0, dev)
    A = torch.from_numpy(A_h).to(dev)
    b = torch.from_numpy(b_h).to(dev)
    hbm_peak, bf16_peak, kind_peak = peaks()
    A64 = A.double()
    gram = A64.T @ A64                                   # A^T A in FP64 (n x n)
    del A64
    ev = torch.linalg.eigvalsh(gram)
    kappa_A = float(torch.sqrt(ev[-1] / ev[0]))

    def kappa_precond(SA):
        R = torch.linalg.qr(SA.double(), mode="r")[1]
        t1 = torch.linalg.solve_triangular(R.T, gram, upper=False)          # R^-T G
        Mx = torch.linalg.solve_triangular(R.T, t1.T.contiguous(), upper=False)   # R^-T G R^-1
        e = torch.linalg.eigvalsh(0.5 * (Mx + Mx.T))
        return float(torch.sqrt(e[-1] / e[0]))

    out = {}
    for name, kind, variant in [("countsketch_sorted", "countsketch", "sorted"),
                                ("countsketch_stream", "countsketch", "stream"),
                                ("sparse_sign_zeta4", "sparse_sign", 4),
                                ("gaussian_tcgen05", "gaussian", "auto"),
                                ("gaussian_tcgen05_2terms", "gaussian", 2),
                                ("gaussian_tcgen05_3terms", "gaussian", 3), ("srht", "srht", "auto")]:
        prob = sns.dense_problem(A, b)
        sk = sns.sketch_desc(D, kind, SKETCH_SEED, variant)
        ws = torch.empty(max(ctx.sketch_workspace(prob, sk), 256), dtype=torch.uint8, device=dev)
        for _ in range(max(3, args.warmup)):
            ctx.sketch_problem(prob, sk, torch.float32, ws=ws)
        torch.cuda.synchronize()
        L.snsolve_profile(1)
        kernel_profile(L)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            ctx.sketch_problem(prob, sk, torch.float32, ws=ws)
        e1.record()
        torch.cuda.synchronize()
        prof = kernel_profile(L)
        L.snsolve_profile(0)
        ms = e0.elapsed_time(e1) / args.steps
        byts = M * (N + 1) * 4.0
        r = {"ms": ms, "GBps": byts / (ms / 1e3) / 1e9, "frac_hbm": byts / (ms / 1e3) / 1e9 / hbm_peak,
             "kernels_ms": {k: v[0] / args.steps for k, v in prof.items()}}
        if kind == "gaussian":
            # algorithmic flops of G [A | b]; the tensor cores run one product per BF16 term
            terms = 1 if variant == "auto" else int(variant)
            fl = 2.0 * D * M * (N + 1)
            r["terms"] = terms
            r["TFLOPs"] = fl / (ms / 1e3) / 1e12
            r["tensor_TFLOPs"] = terms * r["TFLOPs"]
            r["frac_bf16"] = r["tensor_TFLOPs"] / bf16_peak
        SA_k, _ = ctx.sketch_problem(prob, sk, torch.float32, ws=ws)
        r["kappa_A_Rinv"] = kappa_precond(SA_k)
        out[name] = r
    print(json.dumps({"metric": METRIC, "workload": "sketches", "config": {"m": M, "n": N, "d": D},
                      "kappa_A": kappa_A,
                      "peaks": {"hbm_GBps": hbm_peak, "bf16_TFLOPs": bf16_peak, "kind": kind_peak},
                      "sketches": out}))


# ------------------------------------------------------------------ small-problem latency
def run_latency(args):
    """4096 x 64 FP64 N(0,1), x_true N(0,1), noise 1e-3, CountSketch d = 256 with
    sketch seed 0: per-call latency of sketch-and-solve and of a solve to
    eta <= 1e-10 (microseconds, host wall clock around the synchronous call)."""
    import torch
    import paper_2409_14309_gb300 as sns
    dev = torch.device("cuda", 0)
    ctx = sns.Context(0)
    rng = np.random.default_rng(1001)
    m, n, d = 4096, 64, 256
    A_h = rng.standard_normal((m, n))
    b_h = A_h @ rng.standard_normal(n) + 1e-3 * rng.standard_normal(m)
    A = torch.from_numpy(A_h).to(dev)
    b = torch.from_numpy(b_h).to(dev)
    prob = sns.dense_problem(A, b)
    out = {}
    for name, tol in (("sketch_and_solve", 0.0), ("sap_eta_1e-10", 1e-10)):
        op = sns.opts(d, "countsketch", 0, "auto", tol=tol)
        ws = torch.empty(ctx.lstsq_workspace(prob, op), dtype=torch.uint8, device=dev)
        x = torch.empty(n, dtype=torch.float64, device=dev)
        for _ in range(max(3, args.warmup)):
            ctx.lstsq_problem(prob, op, x=x, ws=ws)
        torch.cuda.synchronize()
        ts = []
        info = None
        for _ in range(max(args.steps, 50)):
            t0 = time.perf_counter()
            _, info = ctx.lstsq_problem(prob, op, x=x, ws=ws)
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e6)
        ts.sort()
        out[name] = {"p50_us": ts[len(ts) // 2], "p99_us": ts[min(len(ts) - 1, int(0.99 * len(ts)))],
                     "status": info.status, "iters": info.iters, "outer": info.outer, "eta": info.eta}
    print(json.dumps({"metric": "small-problem solve latency (us)", "workload": "latency", "unit": "us",
                      "higher_is_better": False, "dtype": "f64",
                      "config": {"workload": "dense FP64 N(0,1) 4096 x 64, noise 1e-3, CountSketch d=256 seed 0",
                                 "m": m, "n": n, "d": d}, "latency": out}))


# ------------------------------------------------------------------ sparse workload
def run_profile_case(args):
    """Small cases for profiler captures: inputs above the L2 size, a few hundred MB
    on the device.  solve: 2^18 x 256 FP32 (kappa 1e6, noise 1e-4), CountSketch
    d = 1024, two solves to eta <= 1e-6.  countsketch / srht / gaussian: three
    sketches of a 2^18 x 256 N(0,1) matrix (2^19 rows for countsketch), d = 1024.
    csr: 2^19 x 512 at 1 % plus 64 dense rows x100, d = 2048, two solves to 1e-8.
    batched: 256 problems of the batched workload's shape mix (N(0,1) entries),
    three batched calls (the first tunes the launch shape)."""
    import torch
    import paper_2409_14309_gb300 as sns
    dev = torch.device("cuda", 0)
    ctx = sns.Context(0)
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    if args.case == "solve":
        # the 256 x 256 orthogonal factor on the host (the profiler's environment
        # does not load torch's GPU linear-algebra library)
        n = 256
        Z = torch.randn(n, n, generator=torch.Generator().manual_seed(7), dtype=torch.float64)
        Q, R = torch.linalg.qr(Z)
        Q = Q * torch.sign(torch.diagonal(R))[None, :]
        sig = 1e6 ** (-torch.arange(n, dtype=torch.float64) / (n - 1))
        Mx = (sig[:, None] * Q).float().to(dev)
        A = (torch.randn(1 << 18, n, generator=gen, device=dev) @ Mx).contiguous()
        xt = torch.randn(n, generator=gen, device=dev, dtype=torch.float64)
        b = (A.double() @ xt + 1e-4 * torch.randn(1 << 18, generator=gen, device=dev, dtype=torch.float64)).float()
        for _ in range(2):
            x, info = ctx.lstsq(A, b, 1024, seed=1, tol=1e-6)
        torch.cuda.synchronize()
        print(json.dumps({"case": "solve", "status": info.status, "passes": info.iters, "eta": info.eta}))
    elif args.case == "batched":
        from synth import batched_shapes
        shapes = batched_shapes(256, seed=1004)
        As = [torch.randn(m, n, generator=gen, device=dev) for (m, n, _) in shapes]
        bs = [torch.randn(m, generator=gen, device=dev) for (m, _, _) in shapes]
        for _ in range(3):
            xs, infos = ctx.lstsq_batched(As, bs, [d for (_, _, d) in shapes], list(range(len(shapes))))
        torch.cuda.synchronize()
        print(json.dumps({"case": "batched", "problems": len(shapes), "ok": sum(i.status == 0 for i in infos),
                          "input_bytes": sum(m * (n + 1) * 4 for (m, n, _) in shapes)}))
    elif args.case == "csr":
        rowptr, col, val, b, nnz = _csr_dense_rows(1 << 19, 512, 0.01, 64, gen, dev)
        for _ in range(2):
            x, info = ctx.lstsq_csr(rowptr, col, val, b, 512, 2048, seed=1, tol=1e-8, max_iter=4000)
        torch.cuda.synchronize()
        print(json.dumps({"case": "csr", "status": info.status, "passes": info.iters, "nnz": nnz}))
    else:
        m = (1 << 19) if args.case == "countsketch" else (1 << 18)
        A = torch.randn(m, 256, generator=gen, device=dev)
        b = torch.randn(m, generator=gen, device=dev)
        variant = args.gauss_terms if args.case == "gaussian" else "auto"
        for _ in range(3):
            SA, Sb = ctx.sketch(A, b, 1024, kind=args.case, seed=1, variant=variant)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "m": m, "variant": variant, "norm_SA": float(SA.norm())}))


def _csr_dense_rows(m, n, dens, n_dense, gen, dev):
    """CSR m x n: rows 0..n_dense-1 dense and scaled x100, the others with
    round(dens * n) uniformly random columns (duplicates add); N(0,1) values;
    b = A x_true + 1e-3 noise.  Built on the device."""
    import torch
    k = max(1, int(round(dens * n)))
    cnt = torch.full((m,), k, dtype=torch.int64, device=dev)
    cnt[:n_dense] = n
    rowptr = torch.zeros(m + 1, dtype=torch.int64, device=dev)
    rowptr[1:] = torch.cumsum(cnt, 0)
    nnz = int(rowptr[-1])
    sparse_cols = torch.sort(torch.randint(0, n, (m - n_dense, k), generator=gen, device=dev, dtype=torch.int32),
                             dim=1)[0].reshape(-1)
    dense_cols = torch.arange(n, device=dev, dtype=torch.int32).repeat(n_dense)
    col = torch.cat([dense_cols, sparse_cols]).contiguous()
    val = torch.randn(nnz, generator=gen, device=dev)
    val[: n_dense * n] *= 100.0
    xt = torch.randn(n, generator=gen, device=dev, dtype=torch.float64)
    rows = torch.repeat_interleave(torch.arange(m, device=dev), cnt)
    b = torch.zeros(m, dtype=torch.float64, device=dev).index_add_(0, rows, val.double() * xt[col.long()])
    b = (b + 1e-3 * torch.randn(m, generator=gen, device=dev, dtype=torch.float64)).float()
    return rowptr, col, val, b.contiguous(), nnz


def run_csr(args):
    """CSR 2^21 x 512, density 1 % plus 64 dense rows x100, CountSketch d = 2048:
    preconditioned against unpreconditioned iteration to eta <= 1e-8 (solves/s
    and passes over A), the bitwise reproducible form of the preconditioned solve
    (variant "sorted"), and the CSR sketch's rate (8 B per nonzero + 8 B per row)."""
    import torch
    import paper_2409_14309_gb300 as sns
    from paper_2409_14309_gb300 import abi
    dev = torch.device("cuda", 0)
    ctx = sns.Context(0)
    L = abi.lib()
    m, n, d, tol = 1 << 21, 512, 2048, 1e-8
    gen = torch.Generator(device=dev)
    gen.manual_seed(1003)
    rowptr, col, val, b, nnz = _csr_dense_rows(m, n, 0.01, 64, gen, dev)
    hbm_peak, _, peak_kind = peaks()
    out = {}
    for name, pre, var in (("preconditioned", True, "auto"), ("unpreconditioned", False, "auto"),
                           ("preconditioned_reproducible", True, "sorted")):
        for _ in range(max(1, args.warmup // 3)):
            ctx.lstsq_csr(rowptr, col, val, b, n, d, seed=SKETCH_SEED, tol=tol, max_iter=4000, precondition=pre,
                          variant=var)
        torch.cuda.synchronize()
        L.snsolve_profile(1)
        kernel_profile(L)
        steps = max(2, args.steps // 4)
        t0 = time.perf_counter()
        for _ in range(steps):
            _, info = ctx.lstsq_csr(rowptr, col, val, b, n, d, seed=SKETCH_SEED, tol=tol, max_iter=4000,
                                    precondition=pre, variant=var)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / steps
        prof = kernel_profile(L)
        L.snsolve_profile(0)
        out[name] = {"solves_per_s": 1.0 / dt, "ms_per_solve": dt * 1e3, "status": info.status,
                     "passes": info.iters, "outer": info.outer, "eta": info.eta,
                     "kernels_ms": {k: v[0] / steps for k, v in prof.items()}}
    byts = 8.0 * nnz + 8.0 * m
    gms = out["preconditioned"]["kernels_ms"].get("cs_gather_csr")
    sk = None
    if gms:
        sk = {"kernel": "cs_gather_csr", "ms": gms, "GBps": byts / (gms / 1e3) / 1e9,
              "frac": byts / (gms / 1e3) / 1e9 / hbm_peak, "peak_kind": f"{peak_kind} copy bandwidth",
              "algorithmic_bytes": byts}
    print(json.dumps({"metric": "CSR LS solves/s, preconditioned vs not, to eta <= 1e-8", "workload": "csr",
                      "unit": "solves/s", "higher_is_better": True, "dtype": "f32 passes + f64 QR/solves",
                      "config": {"workload": "CSR 2097152 x 512, 1% + 64 dense rows x100, noise 1e-3, "
                                             "CountSketch d=2048", "m": m, "n": n, "nnz": nnz, "d": d},
                      "solve": out, "sketch_apply": sk}))


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores.  Each step is a complete solve
    of the workload when the whole run fits in about two minutes; otherwise each
    step solves the first m/4 rows and its row-proportional phases are scaled x4."""
    if rank != 0:
        return
    A, b = make_inputs(0, None)
    warm = max(3, args.warmup)
    t_sk, t_qr, t_it, its, _, _ = oracle_solve_sample(A, b, M)    # one untimed warm-up solve
    t_full = t_sk + t_qr + t_it
    frac = 1 if args.steps * t_full <= 120.0 else 4
    rows = M // frac
    ts = []
    for _ in range(args.steps):
        t_sk, t_qr, t_it, its, _, _ = oracle_solve_sample(A, b, rows)
        ts.append(t_sk * frac + t_qr + t_it * frac)
    tot = float(np.sum(ts))
    val = args.steps / tot
    sample = ("complete solve of the workload per step" if frac == 1 else
              f"first {rows} rows per step, row-proportional phase times x{frac}") + f" ({its} LSQR iterations)"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": 1, "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "m": M, "n": N, "d": D, "kappa": KAPPA, "tol_eta": TOL},
            "cpu_baseline": {"kind": "oracle", "cores": cpu_cores(), "value": val, "unit": "solves/s",
                             "sample": sample},
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
