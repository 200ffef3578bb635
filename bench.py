#!/usr/bin/env python3
"""Benchmark of the HOT solver (arXiv 2408.00598) on one GB300.

Default workload (the configuration the headline metric is quoted on): one
256 x 256 pair (M = 65536 bins, 2*256^3 = 3.4e7 flow variables), seeded white
noise, FP32-bulk Algorithm 2 to relative KKT 1e-6, then Algorithm 1 plan
recovery on the device.  One step = one such solve + recovery.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]
                    [--mode solve|batch|serve] [--size S] [--kind white]

Prints ONE JSON line.  `value` (solves/s) is measured with inputs resident in
HBM (device pointers through the C ABI), CUDA events on the solver's stream;
`e2e` repeats the steps through the same ABI from host buffers, with the
host->device copy of the histograms and the device->host copy of the plan
inside the timed region.  With --gpus N (torchrun) each rank solves its own
pair (replicas; weak scaling) and the time is the max over ranks.

`--impl reference` times the FP64 CPU oracle (oracle/, test infrastructure)
on the same pair: each step is a bounded sample of 10 iterations of Algorithm 2
with the KKT check (the model is built once, timed apart), and solves/s scales the measured time
per iteration to the iteration count the oracle itself needs on that pair
(440 at 256 x 256, from its stored full run in tests/golden/oracle_values.json).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of the FP32 sweep
# (k_sweep32<false>) on the 256^3 x 2 state, and the hash of the kernel
# source it was taken on (traffic is reported only while the source matches).
SWEEP_TRAFFIC = {"kernels_sha256": "f2f49a4ec04b63fb0d681fca831200f37ba4f913d3d51de6122535b8e85bd502",
                 "bytes_per_launch": 273730048 + 87800064}

GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_values.json")


def oracle_iterations(S, kind, seed, tol, stop="relative"):
    """Iterations the FP64 oracle takes on this pair to tol, from its stored
    full run (tests/golden/oracle_values.json, written by the oracle alone), or
    None when no run of this pair is stored."""
    try:
        with open(GOLDEN) as f:
            cases = json.load(f)["cases"]
    except Exception:
        return None
    for rec in cases.values():
        if (rec["S"], rec["kind"], rec["seed"], rec["tol"]) == (S, kind, seed, tol) and \
                rec.get("stop", "relative") == stop:
            return int(rec["iters"])
    return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["solve", "batch", "serve"], default="solve")
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--kind", default="white")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--stop", choices=["relative", "absolute"], default="relative",
                    help="stopping rule: relative KKT, eq. (kkt_res), or absolute KKT (Table VI)")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32",
                    help="solve mode: FP32 bulk (the default) or the plain FP64 form")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--acc-tol", type=float, default=5e-10,
                    help="solve mode: tolerance of the plan-accuracy leg (the plan's marginals to 1e-6 in L1)")
    ap.add_argument("--no-accuracy-leg", action="store_true")
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--duration", type=float, default=60.0)
    ap.add_argument("--max-drain", type=float, default=180.0,
                    help="serve mode: seconds to wait for the queue after the arrivals stop; the rest is cancelled")
    ap.add_argument("--compare-fp64", action="store_true",
                    help="batch mode: also solve the same pairs one by one in FP64 mode (the plain GPU form)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


class Dist:
    def __init__(self, use_cuda):
        self.rank, self.local_rank, self.world = dist_env()
        self.pg = None
        if self.world > 1:
            import torch.distributed as td
            backend = "nccl" if use_cuda else "gloo"
            td.init_process_group(backend=backend)
            self.pg = td

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x):
        if not self.pg:
            return x
        import torch
        t = torch.tensor([float(x)], device="cuda" if self.pg.get_backend() == "nccl" else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


class Clocks:
    """nvidia-smi samples (SM clock, power, throttle reasons) during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [s.strip() for s in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def kernels_sha():
    import hashlib
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_2408_00598_gb300", "csrc", "hot_kernels.cu"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()


def recorded_traffic(S, precision):
    """The recorded ncu DRAM traffic of one sweep launch, or None where it was
    not taken (another size or precision) or the kernel source has changed
    since."""
    if SWEEP_TRAFFIC["kernels_sha256"] == kernels_sha() and S == 256 and precision == "fp32":
        return SWEEP_TRAFFIC["bytes_per_launch"]
    return None


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------- oracle --

class OracleSample:
    """The FP64 oracle on a bounded sample of a solve: the model is built once
    (timed), then batches of Algorithm-2 iterations are timed one by one."""

    def __init__(self, mu1, mu2):
        import numpy as np
        from oracle import hot as ohot
        from oracle import reduced_model as rm
        self.np, self.ohot = np, ohot
        self.S = mu1.shape[0]
        t0 = time.perf_counter()
        self.A = rm.build_A(self.S, self.S)
        self.b = rm.build_b(mu1, mu2)
        c = rm.build_c(self.S, self.S)
        self.c = c / ohot.cost_scale(c)
        self.t_build = time.perf_counter() - t0
        self.x = np.zeros(self.c.size)
        self.z = np.zeros(self.c.size)
        self.sigma = float(np.linalg.norm(self.b) / np.linalg.norm(self.c))

    def run(self, n_iter):
        """Seconds for n_iter iterations of the oracle's loop: Steps 1-3
        (oracle.hot.hot_step), the Halpern update of Step 4, and the KKT
        residual eq. (kkt_res) every 10th iteration, as oracle.hot.hot_solve
        runs them (a restart never falls in so short a sample)."""
        t1 = time.perf_counter()
        for k in range(n_iter):
            yb, xb, zb = self.ohot.hot_step(self.A, self.b, self.c, self.sigma, self.x, self.z, self.S, self.S)
            if (k + 1) % 10 == 0:
                self.ohot.kkt_residual(self.A, self.b, self.c, xb, yb, zb)
                self.ohot.kkt_absolute(self.A, self.b, self.c, xb, yb, zb)
            self.x = (k + 1) / (k + 2) * (2.0 * xb - self.x)
            self.z = (k + 1) / (k + 2) * (2.0 * zb - self.z)
        return time.perf_counter() - t1


def cpu_threads():
    return 1   # scipy sparse mat-vecs and the numpy element-wise ops run on one thread


def oracle_baseline(mu1, mu2, kind, seed, tol, gpu_iters, n_iter=50, stop="relative"):
    """cpu_baseline: n_iter oracle iterations measured in one run; solves/s
    scales the measured time per iteration to the oracle's own iteration count
    for this pair (stored full run), else to the GPU solve's (the same when
    their restart decisions agree)."""
    smp = OracleSample(mu1, mu2)
    t = smp.run(n_iter)
    t_iter = t / n_iter
    iters = oracle_iterations(smp.S, kind, seed, tol, stop)
    src = "the oracle's stored full run of this pair"
    if iters is None:
        iters, src = gpu_iters, "the GPU solve of this pair"
    per_solve = smp.t_build + iters * t_iter
    desc = ("oracle (numpy/scipy, FP64) at S=%d: %d Algorithm-2 iterations measured in %.1f s (%.3f s each) + "
            "model build %.1f s; solves/s = 1 / (build + %d iterations, the count of %s)"
            % (smp.S, n_iter, t, t_iter, smp.t_build, iters, src))
    return 1.0 / per_solve, desc


# ------------------------------------------------------------------ modes --

def bench_solve(args, dist):
    import numpy as np
    import torch
    from paper_2408_00598_gb300 import hot
    from paper_2408_00598_gb300 import synthetic as syn

    torch.cuda.set_device(dist.local_rank)
    # a dedicated stream: the library enqueues all its work on it, so CUDA
    # events recorded on it bracket exactly the solver's device work
    stream = torch.cuda.Stream(device=dist.local_rank)
    ctx = hot.Context(device=dist.local_rank, precision=args.precision, stream=stream.cuda_stream, stop=args.stop)
    S = args.size
    mu1, mu2 = syn.make_pair(args.kind, S, 1000 + dist.rank)
    d1 = torch.from_numpy(mu1).cuda()
    d2 = torch.from_numpy(mu2).cuda()
    cap = S * S * (2 * S - 1)
    src = torch.empty(cap, dtype=torch.int32, device="cuda")
    dst = torch.empty(cap, dtype=torch.int32, device="cuda")
    mass = torch.empty(cap, dtype=torch.float64, device="cuda")
    rec = {}

    def step():
        r = ctx.solve(d1, d2, tol=args.tol, max_iter=1000000)
        n, l1 = ctx.recover_plan(r, device_out=(src, dst, mass))
        ctx.release(r)
        rec.update(r=r, n=n, l1=l1)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    dist.barrier()
    clk = Clocks(dist.local_rank)
    clk.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    # the dominant kernel is timed live: the block graphs of the timed solves
    # carry a CUDA event pair (on the library's stream) around one non-check
    # sweep per block of 10 iterations
    ctx.sweep_timing(1)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    live = ctx.sweep_timing(0)
    clocks = clk.stop()
    dist.barrier()
    t = dist.max(ev0.elapsed_time(ev1) / 1000.0)
    r = rec["r"]
    value = dist.world * args.steps / t
    iters = r["iters"]
    launches_per_step = r["kernel_launches"] + 5        # + recovery: count, scan, 2 x L1, write

    # e2e: host buffers through the same ABI, copies inside the timed region
    h1 = torch.from_numpy(mu1).pin_memory()
    h2 = torch.from_numpy(mu2).pin_memory()
    hsrc = torch.empty(cap, dtype=torch.int32).pin_memory()
    hdst = torch.empty(cap, dtype=torch.int32).pin_memory()
    hmass = torch.empty(cap, dtype=torch.float64).pin_memory()
    e2e_rec = {}

    def step_host():
        rr = ctx.solve(h1.numpy(), h2.numpy(), tol=args.tol, max_iter=1000000)
        n, l1 = ctx.recover_plan_host(rr, hsrc, hdst, hmass)
        ctx.release(rr)
        e2e_rec.update(n=n)

    step_host()
    torch.cuda.synchronize()
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_host()
    torch.cuda.synchronize()
    te = dist.max(time.perf_counter() - t0)
    e2e = {"value": dist.world * args.steps / te, "unit": "solves/s",
           "h2d_bytes_per_step": 2 * S * S * 8, "d2h_bytes_per_step": e2e_rec["n"] * 16 + 160}

    # dominant kernel: per-launch device time of the FP32 sweep, from the live
    # event pairs of the timed region; a separate profiled solve (every kernel
    # family bracketed by events, launched without the graph) gives the
    # breakdown of the rest
    rp, kt = ctx.solve_profiled(d1, d2, tol=args.tol, max_iter=1000000)
    ctx.release(rp)
    if live["launches"] > 0:
        sweep_s = live["ms"] / live["launches"] / 1000.0
        achieved = live["bytes"] / live["launches"] / sweep_s / 1e9
        timing = ("CUDA event pair around one non-check sweep per 10-iteration block, inside the timed "
                  "solves' graphs, on the library's stream")
    else:
        sweep_s = kt["sweep_ms"] / max(1, kt["sweep_launches"]) / 1000.0
        achieved = kt["sweep_bytes"] / sweep_s / 1e9
        timing = "CUDA event pairs around every sweep of a separate profiled solve (no graph)"
    peak, peak_kind = measured_peak()
    traffic = recorded_traffic(S, args.precision)
    total_ms = kt["sweep_ms"] + kt["sweep_check_ms"] + kt["solve_ms"] + kt["block_end_ms"]
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "peak_kind": peak_kind,
                "kernel": ("k_sweep32<false>" if args.precision == "fp32" else "k_sweep64")
                          + " (Steps 2-4 fused, non-check iterations)",
                "bytes_per_launch": kt["sweep_bytes"], "avg_launch_us": round(sweep_s * 1e6, 2),
                "timed_launches": live["launches"],
                "timing": timing,
                "share_of_solve_device_time": round(kt["sweep_ms"] / total_ms, 4) if total_ms > 0 else None,
                "device_us_per_iteration": {
                    "sweep": round(1000 * kt["sweep_ms"] / max(1, kt["sweep_launches"]), 2),
                    "sweep_check": round(1000 * kt["sweep_check_ms"] / max(1, kt["sweep_check_launches"]), 2),
                    "prop3_solve": round(1000 * kt["solve_ms"] / max(1, kt["sweep_launches"] + kt["sweep_check_launches"]), 2),
                    "block_end_per_block": round(1000 * kt["block_end_ms"] / max(1, kt["sweep_check_launches"]), 2)}}

    # the plan-accuracy leg: the same pair solved until Algorithm 1's plan
    # matches mu and nu to 1e-6 in L1 (relative KKT about 5e-10 at 256 x 256,
    # against the paper's 1e-6: its marginals are then off by about 1.6e-2)
    accuracy = None
    if not args.no_accuracy_leg and args.precision == "fp32" and dist.world == 1 and args.stop == "relative":
        torch.cuda.synchronize()
        ta0 = time.perf_counter()
        ra = ctx.solve(d1, d2, tol=args.acc_tol, max_iter=5000000)
        na, l1a = ctx.recover_plan(ra, device_out=(src, dst, mass))
        ctx.release(ra)
        torch.cuda.synchronize()
        ta = time.perf_counter() - ta0
        accuracy = {"tol": args.acc_tol, "solves_per_s": round(1.0 / ta, 4), "seconds": round(ta, 3),
                    "iterations": ra["iters"], "restarts": ra["restarts"], "rel_kkt": ra["rel_kkt"],
                    "plan_nnz": na, "plan_marginal_l1": l1a, "converged": ra["status"] == 0,
                    "ot_value": ra["ot_value"], "dual_value": ra["dual_value"],
                    "timing": "one solve + Algorithm 1, host clock around device-resident inputs"}

    solve_s = r["solve_ms"] / 1000.0                    # device time of the last timed solve alone
    per_iter_bytes = (12.0 if args.precision == "fp32" else 24.0) * 2 * S ** 3
    out = {"metric": "solves/s (ms-to-1e-6 KKT) at N=%d" % S, "value": round(value, 4), "unit": "solves/s",
           "n_gpus": dist.world, "steps": args.steps, "warmup": max(3, args.warmup),
           "ms_per_step": round(1000.0 * t / args.steps, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
           "config": {"workload": "single %dx%d pair (%s, seed 1000+rank), %s Algorithm 2 to %s-KKT %g "
                                  "+ Algorithm 1 plan recovery on the device"
                                  % (S, S, args.kind, "FP32-bulk" if args.precision == "fp32" else "FP64",
                                     "rel" if args.stop == "relative" else "abs", args.tol),
                      "S": S, "flow_variables": 2 * S ** 3, "tol": args.tol, "stop": args.stop,
                      "l2": "state %.0f MB > 129 MB L2 every iteration (no flush needed)" % (20 * S ** 3 / 1e6),
                      "parallelism": "replicas" if dist.world > 1 else "single"},
           "iterations_per_solve": iters, "restarts": r["restarts"],
           "ms_per_iteration": round(1000.0 * t / args.steps / iters, 4),
           "hbm_gbs_per_iteration": round(per_iter_bytes / (t / args.steps / iters) / 1e9, 1),
           "hbm_frac_per_iteration": round(per_iter_bytes / (t / args.steps / iters) / 1e9 / peak, 4),
           "hbm_per_iteration_note": ("algorithmic state bytes (12 B per flow variable in FP32 bulk, 24 B in "
                                      "FP64) x iterations / ms_per_step; the step includes plan recovery"),
           "hbm_gbs_per_iteration_solve_only": round(per_iter_bytes * iters / solve_s / 1e9, 1),
           "hbm_frac_per_iteration_solve_only": round(per_iter_bytes * iters / solve_s / 1e9 / peak, 4),
           "plan_nnz": rec["n"], "plan_marginal_l1": rec["l1"], "rel_kkt": r["rel_kkt"],
           "roofline": roofline, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
           "clocks": clocks}
    if accuracy is not None:
        out["plan_accuracy"] = accuracy
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        v, desc = oracle_baseline(mu1, mu2, args.kind, 1000, args.tol, iters, stop=args.stop)
        out["cpu_baseline"] = {"value": round(v, 8), "unit": "solves/s", "cores": cpu_threads(),
                               "host_cpus": os.cpu_count(), "kind": "oracle", "sample": desc}
    ctx.close()
    return out


def bench_reference(args, dist):
    """The FP64 CPU oracle on the same workload (rank 0 only): every step
    times 10 iterations of Algorithm 2 with their KKT check on the pair (the model is built once,
    before the steps); solves/s scales the median time per iteration to the
    oracle's own iteration count for the pair."""
    from paper_2408_00598_gb300 import synthetic as syn
    if dist.rank != 0:
        return None
    S = args.size
    mu1, mu2 = syn.make_pair(args.kind, S, 1000)
    iters = oracle_iterations(S, args.kind, 1000, args.tol)
    src = "the oracle's stored full run of this pair"
    if iters is None:
        iters, src = 1100, "a stated count (no stored run of this pair)"
    smp = OracleSample(mu1, mu2)
    n_iter = 10
    for _ in range(args.warmup):
        smp.run(1)
    steps = [smp.run(n_iter) for _ in range(max(1, args.steps))]
    t_iter = statistics.median(steps) / n_iter
    per = smp.t_build + iters * t_iter
    v = 1.0 / per
    desc = ("oracle (numpy/scipy, FP64) at S=%d: %d steps of %d Algorithm-2 iterations, median %.3f s per "
            "iteration, + model build %.1f s; solves/s = 1 / (build + %d iterations, the count of %s)"
            % (S, len(steps), n_iter, t_iter, smp.t_build, iters, src))
    return {"impl": "reference", "metric": "solves/s (ms-to-1e-6 KKT) at N=%d" % S, "value": round(v, 8),
            "unit": "solves/s", "n_gpus": dist.world, "steps": len(steps), "warmup": args.warmup,
            "ms_per_step": round(1000.0 * statistics.median(steps), 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "single %dx%d pair (%s, seed 1000), Algorithm 2 to rel-KKT %g (FP64 CPU oracle)"
                                   % (S, S, args.kind, args.tol), "S": S,
                       "step": "%d oracle iterations (a bounded sample of one solve)" % n_iter},
            "cpu_baseline": {"value": round(v, 8), "unit": "solves/s", "cores": cpu_threads(),
                             "host_cpus": os.cpu_count(), "kind": "oracle", "sample": desc},
            "e2e": {"value": round(v, 8), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def bench_batch(args, dist):
    """512 independent pairs, S uniform in {32,48,64,96,128}, classes mixed; one
    batched graph-captured device loop with per-instance early termination."""
    import torch
    from paper_2408_00598_gb300 import hot
    from paper_2408_00598_gb300 import synthetic as syn
    torch.cuda.set_device(dist.local_rank)
    stream = torch.cuda.Stream(device=dist.local_rank)
    ctx = hot.Context(device=dist.local_rank, precision="fp32", stream=stream.cuda_stream)
    batch = syn.mixed_batch([32, 48, 64, 96, 128], args.batch, 7 + dist.rank)
    mus = [torch.from_numpy(b[3]).cuda() for b in batch]
    nus = [torch.from_numpy(b[4]).cuda() for b in batch]
    for _ in range(max(1, args.warmup)):
        out = ctx.solve_batch(mus, nus, tol=args.tol)
    torch.cuda.synchronize()
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        out = ctx.solve_batch(mus, nus, tol=args.tol)
    torch.cuda.synchronize()
    t = dist.max(time.perf_counter() - t0)
    iters = sum(o["iters"] for o in out)
    vol = sum(2 * b[1] ** 3 for b in batch)
    # algorithmic state traffic: 12 B per flow variable per iteration (FP32 bulk)
    traffic = sum(12.0 * 2 * b[1] ** 3 * o["iters"] for b, o in zip(batch, out))
    peak, peak_kind = measured_peak()
    fin = sorted(o["solve_ms"] for o in out)              # each pair's completion, from the batch's start
    its = sorted(o["iters"] for o in out)

    def pct(v, q):
        return v[min(len(v) - 1, int(round(q * (len(v) - 1))))]

    extra = {"hbm_gbs": round(traffic / t / 1e9, 1), "hbm_frac": round(traffic / t / 1e9 / peak, 4),
             "hbm_note": ("algorithmic state bytes (12 B per flow variable per iteration of each pair) / batch "
                          "time; peak %s (%s)" % (peak, peak_kind)),
             "converged_at_s": {"50%": round(pct(fin, 0.5) / 1e3, 3), "90%": round(pct(fin, 0.9) / 1e3, 3),
                                "99%": round(pct(fin, 0.99) / 1e3, 3), "100%": round(fin[-1] / 1e3, 3)},
             "iterations_per_pair": {"min": its[0], "p50": pct(its, 0.5), "p90": pct(its, 0.9),
                                     "p99": pct(its, 0.99), "max": its[-1], "mean": round(iters / len(its), 1)},
             "iterations_by_size": {str(S): round(statistics.mean(o["iters"] for b, o in zip(batch, out)
                                                                   if b[1] == S), 1)
                                    for S in sorted(set(b[1] for b in batch))}}
    if args.compare_fp64:
        # the plain FP64 single-instance form on the same pairs, one solve at a time
        ctx64 = hot.Context(device=dist.local_rank, precision="fp64", stream=stream.cuda_stream)
        r64 = [ctx64.solve(mus[0], nus[0], tol=args.tol)]          # warm-up
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        r64 = [ctx64.solve(a, b, tol=args.tol) for a, b in zip(mus, nus)]
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t1
        for r in r64:
            ctx64.release(r)
        ctx64.close()
        rel = [abs(a["dual_value"] - b["dual_value"]) / abs(b["dual_value"]) for a, b in zip(out, r64)]
        relp = [abs(a["ot_value"] - b["ot_value"]) / abs(b["ot_value"]) for a, b in zip(out, r64)]
        extra.update({"fp64_sequential": {"solves_per_s": round(args.batch / t64, 2), "seconds": round(t64, 2),
                                          "converged": sum(1 for r in r64 if r["status"] == 0)},
                      "fp32_batch_vs_fp64": {"max_rel_dual": max(rel), "median_rel_dual": statistics.median(rel),
                                             "max_rel_ot": max(relp), "median_rel_ot": statistics.median(relp)}})
    return {"metric": "batched solves/s (512 pairs, S in {32..128})", "value": round(dist.world * args.batch *
                                                                                     args.steps / t, 2),
            "unit": "solves/s", "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000 * t / args.steps, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch of %d pairs" % args.batch, "tol": args.tol},
            "instance_iterations": iters, "converged": sum(1 for o in out if o["status"] == 0),
            "blocks": out[0]["blocks"], "flow_variables": vol, **extra}


def bench_serve(args, dist):
    """Poisson arrivals (mean rate --rate), S in {32,64,128,256,512} weighted
    40/30/15/10/5 %, for --duration seconds; latency p50/p99 and solves/s."""
    import numpy as np
    import torch
    from paper_2408_00598_gb300 import hot
    from paper_2408_00598_gb300 import synthetic as syn
    torch.cuda.set_device(dist.local_rank)
    rng = np.random.default_rng(11 + dist.rank)
    sizes = [32, 64, 128, 256, 512]
    wts = np.array([0.40, 0.30, 0.15, 0.10, 0.05])
    pool = {S: [syn.make_pair(("white", "gauss", "cauchy", "shapes", "translate")[q % 5], S, 100 + q)
                for q in range(4)] for S in sizes}
    ctx = hot.Context(device=dist.local_rank, precision="fp32")
    t_start = time.perf_counter()
    tickets = []
    nxt = t_start
    while True:
        now = time.perf_counter()
        if now - t_start >= args.duration:
            break
        if now >= nxt:
            S = int(rng.choice(sizes, p=wts))
            a, b = pool[S][int(rng.integers(0, 4))]
            tickets.append(ctx.submit(a, b, tol=args.tol))
            nxt += rng.exponential(1.0 / args.rate)
        else:
            time.sleep(min(0.001, nxt - now))
    # drain: wait for the queue at most --max-drain seconds, then cancel what
    # is left (an offered load above capacity never drains; the run reports
    # how much of it was served)
    done = 0
    unserved = 0
    deadline = t_start + args.duration + args.max_drain
    left = []
    for t in tickets:
        left_ms = max(0.0, (deadline - time.perf_counter()) * 1000.0)
        st, _ = ctx.wait(t, timeout_ms=left_ms)
        if st in (hot.HOT_PENDING, hot.HOT_TIMEOUT):
            left.append(t)
        else:
            done += st == hot.HOT_OK
    # past the deadline: cancel everything still pending at once (queued
    # requests leave at once, admitted ones at their next check), then collect
    for t in left:
        ctx.cancel(t)
    for t in left:
        st, _ = ctx.wait(t, timeout_ms=-1)
        if st == hot.HOT_OK:
            done += 1
        else:
            unserved += 1
    t_all = time.perf_counter() - t_start
    s = ctx.serve_stats()
    ctx.close()
    return {"metric": "serve solves/s and p50/p99 latency", "value": round(done / t_all, 3), "unit": "solves/s",
            "n_gpus": dist.world, "steps": len(tickets), "warmup": 0, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "Poisson %g req/s for %gs, S in %s" % (args.rate, args.duration, sizes)},
            "p50_ms": s["p50_ms"], "p99_ms": s["p99_ms"], "mean_queue_ms": s["mean_queue_ms"],
            "completed": s["completed"], "unserved_cancelled": unserved, "submitted": len(tickets),
            "drain_s": round(t_all - args.duration, 2)}


def main():
    args = parse()
    dist = Dist(use_cuda=args.impl == "ours")
    try:
        if args.impl == "reference":
            out = bench_reference(args, dist)
        elif args.mode == "batch":
            out = bench_batch(args, dist)
        elif args.mode == "serve":
            out = bench_serve(args, dist)
        else:
            out = bench_solve(args, dist)
        if out is not None and dist.rank == 0:
            print(json.dumps(out), flush=True)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
