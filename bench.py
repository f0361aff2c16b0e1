#!/usr/bin/env python
"""Benchmark of the restarted-PDHG conic solver on one B300 per rank.

Workload: the factor-model portfolio SOCP (n = 200,000 assets, k = 200 factors,
1,000 sparse linear limits, one rotated SOC of dimension k + n + 2), generated
from a seed; m = 201,203 rows, n = 200,001 columns, 40.6M nonzeros.

A step is one check period of the method: 64 accepted PDHG iterations (each an
adaptive-step attempt with G xhat, the dual and primal updates and projections,
G^T yhat, maxErr and the reflected Halpern update) plus one restart / termination
check (average candidate, KKT statistics, normalized-gap bisection).  The metric
is PDHG iterations per second over the K timed steps; time to 1e-6 relative KKT
error is reported beside it.

Multi-GPU (torchrun): each rank solves its own instance (seed + rank); there is
no data-path collective, only a barrier and a max over ranks of the timed region
("weak" scaling; a single instance does not shard).

--impl reference times the FP64 CPU oracle (the reference arm of this build) on
the same workload, rank 0 only.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-6 rel. KKT & PDHG iters/s; batched and warm-start vs plain FP64"
UNIT = "PDHG iterations/s"
CHECK_FREQ = 64
# FP64 peak from unit counts and clocks: 148 SMs x 2 DFMA per SM per cycle
# (ncu's sm__sass_thread_inst_executed_op_dfma_pred_on peak_sustained on this
# part) x 2 flops x 2.032 GHz maximum SM clock = 1.203 TFLOP/s (nominal 1.25)
FP64_PEAK_TFLOPS = 148 * 2 * 2 * 2.032e9 / 1e12
# DRAM bytes per launch of the two products (G xhat with the dual step, G^T
# yhat) from one ncu capture, keyed by (workload, precision, source digest of
# spmv.cuh at capture time); missing (traffic null) once the kernel changed.
# The capture ran the n = 100,000 portfolio (20,250,124 nonzeros); traffic
# grows with the nonzeros, so it is scaled by 40,600,072 / 20,250,124 to the
# n = 200,000 workload.
_NNZ_SCALE = 40_600_072 / 20_250_124
NCU_TRAFFIC = {
    ("portfolio", "fp64", "ecbed7b9c912708a"): (170.266e6 * _NNZ_SCALE, 197.234e6 * _NNZ_SCALE),
    ("portfolio", "fp32", "ecbed7b9c912708a"): (88.481e6 * _NNZ_SCALE, 100.594e6 * _NNZ_SCALE),
}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--n", type=int, default=200_000)
    ap.add_argument("--k", type=int, default=200)
    ap.add_argument("--limits", type=int, default=1000)
    ap.add_argument("--workload", default="portfolio", choices=["portfolio", "logistic"],
                    help="portfolio: the factor-model SOCP (the headline); logistic: the "
                         "L1-logistic regression with 200,000 exponential cones")
    ap.add_argument("--tts-cap", type=float, default=90.0,
                    help="time limit (s) of the time-to-tolerance solve; 0 skips it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--oracle-iters", type=int, default=12)
    ap.add_argument("--eager", action="store_true",
                    help="launch kernels from the host (for per-kernel profilers)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra keys (FP32 portfolio, logistic, 4096-instance batch)")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--oracle-procs", type=int, default=8,
                    help="processes of the all-cores oracle leg (independent copies)")
    ap.add_argument("--overlap", type=int, default=0, choices=[0, 1],
                    help="programmatic dependent launches in the captured loops (option "
                         "overlap_launches)")
    ap.add_argument("--ab", action="store_true",
                    help="instead of the bench line: time to 1e-6 on the workload for the "
                         "restart-check period 64 against the paper's 2000, and for the "
                         "bisection tolerance of Algorithm 3 (1e-6 against 1e-3)")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _aggregate(elapsed, iters, ws, dev=None):
    """Whole-job figures of the timed region: the maximum of the ranks'
    barrier-bracketed times and the sum of their iterations (one instance per
    rank, no data-path collective).  Works on any torch.distributed backend
    (NCCL with CUDA tensors, gloo with CPU tensors)."""
    if ws == 1:
        return elapsed, iters
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(iters)], device=dev, dtype=torch.float64)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(c.item())


def _workload(args, rank):
    import workloads
    if getattr(args, "workload", "portfolio") == "logistic":
        p = workloads.logistic_l1(seed=20260103 + rank)
        desc = ("L1-logistic regression in exponential-cone form, 100000 samples x 2000 "
                "features (m=%d, n=%d, nnz=%d, %d exponential cones), %s"
                % (p["m"], p["n"], len(p["val"]), 2 * 100000, args.precision.upper()))
        return p, desc
    p = workloads.portfolio(n=args.n, k=args.k, n_limits=args.limits, seed=20260102 + rank)
    desc = ("factor-model portfolio SOCP n=%d k=%d limits=%d (m=%d, n=%d, nnz=%d), %s"
            % (args.n, args.k, args.limits, p["m"], p["n"], len(p["val"]), args.precision.upper()))
    return p, desc


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def _spmv_digest():
    import hashlib
    src = open(os.path.join(ROOT, "paper_2603_15504_b300", "csrc", "spmv.cuh"), "rb").read()
    return hashlib.sha256(src).hexdigest()[:16]


def _oracle_sample(prob, iters):
    """The FP64 CPU oracle, as it stands, on the same instance: set-up, then
    `iters` accepted PDHG iterations; returns (iterations/s of the loop, setup s)."""
    import oracle
    t0 = time.perf_counter()
    o = oracle.Oracle(oracle.problem_from_dict(prob), oracle.Options(max_iter=iters,
                                                                     check_freq=CHECK_FREQ))
    t1 = time.perf_counter()
    r = o.solve()
    t2 = time.perf_counter()
    return r["iters"] / (t2 - t1), t1 - t0, r["iters"], t2 - t1


def _oracle_child(args, out_path):
    """Run the oracle sample in a child process (one BLAS thread) so it
    overlaps the GPU measurement; writes its result as JSON."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "a=bench._args_from(%r); p,_=bench._workload(a, 0); "
            "v,su,it,dt=bench._oracle_sample(p, a.oracle_iters); "
            "json.dump(dict(value=v, setup_s=su, iters=it, loop_s=dt), open(%r,'w'))"
            % (ROOT, sys.argv[1:], out_path))
    return subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT,
                            stdout=subprocess.DEVNULL, stderr=subprocess.PIPE)


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def _oracle_multi(args, procs):
    """The all-cores leg: `procs` oracle processes (one thread each), each on
    its own copy of the same instance, started together; the aggregate rate
    is the sum of their iterations / s.  Returns the child processes and
    their output files."""
    kids = []
    for _ in range(procs):
        fd, path = tempfile.mkstemp(suffix=".json")
        os.close(fd)
        kids.append((_oracle_child(args, path), path))
    return kids


def _args_from(argv):
    old = sys.argv
    try:
        sys.argv = ["bench.py"] + list(argv)
        return _args()
    finally:
        sys.argv = old


def _timed_window(P, prob, opts, warmup, steps):
    """Iterations / s of `steps` check periods after `warmup` ones (CUDA events
    on the current stream around a pdcs_resume; synchronised)."""
    import torch
    with P.Solver(prob, **dict(opts, max_iter=warmup * CHECK_FREQ, profile=0)) as s:
        r0 = s.solve()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        r1 = s.resume(max_iter=r0["iters"] + steps * CHECK_FREQ)
        e1.record()
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) / 1000.0
    return (r1["iters"] - r0["iters"]) / dt


def _tts(P, prob, opts, cap):
    with P.Solver(prob, **dict(opts, time_limit=cap, max_iter=2**62, profile=0)) as st:
        t = time.perf_counter()
        r = st.solve()
        dt = time.perf_counter() - t
    return r, {"reached": r["exit_code"] == 0, "seconds": dt, "iters": r["iters"],
               "rel_kkt": max(r["err_rel_p"], r["err_rel_d"], r["err_rel_gap"]),
               "status": r["status"]}


def _extra_fp32(P, prob, ref64, cap):
    """FP32 mode (FP32 matrix values and float-float products, FP64 vectors,
    FP64 products at the checks) on the headline instance: its rate, time to
    1e-6, and the distance of its result from the FP64 path's (which the
    parity tests tie to the oracle)."""
    opts = dict(precision="fp32", check_freq=CHECK_FREQ, time_limit=3600.0)
    out = {"iters_per_s": _timed_window(P, prob, opts, 3, 10)}
    r, out["time_to_tol"] = _tts(P, prob, opts, cap)
    if ref64 is not None:
        def rel(a, b):
            return float(np.linalg.norm(a - b) / max(1e-300, np.linalg.norm(b)))
        out["error_vs_fp64_path"] = {
            "pobj_rel": abs(r["pobj"] - ref64["pobj"]) / (1.0 + abs(ref64["pobj"])),
            "x_rel": rel(r["x"], ref64["x"]), "y_rel": rel(r["y"], ref64["y"])}
    return out


def _extra_logistic(P, cap):
    """The L1-logistic regression (100,000 samples x 2,000 features, 200,000
    exponential cones), FP64: rate, time to 1e-6 and the exponential-cone
    projection's share and throughput (cones / s over its launches)."""
    import torch
    import workloads
    prob = workloads.logistic_l1(seed=20260103)
    opts = dict(precision="fp64", check_freq=CHECK_FREQ, time_limit=3600.0)
    out = {"workload": "L1-logistic 100000 x 2000 (m=%d, n=%d, nnz=%d, 200000 exp cones)"
                       % (prob["m"], prob["n"], len(prob["val"]))}
    out["iters_per_s"] = _timed_window(P, prob, opts, 3, 10)
    _, out["time_to_tol"] = _tts(P, prob, opts, cap)
    with P.Solver(prob, **dict(opts, profile=1, max_iter=10 * CHECK_FREQ)) as sp:
        torch.cuda.synchronize()
        t = time.perf_counter()
        sp.solve()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t
        kt = sp.kernel_times()
    tot = sum(v[0] for v in kt.values())
    exp_s, exp_n = kt.get("exp", (0.0, 0))
    # rows carry 200,000 cones; each launch projects two vectors of them
    out["exp_projection"] = {"share_of_kernel_time": exp_s / tot if tot else None,
                             "launches": exp_n, "us_per_launch": 1e6 * exp_s / exp_n if exp_n else None,
                             "cones_per_s": 2 * 200000 * exp_n / exp_s if exp_s else None,
                             "window_s": wall}
    return out


def _extra_batch(P, count):
    """4096 portfolio SOCPs of uneven size (n ~ U{50..2000}, k = n/20,
    ceil(n/200) limits) in one persistent launch, FP64: solves / s, per-instance
    time to tolerance p50 / p99, and the plain FP64 path (one set-up and solve
    per problem) on an evenly spaced sample of 16, scaled to the batch."""
    import workloads
    t = time.perf_counter()
    probs = workloads.portfolio_batch(count=count)
    gen = time.perf_counter() - t
    nnz = np.array([len(p["val"]) for p in probs])
    t = time.perf_counter()
    b = P.Batch(probs, precision="fp64", time_limit=600.0)
    setup = time.perf_counter() - t
    t = time.perf_counter()
    res = b.solve()
    solve_s = time.perf_counter() - t
    b.close()
    per = np.array([r["solve_time_s"] for r in res])
    ok = np.array([r["exit_code"] == 0 for r in res])
    order = np.argsort(nnz)
    pick = order[np.linspace(0, len(order) - 1, min(16, len(order))).astype(int)]
    plain, agree = [], []
    for k in pick:
        t = time.perf_counter()
        g = P.solve(probs[k], time_limit=600.0)
        plain.append(time.perf_counter() - t)
        agree.append(abs(g["pobj"] - res[k]["pobj"]) / (1.0 + abs(g["pobj"])))
    plain_est = float(np.mean(plain) * count)
    return {"workload": "%d portfolio SOCPs, n ~ U{50..2000}, k = n/20 (%.0fM nonzeros)"
                        % (count, nnz.sum() / 1e6),
            "solves_per_s": count / solve_s, "batch_solve_s": solve_s, "setup_s": setup,
            "generate_s": gen, "per_instance_s_p50": float(np.percentile(per, 50)),
            "per_instance_s_p99": float(np.percentile(per, 99)), "all_reached": bool(ok.all()),
            "reached": int(ok.sum()), "plain_fp64_sample": len(pick),
            "plain_fp64_s_mean": float(np.mean(plain)), "plain_fp64_total_s_estimate": plain_est,
            "speedup_vs_plain_estimate": plain_est / solve_s,
            "objective_rel_diff_max_vs_plain": float(max(agree))}


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2603_15504_b300 as P

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    oracle_proc, oracle_out, oracle_kids = None, None, []
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        fd, oracle_out = tempfile.mkstemp(suffix=".json")
        os.close(fd)
        oracle_proc = _oracle_child(args, oracle_out)

    prob, desc = _workload(args, rank)
    # the timed window runs without the in-kernel timers (they cost about 4 %
    # of a step); the per-kernel times and the roofline come from a second,
    # profiled window over the same number of steps right after it
    opts = dict(precision=args.precision, check_freq=CHECK_FREQ, profile=0, time_limit=3600.0,
                eager=int(args.eager), overlap_launches=args.overlap)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()

    t0 = time.perf_counter()
    s = P.Solver(prob, **dict(opts, max_iter=args.warmup * CHECK_FREQ))
    setup_s = time.perf_counter() - t0
    r0 = s.solve()  # warm-up periods; the timed steps continue this trajectory
    it0 = r0["iters"]
    kb0 = r0["attempts"]
    clocks = Clocks(local)
    barrier()
    clocks.start()
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    r1 = s.resume(max_iter=it0 + args.steps * CHECK_FREQ)
    ev1.record(stream)
    barrier()
    elapsed = ev0.elapsed_time(ev1) / 1000.0
    ck = clocks.stop()
    counts = s.profile()  # launch counts (kept without timers)
    iters = r1["iters"] - it0
    attempts = r1["attempts"] - kb0
    tmax, it_all = _aggregate(elapsed, iters, ws, dev)
    value = it_all / tmax
    s.close()

    # profiled window: same warm-up and step count, in-kernel timers on
    with P.Solver(prob, **dict(opts, profile=1, max_iter=args.warmup * CHECK_FREQ)) as sp:
        p0 = sp.solve()
        barrier()
        evp0 = torch.cuda.Event(enable_timing=True)
        evp1 = torch.cuda.Event(enable_timing=True)
        evp0.record(stream)
        sp.resume(max_iter=p0["iters"] + args.steps * CHECK_FREQ)
        evp1.record(stream)
        barrier()
        elapsed_prof = evp0.elapsed_time(evp1) / 1000.0
        prof = sp.profile()
        ktimes = sp.kernel_times()

    # roofline of the dominant kernel (the two sparse products), measured live
    peaks, peak_kind = _peaks()
    sp_time = prof["g_seconds"] + prof["gt_seconds"]
    sp_bytes = prof["g_bytes"] * prof["g_launches"] + prof["gt_bytes"] * prof["gt_launches"]
    launches = prof["g_launches"] + prof["gt_launches"]
    achieved = sp_bytes / sp_time / 1e9 if sp_time > 0 else None
    tr = NCU_TRAFFIC.get((args.workload, args.precision, _spmv_digest()))
    traffic = ((tr[0] * prof["g_launches"] + tr[1] * prof["gt_launches"]) / launches
               if tr and launches else None)
    hbm = {"bound": "hbm", "kernel": "k_spmv (G xhat and G^T yhat)",
           "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": achieved / peaks["hbm_gbs"] if achieved else None,
           "traffic": traffic, "peak_source": peak_kind,
           "algorithmic_bytes_per_launch": sp_bytes / launches if launches else None,
           "avg_launch_us": 1e6 * sp_time / launches if launches else None,
           "launches": launches,
           "spmv_time_share": sp_time / elapsed_prof if elapsed_prof else None,
           "window": "profiled window of %d steps after the timed one (in-kernel timers, "
                     "first CTA start to last CTA end per launch)" % args.steps}
    roofline = hbm
    if args.precision == "fp64" and sp_time > 0:
        # one FP64 FMA per nonzero: against the FP64 rate of the part (derived
        # above from its DFMA units and clock), the product is closer to its
        # arithmetic bound than to HBM once the column runs drop most index
        # bytes
        flops = prof["nnz_flops"] * launches / sp_time / 1e12
        alu = dict(hbm, bound="alu", achieved=flops, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s",
                   frac=flops / FP64_PEAK_TFLOPS,
                   peak_source="derived: 148 SMs x 2 DFMA/cycle x 2 flops x 2.032 GHz "
                               "(no measured FP64 peak)")
        if alu["frac"] > (hbm["frac"] or 0.0):
            roofline = alu
            roofline["hbm"] = {k: hbm[k] for k in ("achieved", "peak", "unit", "frac", "traffic",
                                                   "peak_source")}
        else:
            roofline["fp64_alu"] = {k: alu[k] for k in ("achieved", "peak", "unit", "frac",
                                                        "peak_source")}

    # end to end through the public API: set-up from pinned host arrays (H2D
    # inside the timed region), K periods from a cold start, solution back to
    # pinned host buffers.
    e2e = None
    if not args.no_e2e:
        import torch as _t
        host = {}
        h2d = 0
        for key in ("row_ptr", "col_idx", "val", "h", "c", "lo", "hi"):
            a = _t.from_numpy(np.ascontiguousarray(prob[key])).pin_memory()
            host[key] = a
            h2d += a.numel() * a.element_size()
        hp = dict(prob, **host)
        outs = tuple(_t.empty(k, dtype=_t.float64).pin_memory() for k in (prob["n"], prob["m"], prob["m"]))
        barrier()
        t1 = time.perf_counter()
        with P.Solver(hp, **dict(opts, max_iter=args.steps * CHECK_FREQ, profile=0)) as se:
            re = se.solve(out=outs)
        barrier()
        te = time.perf_counter() - t1
        d2h = sum(o.numel() * o.element_size() for o in outs)
        e2e = {"value": re["iters"] / te, "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "seconds": te, "includes": "pdcs_setup from pinned host CSR + pdcs_solve of "
               "%d iterations + copy of x, y, s to pinned host" % (args.steps * CHECK_FREQ)}

    # time to 1e-6 relative KKT error
    tts = None
    rt = None
    if args.tts_cap > 0 and rank == 0:
        with P.Solver(prob, **dict(opts, time_limit=args.tts_cap, max_iter=2**62, profile=0)) as st:
            t2 = time.perf_counter()
            rt = st.solve()
            tt = time.perf_counter() - t2
        tts = {"reached": rt["exit_code"] == 0, "seconds": tt, "setup_s": setup_s,
               "iters": rt["iters"], "attempts": rt["attempts"], "restarts": rt["restarts"],
               "rel_kkt": max(rt["err_rel_p"], rt["err_rel_d"], rt["err_rel_gap"]),
               "status": rt["status"], "time_cap_s": args.tts_cap}
        if args.precision == "fp32":
            # error of the FP32 result against the FP64 path (the path the
            # parity tests tie to the FP64 oracle), same instance and cap
            with P.Solver(prob, **dict(opts, precision="fp64", time_limit=args.tts_cap,
                                       max_iter=2**62, profile=0)) as s64:
                r64 = s64.solve()
            def rel(a, b):
                return float(np.linalg.norm(a - b) / max(1e-300, np.linalg.norm(b)))
            tts["error_vs_fp64_path"] = {
                "pobj_rel": abs(rt["pobj"] - r64["pobj"]) / (1.0 + abs(r64["pobj"])),
                "x_rel": rel(rt["x"], r64["x"]), "y_rel": rel(rt["y"], r64["y"]),
                "fp64_rel_kkt": max(r64["err_rel_p"], r64["err_rel_d"], r64["err_rel_gap"]),
                "fp64_reached": r64["exit_code"] == 0}

    # extra workloads of the same metric (N = 1 only): FP32 mode of the
    # headline instance, the exponential-cone program, the 4096-instance batch
    extras = None
    if rank == 0 and ws == 1 and not args.no_extras and args.workload == "portfolio":
        extras = {}
        for name, fn in (("fp32_portfolio", lambda: _extra_fp32(
                              P, prob, rt if args.precision == "fp64" else None, args.tts_cap)),
                         ("logistic_exp_cones", lambda: _extra_logistic(P, 120.0)),
                         ("batch_4096_portfolios", lambda: _extra_batch(P, args.batch_count))):
            try:
                extras[name] = fn()
            except Exception as e:  # noqa: BLE001 -- reported, not fatal for the line
                extras[name] = {"error": repr(e)[:300]}

    cpu = None
    if oracle_proc is not None:
        _, err = oracle_proc.communicate(timeout=1800)
        try:
            o = json.load(open(oracle_out))
            cpu = {"value": o["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
                   "cpu_model": _cpu_model(), "host_cores": os.cpu_count(),
                   "sample": "FP64 CPU oracle on the same instance: %d accepted PDHG iterations "
                             "after its set-up (%.0f s, not counted)" % (o["iters"], o["setup_s"])}
        except (OSError, ValueError, KeyError):
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": "oracle run failed: %s" % err.decode()[-200:]}
        os.unlink(oracle_out)
        # the all-cores leg, after the GPU work (independent processes, one
        # thread each, each on its own copy of the instance)
        nproc = max(1, min(args.oracle_procs, os.cpu_count() or 1))
        if nproc > 1:
            kids = _oracle_multi(args, nproc)
            rates = []
            for kp, path in kids:
                kp.communicate(timeout=1800)
                try:
                    rates.append(json.load(open(path))["value"])
                except (OSError, ValueError, KeyError):
                    pass
                os.unlink(path)
            cpu["all_cores"] = {"value": sum(rates) if len(rates) == nproc else None,
                                "unit": UNIT, "cores": nproc, "kind": "oracle",
                                "sample": "%d oracle processes at once, each %d accepted "
                                          "iterations of its own copy of the instance; value = "
                                          "sum of their rates" % (nproc, args.oracle_iters)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000.0 * tmax / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else "f32",
                "data": "synthetic (seeded %s generator)" % (
                    "L1-logistic" if args.workload == "logistic" else "factor-model portfolio"),
                "config": {"workload": desc, "step": "%d accepted PDHG iterations + 1 restart check"
                           % CHECK_FREQ, "parallelism": "replicas" if ws > 1 else "single",
                           "l2": "inputs larger than L2 (two CSR copies of G, %.0f MB)"
                           % (2 * len(prob["val"]) * (12 if args.precision == "fp64" else 8) / 1e6)},
                "attempts_per_s": attempts / elapsed, "setup_s": setup_s,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": counts["kernel_launches"], "graph_launches": counts["graph_launches"],
                "clocks": ck, "time_to_tol": tts,
                "profiled_ms_per_step": 1000.0 * elapsed_prof / args.steps,
                "kernel_seconds": {k: [round(v[0], 6), v[1]] for k, v in ktimes.items()},
                "extras": extras}
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def run_ab(args):
    """A/B of method options on the workload (one JSON line, not the bench
    contract line): time and iterations to 1e-6 relative KKT error."""
    import paper_2603_15504_b300 as P
    prob, desc = _workload(args, 0)
    arms = [("check_freq=64, bisect_rel_tol=1e-3 (defaults)", dict(check_freq=64)),
            ("check_freq=2000 (the paper's restart frequency)", dict(check_freq=2000)),
            ("check_freq=64, bisect_rel_tol=1e-6", dict(check_freq=64, bisect_rel_tol=1e-6))]
    out = []
    for name, o in arms:
        opts = dict(precision=args.precision, profile=0, time_limit=3600.0, **o)
        _, t = _tts(P, prob, opts, args.tts_cap)
        t["arm"] = name
        out.append(t)
    print(json.dumps({"ab": out, "workload": desc, "cap_s": args.tts_cap}))


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    prob, desc = _workload(args, 0)
    import oracle
    o = oracle.Oracle(oracle.problem_from_dict(prob),
                      oracle.Options(max_iter=args.warmup + args.steps, check_freq=CHECK_FREQ))
    # one step = one accepted PDHG iteration of the oracle; warm-up iterations
    # are run first, the timed steps continue the same trajectory
    trace = []
    t_marks = []

    class Clock(list):
        def append(self, rec):
            t_marks.append(time.perf_counter())
            super().append(rec)

    tr = Clock()
    t0 = time.perf_counter()
    o.solve(trace=tr)
    del trace
    n = len(t_marks)
    if n > args.warmup:
        dt = t_marks[-1] - t_marks[args.warmup - 1] if args.warmup > 0 else t_marks[-1] - t0
        steps = n - args.warmup
    else:
        dt, steps = t_marks[-1] - t0, n
    value = steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded factor-model portfolio generator)",
            "config": {"workload": desc, "step": "1 accepted PDHG iteration of the FP64 CPU oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d timed oracle iterations after %d warm-up iterations"
                                       % (steps, args.warmup)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    elif a.ab:
        run_ab(a)
    else:
        run_ours(a)
