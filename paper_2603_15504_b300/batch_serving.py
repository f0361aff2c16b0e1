"""Batched serving workload: many independent factor-model portfolio SOCPs of
uneven size (n ~ U{50..2000} assets, n / 20 factors, ceil(n / 200) limits)
solved in one persistent kernel launch (pdcs_setup_batch / pdcs_solve_batch,
FP32 bulk with FP64 reductions and control), against the plain FP64 path
(one pdcs_setup + pdcs_solve per problem) on an evenly spaced sample.

    python -m paper_2603_15504_b300.batch_serving --count 4096 --sample 64

Prints one JSON object: per-problem time to tolerance on its thread block
(p50 / p99), the batch's wall time and solves per second, iterations, and
the plain path's time per problem on the sample, scaled to the whole batch.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

from . import Batch, solve


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=4096)
    ap.add_argument("--n-lo", type=int, default=50)
    ap.add_argument("--n-hi", type=int, default=2000)
    ap.add_argument("--sample", type=int, default=64)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--seed", type=int, default=20260104)
    args = ap.parse_args()
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads  # seeded instance generator (no solver arithmetic)

    t0 = time.perf_counter()
    probs = workloads.portfolio_batch(count=args.count, n_lo=args.n_lo, n_hi=args.n_hi,
                                      seed=args.seed)
    t_gen = time.perf_counter() - t0
    nnz = np.array([len(p["val"]) for p in probs])
    t1 = time.perf_counter()
    b = Batch(probs, precision=args.precision, time_limit=600.0)
    t_setup = time.perf_counter() - t1
    t2 = time.perf_counter()
    out = b.solve()
    t_solve = time.perf_counter() - t2
    b.close()
    per = np.array([r["solve_time_s"] for r in out])
    its = np.array([r["iters"] for r in out])
    ok = np.array([r["exit_code"] == 0 for r in out])
    # plain FP64 path on an evenly spaced sample (by size order), scaled by nnz
    order = np.argsort(nnz)
    pick = order[np.linspace(0, len(order) - 1, min(args.sample, len(order))).astype(int)]
    plain_t, plain_ok, agree = [], [], []
    for k in pick:
        t3 = time.perf_counter()
        g = solve(probs[k], time_limit=600.0)
        plain_t.append(time.perf_counter() - t3)
        plain_ok.append(g["exit_code"] == 0)
        agree.append(abs(g["pobj"] - out[k]["pobj"]) / (1.0 + abs(g["pobj"])))
    plain_t = np.array(plain_t)
    plain_total_est = float(np.sum(plain_t) * args.count / len(pick))
    print(json.dumps({
        "workload": "%d portfolio SOCPs, n ~ U{%d..%d}, k = n/20, ceil(n/200) limits"
                    % (args.count, args.n_lo, args.n_hi),
        "precision": args.precision, "total_nnz": int(nnz.sum()),
        "generate_s": t_gen, "setup_s": t_setup, "batch_solve_s": t_solve,
        "solves_per_s": args.count / t_solve,
        "per_problem_s_p50": float(np.percentile(per, 50)),
        "per_problem_s_p99": float(np.percentile(per, 99)),
        "iters_p50": float(np.percentile(its, 50)), "iters_p99": float(np.percentile(its, 99)),
        "all_reached_tol": bool(ok.all()), "reached": int(ok.sum()),
        "plain_fp64_sample": int(len(pick)), "plain_fp64_s_mean": float(plain_t.mean()),
        "plain_fp64_total_s_estimate": plain_total_est,
        "plain_all_reached_tol": bool(all(plain_ok)),
        "objective_rel_diff_max": float(max(agree)),
        "speedup_vs_plain_estimate": plain_total_est / t_solve,
    }))


if __name__ == "__main__":
    main()
