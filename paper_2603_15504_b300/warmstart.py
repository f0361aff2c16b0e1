"""Learned warm start for a parameterised problem family.

The solver produces (parameter, solution) pairs for the family; a network
(pdcs_mlp: BF16 tensor-core GEMMs, Adam) learns the map from the instance
parameters to the solution, both standardised per coordinate; a new instance
is then solved from the network's prediction (x0, y0) unless the solver's own
KKT error of that point (pdcs_kkt, the termination definitions) is larger
than the cold start's, in which case it is solved from the cold start.

Run as a module for the parameterised portfolio family (20,000 assets, 100
factors, 100 limits; mu ~ N(0.05, 0.02^2) and risk aversion log-uniform on
[0.1, 10] per instance):

    python -m paper_2603_15504_b300.warmstart --n 20000 --train 2048 --test 64
"""
import argparse
import json
import os
import sys
import threading
import time

import numpy as np

from . import Batch, Mlp, Solver


class Standardiser:
    """Per-coordinate z-scores with a floor on the spread (constant
    coordinates map to 0)."""

    def __init__(self, data, floor=1e-12):
        self.mean = data.mean(axis=0)
        sd = data.std(axis=0)
        self.sd = np.where(sd > floor, sd, 1.0)

    def encode(self, v):
        return (v - self.mean) / self.sd

    def decode(self, z):
        return self.mean + self.sd * z


def collect(factories, workers=8, **options):
    """Build and solve every instance (the plain path, cold start) with up to
    `workers` concurrent solver handles.  factories[i]() returns (problem,
    parameters).  Returns (parameters [N x p], solutions [N x (n + m)],
    per-instance results)."""
    params = [None] * len(factories)
    sols = [None] * len(factories)
    res = [None] * len(factories)
    lock = threading.Lock()
    nxt = [0]
    errors = []

    def work():
        while True:
            with lock:
                i = nxt[0]
                nxt[0] += 1
            if i >= len(factories) or errors:
                return
            try:
                prob, par = factories[i]()
                with Solver(prob, **options) as s:
                    r = s.solve()
            except Exception as e:  # noqa: BLE001
                errors.append(e)
                return
            params[i] = par
            sols[i] = np.concatenate([r["x"], r["y"]])
            res[i] = {k: r[k] for k in ("iters", "solve_time_s", "exit_code", "err_rel_p",
                                        "err_rel_d", "err_rel_gap")}

    threads = [threading.Thread(target=work) for _ in range(max(1, workers))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    return np.array(params), np.array(sols), res


def _progress(**kw):
    print(json.dumps(kw), file=sys.stderr, flush=True)


def collect_batched(factories, chunk=512, verbose=False, **options):
    """As collect, but every `chunk` instances are solved together in one
    persistent launch of the batched engine (pdcs_setup_batch /
    pdcs_solve_batch; FP64, each instance with its own step sizes, restarts
    and termination)."""
    params, sols, res = [], [], []
    for c0 in range(0, len(factories), chunk):
        t0 = time.perf_counter()
        probs = []
        for f in factories[c0:c0 + chunk]:
            prob, par = f()
            probs.append(prob)
            params.append(par)
        with Batch(probs, **options) as b:
            out = b.solve()
        for r in out:
            sols.append(np.concatenate([r["x"], r["y"]]))
            res.append({k: r[k] for k in ("iters", "solve_time_s", "exit_code", "err_rel_p",
                                          "err_rel_d", "err_rel_gap")})
        if verbose:
            _progress(stage="data", done=len(res), chunk_s=time.perf_counter() - t0,
                      reached=int(sum(r["exit_code"] == 0 for r in res[-len(out):])))
    return np.array(params), np.array(sols), res


class WarmStart:
    """Network from instance parameters to (x, y), with the standardisers."""

    def __init__(self, params, sols, n, hidden=512, n_hidden=3, batch=256, lr=1e-3, seed=1):
        self.n = n
        self.fin = Standardiser(params)
        self.fout = Standardiser(sols)
        self.batch = batch
        self.net = Mlp(params.shape[1], sols.shape[1], hidden=hidden, n_hidden=n_hidden,
                       max_batch=batch, lr=lr, seed=seed)
        self.X = self.fin.encode(params).astype(np.float32)
        self.T = self.fout.encode(sols).astype(np.float32)

    def fit(self, steps, seed=0):
        rng = np.random.default_rng(seed)
        N = self.X.shape[0]
        losses = []
        for _ in range(steps):
            idx = rng.choice(N, size=min(self.batch, N), replace=False)
            losses.append(self.net.train_step(self.X[idx], self.T[idx]))
        return losses

    def predict(self, params):
        z = self.net.predict(self.fin.encode(np.atleast_2d(params)).astype(np.float32))
        s = self.fout.decode(z.astype(np.float64))
        return s[:, :self.n], s[:, self.n:]

    def solve(self, prob, params, **options):
        """Solve from the prediction, or from the cold start when the
        prediction's KKT error is the larger one.  Returns the result plus
        `warm` (start used), the two KKT errors and the prediction time."""
        t0 = time.perf_counter()
        x0, y0 = self.predict(params)
        t_pred = time.perf_counter() - t0
        with Solver(prob, **options) as s:
            t1 = time.perf_counter()
            kw = s.kkt(x0[0], y0[0])["max_rel"]
            kc = s.kkt()["max_rel"]
            warm = kw <= kc
            r = s.solve(x0[0] if warm else None, y0[0] if warm else None)
            t_solve = time.perf_counter() - t1
        r.update(warm=warm, kkt_pred=kw, kkt_cold=kc, predict_s=t_pred, wall_s=t_pred + t_solve)
        return r


def _main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--k", type=int, default=100)
    ap.add_argument("--limits", type=int, default=100)
    ap.add_argument("--train", type=int, default=2048)
    ap.add_argument("--test", type=int, default=64)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--data-tol", type=float, default=1e-6)
    ap.add_argument("--plain-data", action="store_true",
                    help="generate the training data with one plain solve per instance")
    ap.add_argument("--chunk", type=int, default=592,
                    help="instances per batched launch of the data generation")
    args = ap.parse_args()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import workloads  # seeded generators of the family (no solver arithmetic)
    fam = workloads.portfolio_family(n=args.n, k=args.k, n_limits=args.limits)
    make = lambda split, i: workloads.portfolio_family_instance(fam, i, split_seed=split)  # noqa: E731
    opts = dict(rel_tol=args.data_tol, time_limit=600.0)
    t0 = time.perf_counter()
    facs = [(lambda i=i: make(0, i)) for i in range(args.train)]
    if args.plain_data:
        params, sols, res = collect(facs, workers=args.workers, **opts)
    else:
        params, sols, res = collect_batched(facs, chunk=args.chunk, verbose=True, **opts)
    t_data = time.perf_counter() - t0
    t1 = time.perf_counter()
    ws = WarmStart(params, sols, n=args.n + 1)
    losses = ws.fit(args.steps)
    t_train = time.perf_counter() - t1
    _progress(stage="train", seconds=t_train, loss_first=losses[0],
              loss_last=float(np.mean(losses[-20:])))
    rows = []
    for i in range(args.test):
        prob, p = make(1, i)
        with Solver(prob, rel_tol=1e-6, time_limit=600.0) as s:
            c = s.solve()
        w = ws.solve(prob, p, rel_tol=1e-6, time_limit=600.0)
        x0, y0 = ws.predict(p)
        ex = np.linalg.norm(x0[0] - c["x"]) / max(1e-300, np.linalg.norm(c["x"]))
        ey = np.linalg.norm(y0[0] - c["y"]) / max(1e-300, np.linalg.norm(c["y"]))
        _progress(stage="test", i=i, cold_iters=c["iters"], warm_iters=w["iters"],
                  warm=bool(w["warm"]), cold_s=c["solve_time_s"], warm_s=w["wall_s"])
        rows.append(dict(cold_iters=c["iters"], cold_s=c["solve_time_s"], warm_iters=w["iters"],
                         err_x=ex, err_y=ey,
                         warm_s=w["wall_s"], warm=bool(w["warm"]), kkt_pred=w["kkt_pred"],
                         kkt_cold=w["kkt_cold"], cold_ok=c["exit_code"] == 0,
                         warm_ok=w["exit_code"] == 0))
    ci = np.array([r["cold_iters"] for r in rows], float)
    wi = np.array([r["warm_iters"] for r in rows], float)
    cs = np.array([r["cold_s"] for r in rows])
    wsec = np.array([r["warm_s"] for r in rows])
    data_ok = all(r["exit_code"] == 0 for r in res)
    print(json.dumps({
        "family": "portfolio n=%d k=%d limits=%d" % (args.n, args.k, args.limits),
        "train_instances": args.train, "test_instances": args.test,
        "data_seconds": t_data, "data_mean_iters": float(np.mean([r["iters"] for r in res])),
        "data_all_reached_tol": bool(data_ok),
        "data_generation": "one plain solve per instance" if args.plain_data else
                           "batched engine, %d instances per launch" % args.chunk,
        "train_seconds": t_train, "train_steps": args.steps,
        "loss_first": losses[0], "loss_last": float(np.mean(losses[-20:])),
        "cold_iters_mean": ci.mean(), "warm_iters_mean": wi.mean(),
        "iters_ratio_median": float(np.median(wi / ci)),
        "cold_seconds_mean": cs.mean(), "warm_seconds_mean": wsec.mean(),
        "warm_used": int(sum(r["warm"] for r in rows)),
        "pred_rel_err_x_median": float(np.median([r["err_x"] for r in rows])),
        "pred_rel_err_y_median": float(np.median([r["err_y"] for r in rows])),
        "kkt_pred_median": float(np.median([r["kkt_pred"] for r in rows])),
        "kkt_cold_median": float(np.median([r["kkt_cold"] for r in rows])),
        "all_reached_tol": bool(all(r["cold_ok"] and r["warm_ok"] for r in rows)),
    }))


if __name__ == "__main__":
    _main()
