"""Batched persistent solves (pdcs_setup_batch / pdcs_solve_batch): every
problem of a mixed batch reaches the tolerance with the objective of its own
single-problem solve, the outputs are deterministic, and an FP32-bulk batch
of portfolios of uneven size agrees with FP64 single solves."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_15504_b300 as P
    return P


def _mixed():
    probs = [workloads.tiny_conic(seed=s, m_nonneg=20, soc_rows=(6, 5), nb=30, soc_cols=(5, 4))
             for s in range(3)]
    probs += [workloads.portfolio_small_instance(n, seed) for n, seed in ((50, 1), (120, 2), (300, 3))]
    probs.append(workloads.logistic_l1(N=60, p=8, density=0.3, support=3, seed=4))
    return probs


def test_mixed_batch_matches_single_solves_and_is_deterministic():
    P = _P()
    probs = _mixed()
    with P.Batch(probs, time_limit=120.0) as b:
        out = b.solve()
        out2 = b.solve()
    for k, (prob, r) in enumerate(zip(probs, out)):
        assert r["exit_code"] == 0, (k, r["status"])
        assert max(r["err_rel_p"], r["err_rel_d"], r["err_rel_gap"]) <= 1e-6, k
        g = P.solve(prob, time_limit=120.0)
        assert abs(r["pobj"] - g["pobj"]) <= 1e-5 * (1.0 + abs(g["pobj"])), (k, r["pobj"], g["pobj"])
        if "opt" in prob["meta"]:
            assert abs(r["pobj"] - prob["meta"]["opt"]) <= 1e-5 * (1.0 + abs(prob["meta"]["opt"]))
    for r, r2 in zip(out, out2):
        assert np.array_equal(r["x"], r2["x"]) and np.array_equal(r["y"], r2["y"])
        assert r["iters"] == r2["iters"]


def test_fp32_batch_of_uneven_portfolios():
    P = _P()
    probs = workloads.portfolio_batch(count=48, n_lo=50, n_hi=400, seed=31)
    with P.Batch(probs, precision="fp32", time_limit=120.0) as b:
        out = b.solve()
    assert all(r["exit_code"] == 0 for r in out), [r["status"] for r in out]
    for k in (0, 17, 33, 47):
        g = P.solve(probs[k], time_limit=120.0)
        assert abs(out[k]["pobj"] - g["pobj"]) <= 1e-4 * (1.0 + abs(g["pobj"])), k
    assert all(r["finish_s"] > 0 for r in out)
