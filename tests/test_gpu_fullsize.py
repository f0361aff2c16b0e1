"""Parity at the full sizes of the benchmark workloads, in the launch
configuration the benchmark times (FP64, graph mode, restart checks every 64
accepted iterations).

* Portfolio SOCP, n = 200,000 (the benchmark instance): the oracle's complete
  state after one iteration is loaded into the GPU solver, one iteration runs,
  and the whole state must equal the oracle's after two iterations within
  1e-9 (the grid-wide SOC projection of the 200,202-dimensional block, both
  products, the step test, the reflection and the Halpern update at full size).
* L1-logistic regression, 100,000 samples x 2,000 features (200,000 exponential
  cones): one oracle iteration takes about a minute here, so the check is on
  sampled outputs: after 5 GPU iterations the accepted PDHG point of the next
  iteration is recomputed on the CPU from the GPU's state with the oracle's own
  projections, for every primal coordinate, every nonnegative row and 2,000
  random exponential cones."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import workloads
from oracle import cones as oc
from test_gpu_parity import _compare_state, _to_gpu_state

pytestmark = pytest.mark.gpu


def _P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_15504_b300 as P
    return P


def test_portfolio_full_size_one_step_parity():
    P = _P()
    prob = workloads.portfolio()  # n = 200,000, k = 200, 1,000 limits (the benchmark instance)
    states = {1: None, 2: None}
    oracle.solve(oracle.problem_from_dict(prob), max_iter=2, check_freq=64, states=states)
    with P.Solver(prob, check_freq=64, time_limit=120.0) as s:
        s.set_state(_to_gpu_state(states[1]))
        s.resume(max_iter=2)
        _compare_state(s.get_state(), states[2], 1)


def test_logistic_full_size_sampled_step():
    P = _P()
    prob = workloads.logistic_l1()  # 100,000 x 2,000, 200,000 exponential cones
    spb = oracle.ScaledProblem(oracle.problem_from_dict(prob))
    with P.Solver(prob, check_freq=64, max_iter=5, time_limit=300.0) as s:
        s.solve()
        st = s.get_state()
        s.resume(max_iter=6)
        st1 = s.get_state()
        assert st1["iter"] == 6
        xh, yh = s.get_iterate(2)  # the accepted PDHG point of iteration 6
    eta, omega = st1["eta_last"], st1["omega"]
    tau, sigma = eta / omega, eta * omega
    x, y = st["x"], st["y"]
    G = sp.csr_matrix(spb.G)
    xh_ref = x - tau * (spb.c - G.T @ y)
    xh_ref[:spb.nb] = np.clip(xh_ref[:spb.nb], spb.lo, spb.hi)
    assert np.linalg.norm(xh - xh_ref) <= 1e-9 * max(1.0, np.linalg.norm(xh_ref))
    v = y + sigma * (spb.h - G @ (2.0 * xh_ref - x))
    offs = np.concatenate([[0], np.cumsum([d for _, d in spb.row_cones])])
    nonneg = np.concatenate([np.arange(offs[b], offs[b + 1]) for b, (t, _) in enumerate(spb.row_cones)
                             if t == oc.NONNEG])
    assert np.allclose(yh[nonneg], np.maximum(v[nonneg], 0.0), rtol=1e-9, atol=1e-9 * np.abs(v).max())
    exp_blocks = [(offs[b], t) for b, (t, _) in enumerate(spb.row_cones) if t in (oc.EXP, oc.DUAL_EXP)]
    rng = np.random.default_rng(0)
    pick = rng.choice(len(exp_blocks), size=2000, replace=False)
    idx = np.concatenate([np.arange(exp_blocks[k][0], exp_blocks[k][0] + 3) for k in pick])
    cones = [(exp_blocks[k][1], 3) for k in pick]
    want = oc.proj_cone_product(v[idx], cones, 1.0 / spb.d1[idx], dual=True)
    err = np.abs(yh[idx] - want) / (1.0 + np.abs(want))
    assert err.max() <= 1e-9, err.max()
