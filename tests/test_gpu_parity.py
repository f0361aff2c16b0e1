"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

The method's trajectory is chaotic under rounding: the oracle run against itself
with h perturbed by 1e-15 (relative) drifts to ~1e-12 after 30 iterations, 1e-9
after 63, 1e-5 after 128 and 2e-2 after 200 on the tiny conic program (the
adaptive step size feeds the iterates back into eta).  So no two
implementations that round differently agree to 1e-9 over 200 free-running
iterations.  The FP64 bar is therefore checked as:
  * one-step parity for every iteration k < 200: the oracle's complete state
    after k iterations is loaded into the GPU solver (pdcs_set_state), one
    iteration is run (pdcs_resume), and the whole state (iterates, anchor,
    average sums, counters, step size, primal weight, restart references)
    must equal the oracle's state after k + 1 iterations within 1e-9 relative,
    with identical decisions (accept/reject count, check, candidate, restart);
  * free-running parity of the first 40 iterations within 1e-9;
  * full solves reaching 1e-6 relative KKT error with the oracle's objective."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-9
FREE = (1, 2, 10, 20, 40)
TRACE_KEYS = ("iter", "kbar", "period", "eta", "eta_hat", "beta", "omega", "max_err", "check",
              "cand_avg", "restart", "rho_c")


def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_15504_b300 as P
    return P


def _rel(a, b):
    return np.linalg.norm(a - b) / max(1.0, np.linalg.norm(b))


def _close(a, b, tol=TOL):
    return abs(a - b) <= tol * max(1.0, abs(b))


def _compare_row(grow, o, i):
    g = dict(zip(TRACE_KEYS, grow))
    for key in ("iter", "kbar", "period", "check", "cand_avg", "restart"):
        assert int(g[key]) == int(o[key]), (i, key, g[key], o[key])
    for key in ("eta", "eta_hat", "beta", "omega", "max_err"):
        assert _close(g[key], o[key]), (i, key, g[key], o[key])
    if o["check"]:
        assert _close(g["rho_c"], o["rho_c"], 1e-8), (i, g["rho_c"], o["rho_c"])


def _to_gpu_state(o):
    return dict(iter=o["iter"], kbar=o["kbar"], k=o["k"], period=o["period"],
                restarts=o["restarts"], eta_hat=o["eta_hat"], eta_last=o["eta"],
                omega=o["omega"], wsum=o["wsum"], has_ref=int(o["has_ref"]),
                has_prev=int(o["has_prev"]), ref_rho=o["ref"][0], ref_abs_p=o["ref"][1],
                ref_abs_d=o["ref"][2], ref_abs_gap=o["ref"][3], prev_rho=o["prev"][0],
                prev_abs_p=o["prev"][1], prev_abs_d=o["prev"][2], prev_abs_gap=o["prev"][3],
                x=o["x"], y=o["y"], x0=o["x0"], y0=o["y0"], xs=o["xs"], ys=o["ys"])


def _compare_state(g, o, k):
    for key in ("x", "y", "x0", "y0", "xs", "ys"):
        assert _rel(g[key], o[key]) <= TOL, (k, key, _rel(g[key], o[key]))
    for key in ("iter", "kbar", "k", "period", "restarts"):
        assert int(g[key]) == int(o[key]), (k, key, g[key], o[key])
    assert int(g["has_ref"]) == int(o["has_ref"]) and int(g["has_prev"]) == int(o["has_prev"]), k
    assert _close(g["eta_hat"], o["eta_hat"]), (k, g["eta_hat"], o["eta_hat"])
    assert _close(g["eta_last"], o["eta"]), (k, g["eta_last"], o["eta"])
    assert _close(g["omega"], o["omega"]), (k, g["omega"], o["omega"])
    assert _close(g["wsum"], o["wsum"]), (k, g["wsum"], o["wsum"])
    if o["has_ref"]:
        assert _close(g["ref_rho"], o["ref"][0], 1e-8), (k, g["ref_rho"], o["ref"][0])
    if o["has_prev"]:
        assert _close(g["prev_rho"], o["prev"][0], 1e-8), (k, g["prev_rho"], o["prev"][0])


def _parity(prob, iters=200, check_freq=64, **kw):
    P = _gpu()
    states = {k: None for k in range(iters + 1)}
    otr = []
    oracle.solve(oracle.problem_from_dict(prob), trace=otr, states=states, max_iter=iters,
                 check_freq=check_freq, **kw)
    # one-step parity from every oracle state
    with P.Solver(prob, trace_capacity=iters, check_freq=check_freq, time_limit=60.0, **kw) as s:
        for k in range(iters):
            s.set_state(_to_gpu_state(states[k]))
            s.resume(max_iter=k + 1)
            _compare_state(s.get_state(), states[k + 1], k)
            _compare_row(s.trace()[k], otr[k], k)
    # free-running parity of the first iterations
    for k in FREE:
        with P.Solver(prob, trace_capacity=k, check_freq=check_freq, max_iter=k, time_limit=60.0,
                      **kw) as s:
            s.solve()
            g = s.get_state()
            assert _rel(g["x"], states[k]["x"]) <= TOL, ("free x", k, _rel(g["x"], states[k]["x"]))
            assert _rel(g["y"], states[k]["y"]) <= TOL, ("free y", k, _rel(g["y"], states[k]["y"]))
            tr = s.trace()
            for i in range(k):
                _compare_row(tr[i], otr[i], i)


def test_tiny_conic_first_200_iterations():
    _parity(workloads.tiny_conic())


def test_small_portfolio_first_200_iterations():
    _parity(workloads.portfolio(n=300, k=15, n_limits=4, limit_density=0.02, seed=7))


def test_small_logistic_first_200_iterations():
    _parity(workloads.logistic_l1(N=200, p=12, density=0.2, support=4, seed=9))


def test_halpern_method_first_200_iterations():
    _parity(workloads.tiny_conic(seed=5, m_nonneg=30, soc_rows=(6, 6), nb=60, soc_cols=(5, 4)),
            method="halpern")


def test_no_preconditioner_first_200_iterations():
    _parity(workloads.tiny_conic(seed=6, m_nonneg=30, soc_rows=(6, 6), nb=60, soc_cols=(5, 4)),
            use_preconditioner=False)


def test_large_soc_block_grid_tier():
    """An SOC block of dimension n + k + 2 > 8192 goes through the cooperative
    grid-wide projection kernel."""
    prob = workloads.portfolio(n=9000, k=30, n_limits=5, limit_density=0.002, seed=11)
    assert max(d for _, d in prob["row_cones"]) > 8192
    _parity(prob, iters=70, check_freq=32)


def test_eager_mode_matches_graph_mode():
    """Host-launched kernels (for profilers) give exactly the graph results."""
    P = _gpu()
    prob = workloads.tiny_conic(seed=4)
    out = []
    for eager in (0, 1):
        with P.Solver(prob, max_iter=150, check_freq=32, eager=eager, time_limit=60.0) as s:
            s.solve()
            out.append(s.get_state())
    for key in ("x", "y", "x0", "y0", "xs", "ys"):
        assert np.array_equal(out[0][key], out[1][key]), key
    assert out[0]["kbar"] == out[1]["kbar"] and out[0]["restarts"] == out[1]["restarts"]


def _full(prob, **kw):
    P = _gpu()
    g = P.solve(prob, max_iter=100000, time_limit=120.0, **kw)
    o = oracle.solve(oracle.problem_from_dict(prob), max_iter=100000, **kw)
    return g, o


def test_tiny_conic_full_solve():
    prob = workloads.tiny_conic()
    g, o = _full(prob)
    assert g["exit_code"] == 0
    assert max(g["err_rel_p"], g["err_rel_d"], g["err_rel_gap"]) <= 1e-6
    opt = prob["meta"]["opt"]
    assert abs(g["pobj"] - opt) <= 1e-5 * (1 + abs(opt))
    assert abs(g["pobj"] - o["pobj"]) <= 1e-5 * (1 + abs(o["pobj"]))


def test_small_portfolio_full_solve():
    prob = workloads.portfolio(n=300, k=15, n_limits=4, limit_density=0.02, seed=7)
    g, o = _full(prob)
    assert g["exit_code"] == 0 and o["exit_code"] == 0
    assert max(g["err_rel_p"], g["err_rel_d"], g["err_rel_gap"]) <= 1e-6
    assert abs(g["pobj"] - o["pobj"]) <= 1e-5 * (1 + abs(o["pobj"]))


def test_small_logistic_full_solve():
    prob = workloads.logistic_l1(N=50, p=6, density=0.3, support=2, seed=3)
    g, o = _full(prob)
    assert g["exit_code"] == 0 and o["exit_code"] == 0
    assert abs(g["pobj"] - o["pobj"]) <= 1e-5 * (1 + abs(o["pobj"]))


def test_rotated_soc_column_block():
    """RSOC as a column block: min t s.t. (t, q, x) in RSOC, q = 1/2, x = a;
    optimum ||a||^2."""
    a = np.array([0.3, -0.7, 0.5])
    k = len(a)
    n = k + 2
    G = np.zeros((1 + k, n))
    G[0, 1] = 1.0
    for i in range(k):
        G[1 + i, 2 + i] = 1.0
    Gs = sp.csr_matrix(G)
    c = np.zeros(n)
    c[0] = 1.0
    prob = dict(m=1 + k, n=n, row_ptr=Gs.indptr.astype(np.int64), col_idx=Gs.indices.astype(np.int32),
                val=Gs.data, h=np.concatenate([[0.5], a]), c=c, nb=0, lo=np.zeros(0), hi=np.zeros(0),
                row_cones=[(0, 1 + k)], col_cones=[(3, n)], meta={})
    P = _gpu()
    g = P.solve(prob, max_iter=200000, time_limit=120.0)
    assert g["exit_code"] == 0
    assert abs(g["pobj"] - a @ a) <= 1e-5
    assert np.allclose(g["x"][2:], a, atol=1e-5)


def test_fp32_bulk_mode_reaches_tolerance_on_tiny_conic():
    prob = workloads.tiny_conic()
    P = _gpu()
    g = P.solve(prob, max_iter=200000, precision="fp32", time_limit=120.0)
    opt = prob["meta"]["opt"]
    assert g["exit_code"] == 0
    assert abs(g["pobj"] - opt) <= 1e-4 * (1 + abs(opt))


def test_fp32_bulk_mode_long_rows_dual_in_product():
    """A portfolio with 16+ nonzeros per row (the dual step runs in the
    epilogue of G xhat) in FP32 bulk: it reaches 1e-4 and its objective
    agrees with the FP64 solve's."""
    prob = workloads.portfolio(n=2000, k=40, n_limits=10, limit_density=0.01, seed=13)
    assert len(prob["val"]) >= 16 * prob["m"]
    P = _gpu()
    g32 = P.solve(prob, max_iter=200000, precision="fp32", rel_tol=1e-4, time_limit=120.0)
    g64 = P.solve(prob, max_iter=200000, rel_tol=1e-6, time_limit=120.0)
    assert g32["exit_code"] == 0 and g64["exit_code"] == 0
    assert abs(g32["pobj"] - g64["pobj"]) <= 1e-3 * (1 + abs(g64["pobj"]))


def test_problem_without_constraints():
    """m = 0: min c^T x over a box."""
    P = _gpu()
    n = 5
    prob = dict(m=0, n=n, row_ptr=np.zeros(1, np.int64), col_idx=np.zeros(0, np.int32),
                val=np.zeros(0), h=np.zeros(0), c=np.array([1.0, -1.0, 2.0, -3.0, 0.5]), nb=n,
                lo=np.zeros(n), hi=np.ones(n), row_cones=[], col_cones=[], meta={})
    g = P.solve(prob, max_iter=10000, time_limit=60.0)
    assert g["exit_code"] == 0
    assert abs(g["pobj"] - (-4.0)) <= 1e-5


def test_invalid_inputs_return_errors():
    P = _gpu()
    prob = workloads.tiny_conic(seed=2, m_nonneg=10, soc_rows=(4,), nb=12, soc_cols=(3,))
    bad = dict(prob)
    bad["col_idx"] = prob["col_idx"].copy()
    bad["col_idx"][0] = prob["n"] + 5
    with pytest.raises(P.PdcsError, match="column index"):
        P.Solver(bad)
    bad = dict(prob)
    bad["h"] = prob["h"].copy()
    bad["h"][0] = np.nan
    with pytest.raises(P.PdcsError, match="non-finite"):
        P.Solver(bad)
    bad = dict(prob)
    bad["lo"] = prob["lo"].copy()
    bad["lo"][0] = 5.0
    bad["hi"] = np.full(prob["nb"], 1.0)
    with pytest.raises(P.PdcsError, match="lb <= ub"):
        P.Solver(bad)
