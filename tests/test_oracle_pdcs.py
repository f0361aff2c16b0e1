"""Pins for the oracle's solver loop, KKT measures, normalized duality gap and
scaling (CPU only).  Each check compares with something independent of the
oracle: a planted optimum, brute-force vertex enumeration, a closed form, a
library optimiser, or an exact piecewise solution."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import minimize

import oracle
import workloads
from oracle import cones as C
from oracle.problem import ConicProblem, compute_scaling


def _solve(prob_dict, **kw):
    return oracle.solve(oracle.problem_from_dict(prob_dict), **kw)


# ------------------------------------------------------------ planted optimum
def test_small_planted_socp_reaches_optimum():
    p = workloads.tiny_conic(seed=11, m_nonneg=16, soc_rows=(4, 5), nb=24, soc_cols=(4, 3),
                             density=0.2)
    res = _solve(p, max_iter=40000)
    assert res["exit_code"] == 0
    opt = p["meta"]["opt"]
    assert abs(res["pobj"] - opt) <= 1e-5 * (1 + abs(opt))
    assert max(res["err_rel_p"], res["err_rel_d"], res["err_rel_gap"]) <= 1e-6


@pytest.mark.slow
def test_tiny_conic_default_size_reaches_planted_optimum():
    p = workloads.tiny_conic()
    res = _solve(p, max_iter=40000)
    assert res["exit_code"] == 0
    opt = p["meta"]["opt"]
    assert abs(res["pobj"] - opt) <= 1e-5 * (1 + abs(opt))


def test_kkt_zero_at_planted_optimum():
    """The planted (x*, y*) has zero residuals and zero gap (unscaled errors)."""
    p = workloads.tiny_conic(seed=3)
    o = oracle.Oracle(oracle.problem_from_dict(p), oracle.Options(use_preconditioner=False))
    from oracle.kkt import unscaled_errors, scaled_errors
    e = unscaled_errors(o.sp, p["meta"]["x_star"], p["meta"]["y_star"])
    assert e["max_rel"] < 1e-12
    e2 = scaled_errors(o.sp, p["meta"]["x_star"], p["meta"]["y_star"])
    assert e2["max_err"] < 1e-12


def test_kkt_errors_hand_computed():
    """2 x 3 example: G = [[1, 0, 2], [0, 1, 1]], rows: zero then nonneg,
    x in box [0, 1]^3, h = (1, 0.5), c = (1, 1, 1)."""
    G = sp.csr_matrix(np.array([[1.0, 0.0, 2.0], [0.0, 1.0, 1.0]]))
    prob = ConicProblem(G, [1.0, 0.5], [1.0, 1.0, 1.0], 3, np.zeros(3), np.ones(3),
                        [(C.ZERO, 1), (C.NONNEG, 1)], [])
    o = oracle.Oracle(prob, oracle.Options(use_preconditioner=False))
    from oracle.kkt import unscaled_errors, scaled_errors
    x = np.array([0.5, 0.0, 0.0])
    y = np.array([2.0, -1.0])
    # Gx - h = (0.5 - 1, 0 - 0.5) = (-0.5, -0.5): zero row residual 0.5, nonneg 0.5
    # lambda = c - G^T y = (1 - 2, 1 + 1, 1 - 4 + 1) = (-1, 2, -2); all bounds finite
    # so Lambda = R and dual residual 0; y_2 = -1 is not in R_+ but the dual
    # residual only measures lambda.  pobj = 0.5, dobj = h^T y + l^T lam+ - u^T lam-
    # = 2 - 0.5 + 0 - (1 + 2) = -1.5.
    e = scaled_errors(o.sp, x, y)
    assert np.isclose(e["abs_p"], np.sqrt(0.5))
    assert np.isclose(e["abs_d"], 0.0)
    assert np.isclose(e["pobj"], 0.5) and np.isclose(e["dobj"], -1.5)
    assert np.isclose(e["abs_gap"], 2.0)
    assert np.isclose(e["rel_p"], np.sqrt(0.5) / 2.5)
    assert np.isclose(e["rel_gap"], 2.0 / 3.0)
    u = unscaled_errors(o.sp, x, y)
    assert np.isclose(u["abs_p"], 0.5)
    # denominators: 1 + max(|h|_inf=1, |Gx|_inf=0.5, |P(Gx-h)|_inf=0) = 2
    assert np.isclose(u["rel_p"], 0.25)
    assert np.isclose(u["rel_gap"], 2.0 / 2.5)


# ------------------------------------------------------- LP vertex enumeration
def _random_lp(seed, n=3, m_ineq=3, m_eq=1):
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(0.5, 2.0, size=n)
    Aeq = rng.standard_normal((m_eq, n))
    Ain = rng.standard_normal((m_ineq, n))
    beq = Aeq @ x0
    bin_ = Ain @ x0 - rng.uniform(0.1, 1.0, size=m_ineq)
    c = rng.standard_normal(n)
    G = np.vstack([Aeq, Ain])
    h = np.concatenate([beq, bin_])
    lo = np.zeros(n)
    hi = np.full(n, 3.0)
    return G, h, c, lo, hi


def _vertex_enumeration(G, h, c, lo, hi, m_eq):
    n = G.shape[1]
    rows = [(G[i], h[i]) for i in range(m_eq, G.shape[0])]
    rows += [(np.eye(n)[j], lo[j]) for j in range(n)]
    rows += [(-np.eye(n)[j], -hi[j]) for j in range(n)]
    best = np.inf
    for subset in itertools.combinations(range(len(rows)), n - m_eq):
        A = np.vstack([G[:m_eq]] + [rows[i][0] for i in subset])
        b = np.concatenate([h[:m_eq], [rows[i][1] for i in subset]])
        if abs(np.linalg.det(A)) < 1e-10:
            continue
        x = np.linalg.solve(A, b)
        if np.all(G[m_eq:] @ x >= h[m_eq:] - 1e-9) and np.all(x >= lo - 1e-9) and np.all(x <= hi + 1e-9):
            best = min(best, c @ x)
    return best


@pytest.mark.parametrize("seed", range(4))
def test_lp_matches_vertex_enumeration(seed):
    G, h, c, lo, hi = _random_lp(seed)
    prob = ConicProblem(sp.csr_matrix(G), h, c, 3, lo, hi, [(C.ZERO, 1), (C.NONNEG, 3)], [])
    res = oracle.solve(prob, max_iter=200000)
    best = _vertex_enumeration(G, h, c, lo, hi, 1)
    assert res["exit_code"] == 0
    assert abs(res["pobj"] - best) <= 1e-5 * (1 + abs(best))


# -------------------------------------------------------- closed-form problems
def test_rsoc_closed_form():
    """min t s.t. (t, 1/2, x) in RSOC, x = a  ->  t* = ||a||^2."""
    a = np.array([0.3, -0.7, 0.5])
    k = len(a)
    n = 1 + k
    rows = [np.eye(n)[1 + i] for i in range(k)]                 # zero rows: x_i - a_i
    G = np.vstack(rows + [np.eye(n)[0], np.zeros(n)] + [np.eye(n)[1 + i] for i in range(k)])
    h = np.concatenate([a, [0.0, -0.5], np.zeros(k)])
    c = np.zeros(n)
    c[0] = 1.0
    prob = ConicProblem(sp.csr_matrix(G), h, c, n, np.full(n, -np.inf), np.full(n, np.inf),
                        [(C.ZERO, k), (C.RSOC, k + 2)], [])
    res = oracle.solve(prob, max_iter=100000)
    assert res["exit_code"] == 0
    assert abs(res["pobj"] - a @ a) <= 1e-5


def test_exp_closed_form():
    """min z s.t. (a, 1, z) in K_exp  ->  z* = e^a (rows: x = a, y = 1 zero rows)."""
    a = 0.4
    G = np.vstack([np.eye(3)[0], np.eye(3)[1], np.eye(3)])
    h = np.array([a, 1.0, 0.0, 0.0, 0.0])
    c = np.array([0.0, 0.0, 1.0])
    prob = ConicProblem(sp.csr_matrix(G), h, c, 3, np.full(3, -np.inf), np.full(3, np.inf),
                        [(C.ZERO, 2), (C.EXP, 3)], [])
    res = oracle.solve(prob, max_iter=100000)
    assert res["exit_code"] == 0
    assert abs(res["pobj"] - np.exp(a)) <= 1e-5 * np.exp(a)


def test_logistic_matches_library_optimiser():
    p = workloads.logistic_l1(N=40, p=4, density=0.5, support=2, seed=5)
    res = _solve(p, max_iter=200000)
    assert res["exit_code"] == 0
    A = workloads.to_scipy(p)
    N, pp, lam = p["meta"]["N"], p["meta"]["p"], p["meta"]["lam"]
    # rows 2p + N + 6 i hold -y_i a_i on the w columns
    M = A[2 * pp + N + 6 * np.arange(N)][:, :pp].toarray()    # = -y_i a_i

    def f(wpm):
        w = wpm[:pp] - wpm[pp:]
        z = M @ w
        return np.sum(np.logaddexp(0.0, z)) + lam * np.sum(wpm)

    def g(wpm):
        w = wpm[:pp] - wpm[pp:]
        z = M @ w
        s = 1.0 / (1.0 + np.exp(-z))
        gw = M.T @ s
        return np.concatenate([gw + lam, -gw + lam])

    r = minimize(f, np.zeros(2 * pp), jac=g, bounds=[(0, None)] * (2 * pp), method="L-BFGS-B",
                 options=dict(ftol=1e-15, gtol=1e-12, maxiter=10000))
    assert abs(res["pobj"] - r.fun) <= 2e-5 * (1 + abs(r.fun))


def test_preconditioning_does_not_change_the_optimum():
    """Algorithm 2: solving the rescaled problem and unscaling gives the same
    optimal value as solving the original problem."""
    p = workloads.tiny_conic(seed=21, m_nonneg=10, soc_rows=(4,), nb=12, soc_cols=(3,), density=0.3)
    a = _solve(p, max_iter=50000)
    b = _solve(p, max_iter=50000, use_preconditioner=False)
    assert a["exit_code"] == 0 and b["exit_code"] == 0
    assert abs(a["pobj"] - b["pobj"]) <= 1e-5 * (1 + abs(a["pobj"]))


# --------------------------------------------------- normalized duality gap
def _free_problem(rng, m, n, lo=None, hi=None):
    G = sp.csr_matrix(rng.standard_normal((m, n)))
    lo = np.full(n, -np.inf) if lo is None else lo
    hi = np.full(n, np.inf) if hi is None else hi
    return ConicProblem(G, rng.standard_normal(m), rng.standard_normal(n), n, lo, hi,
                        [(C.ZERO, m)], [])


def test_normalized_gap_closed_form_whole_space():
    """X x Y = whole space: z(t) = z + t N^{-1} b, so rho^N(r; z) equals
    sqrt(tau ||b1||^2 + sigma ||b2||^2) for every r > 0."""
    rng = np.random.default_rng(0)
    prob = _free_problem(rng, 5, 7)
    o = oracle.Oracle(prob, oracle.Options(use_preconditioner=False, bisect_rel_tol=1e-6))
    for _ in range(10):
        x = rng.standard_normal(7)
        y = rng.standard_normal(5)
        tau, sigma = rng.uniform(0.1, 2.0, size=2)
        r = rng.uniform(0.01, 10.0)
        b1 = o.sp.GT @ y - o.sp.c
        b2 = o.sp.h - o.sp.G @ x
        exact = np.sqrt(tau * b1 @ b1 + sigma * b2 @ b2)
        assert abs(o.normalized_gap(x, y, r, tau, sigma) - exact) <= 3e-6 * exact


def _box_gap_exact(x, y, b1, b2, lo, hi, r, tau, sigma):
    """Exact rho^N for X = box, Y = whole space, z inside the box: the distance
    ||z(t) - z||_N^2 is piecewise quadratic in t with breakpoints where a
    coordinate reaches its bound; solve in the right piece."""
    v = tau * b1
    with np.errstate(divide="ignore", invalid="ignore"):
        tb = np.where(v > 0, (hi - x) / v, np.where(v < 0, (lo - x) / v, np.inf))
    order = np.argsort(tb)
    sat = np.zeros(len(x), bool)
    t_prev = 0.0
    for j in list(order) + [None]:
        t_next = tb[j] if j is not None else np.inf
        a = np.sum(tau * b1[~sat] ** 2) + sigma * (b2 @ b2)          # t^2 coefficient
        const = np.sum(((np.where(v > 0, hi, lo) - x)[sat]) ** 2) / tau
        # dist^2 = a t^2 + const on [t_prev, t_next]
        if a * t_next ** 2 + const >= r * r:
            t = np.sqrt((r * r - const) / a)
            xt = np.clip(x + t * v, lo, hi)
            return (b1 @ (xt - x) + b2 @ (t * sigma * b2)) / r
        sat[j] = True
        t_prev = t_next
    raise AssertionError("radius not reached")


def test_normalized_gap_box_matches_exact_piecewise_solution():
    rng = np.random.default_rng(1)
    n, m = 8, 4
    lo = -rng.uniform(0.1, 1.0, size=n)
    hi = rng.uniform(0.1, 1.0, size=n)
    prob = _free_problem(rng, m, n, lo, hi)
    # the routine converged tightly, and at the solver's default tolerance
    # (1e-3 of t_right, reading c9), which leaves the value within ~1e-3
    o = oracle.Oracle(prob, oracle.Options(use_preconditioner=False, bisect_rel_tol=1e-6))
    od = oracle.Oracle(prob, oracle.Options(use_preconditioner=False))
    assert od.opts.bisect_rel_tol == 1e-3
    for _ in range(20):
        x = rng.uniform(lo, hi)
        y = rng.standard_normal(m)
        tau, sigma = rng.uniform(0.1, 2.0, size=2)
        r = rng.uniform(0.05, 3.0)
        b1 = o.sp.GT @ y - o.sp.c
        b2 = o.sp.h - o.sp.G @ x
        exact = _box_gap_exact(x, y, b1, b2, lo, hi, r, tau, sigma)
        got = o.normalized_gap(x, y, r, tau, sigma)
        assert abs(got - exact) <= 1e-5 * abs(exact) + 1e-12
        got_d = od.normalized_gap(x, y, r, tau, sigma)
        assert abs(got_d - exact) <= 2e-3 * abs(exact) + 1e-12


def test_gap_pin_detects_a_planted_mistake(monkeypatch):
    """Swapping tau and sigma inside the N-norm must break the closed form."""
    rng = np.random.default_rng(2)
    prob = _free_problem(rng, 5, 7)
    o = oracle.Oracle(prob, oracle.Options(use_preconditioner=False))
    good = o.normalized_gap
    monkeypatch.setattr(o, "normalized_gap", lambda x, y, r, tau, sigma: good(x, y, r, sigma, tau))
    x, y = rng.standard_normal(7), rng.standard_normal(5)
    tau, sigma, r = 0.3, 1.7, 1.0
    b1 = o.sp.GT @ y - o.sp.c
    b2 = o.sp.h - o.sp.G @ x
    exact = np.sqrt(tau * b1 @ b1 + sigma * b2 @ b2)
    assert abs(o.normalized_gap(x, y, r, tau, sigma) - exact) > 1e-3 * exact


# ----------------------------------------------------------------- scaling
def test_ruiz_equilibrates_infinity_norms():
    rng = np.random.default_rng(4)
    G = sp.random(60, 40, density=0.2, random_state=5, data_rvs=lambda k: rng.standard_normal(k) * 10 ** rng.uniform(-3, 3, k))
    G = sp.csr_matrix(G)
    d1, d2 = compute_scaling(G, ruiz_iters=25, pc_alpha=-1.0)
    S = abs(sp.diags(d1) @ G @ sp.diags(d2)).tocsr()
    rn = np.asarray(S.max(axis=1).todense()).ravel()
    cn = np.asarray(S.max(axis=0).todense()).ravel()
    assert np.all(np.abs(rn[rn > 0] - 1) < 1e-3)
    assert np.all(np.abs(cn[cn > 0] - 1) < 1e-3)


def test_pock_chambolle_alpha1_unit_row_and_column_sums():
    """After one PC pass (no Ruiz) on a matrix whose rows and columns all have
    the same 1-norm s, every entry is divided by s: rows and columns sum to 1."""
    G = sp.csr_matrix(np.array([[1.0, -2.0, 0.0], [0.0, 1.0, -2.0], [-2.0, 0.0, 1.0]]))
    d1, d2 = compute_scaling(G, ruiz_iters=0, pc_alpha=1.0)
    S = abs(sp.diags(d1) @ G @ sp.diags(d2)).toarray()
    assert np.allclose(S.sum(axis=0), 1.0) and np.allclose(S.sum(axis=1), 1.0)


# --------------------------------------------------------------- controller
def test_trace_records_restart_at_first_check_and_monotone_counters():
    p = workloads.tiny_conic(seed=8, m_nonneg=10, soc_rows=(4,), nb=12, soc_cols=(3,), density=0.3)
    tr = []
    _solve(p, max_iter=300, trace=tr, check_freq=32)
    assert tr[31]["check"] == 1 and tr[31]["restart"] == 1       # reading c8
    assert all(t["check"] == (1 if t["iter"] % 32 == 0 else 0) for t in tr)
    assert all(b["kbar"] >= a["kbar"] + 1 for a, b in zip(tr, tr[1:]))
    assert all(0.0 <= t["beta"] <= 1.0 for t in tr)


# ------------------------------------------- option modes (readings c21, c22)
@pytest.mark.parametrize("opts", [
    dict(use_adaptive_step_size_weight=False),
    dict(use_kkt_restart=True, kkt_restart_freq=48),
    dict(use_duality_gap_restart=False, use_kkt_restart=True, kkt_restart_freq=64),
    dict(use_duality_gap_restart=False),
])
def test_option_modes_reach_planted_optimum(opts):
    p = workloads.tiny_conic(seed=11, m_nonneg=16, soc_rows=(4, 5), nb=24, soc_cols=(4, 3),
                             density=0.2)
    tr = []
    res = _solve(p, max_iter=60000, trace=tr, **opts)
    assert res["exit_code"] == 0
    opt = p["meta"]["opt"]
    assert abs(res["pobj"] - opt) <= 1e-5 * (1 + abs(opt))
    checks = [r for r in tr if r["check"]]
    if not opts.get("use_adaptive_step_size_weight", True):
        assert res["attempts"] == res["iters"]          # every attempt accepted
        assert len({r["eta"] for r in tr}) == 1
    if opts.get("use_kkt_restart") and not opts.get("use_duality_gap_restart", True):
        assert checks and all(r["fallback"] == 1 for r in checks)   # KKT_omega throughout
    if opts.get("use_kkt_restart") and opts.get("use_duality_gap_restart", True):
        kkt_only = [r for r in checks if r["iter"] % 64 != 0]
        assert kkt_only and all(r["fallback"] == 1 for r in kkt_only)


def test_continuing_from_a_recorded_state_reproduces_the_run():
    """init_state restarts the loop from a recorded state: the continuation
    must equal the uninterrupted run bit for bit (same trace, same iterate)."""
    p = workloads.tiny_conic(seed=4, m_nonneg=10, soc_rows=(4,), nb=20, soc_cols=(3,), density=0.3)
    prob = oracle.problem_from_dict(p)
    states = {70: None, 150: None}
    tr = []
    oracle.solve(prob, trace=tr, states=states, max_iter=150, check_freq=16)
    tr2 = []
    states2 = {150: None}
    oracle.solve(prob, trace=tr2, states=states2, max_iter=150, check_freq=16,
                 init_state=states[70])
    # (the infeasibility record needs the previous check's candidate, which a
    # continuation does not have)
    strip = lambda rows: [{k: v for k, v in r.items() if k != "infeas"} for r in rows]  # noqa: E731
    assert strip(tr2) == strip(tr[70:])
    assert np.array_equal(states2[150]["x"], states[150]["x"])
    assert np.array_equal(states2[150]["y"], states[150]["y"])
