"""Pins for the oracle's controller scalars (CPU only).

Each function of the restart / step-size controller is checked against values
derived by hand from the paper's formulas (the derivation is written beside
each row), and each table is run once more against a copy of the function with
one plausible slip planted in it (a wrong exponent, constant, sign or
comparison), which the table must reject.  A last group checks that the solver
loop really goes through these functions: replacing one of them changes the
trace."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import oracle.pdcs as OP
import workloads
from oracle import cones as C
from oracle.kkt import kkt_omega
from oracle.problem import ConicProblem


def _table_ok(fn, rows, tol=1e-13):
    """True if fn(*args) matches every expected value of the table."""
    for args, want in rows:
        got = fn(*args)
        if isinstance(want, tuple):
            if tuple(bool(g) for g in got) != want:
                return False
        elif isinstance(want, bool):
            if bool(got) != want:
                return False
        elif math.isinf(want):
            if not (math.isinf(got) and got > 0):
                return False
        elif abs(got - want) > tol * max(1.0, abs(want)):
            return False
    return True


# ---------------------------------------------------------- Function 1
# eta_bar = (1/2)(omega ||dx||^2 + ||dy||^2 / omega) / |dy^T G dx|   (eq. adaptive_step_size)
STEP_BOUND = [
    ((3.0, 8.0, -5.0, 2.0), 1.0),        # (1/2)(2*3 + 8/2) / 5 = 1
    ((1.0, 1.0, 0.25, 1.0), 4.0),        # (1/2)(1 + 1) / 0.25 = 4
    ((2.0, 0.5, 0.0, 4.0), math.inf),    # dy^T G dx = 0 -> +inf (reading c4)
]

# eta' = min((1 - (kbar+1)^-0.3) eta_bar, (1 + (kbar+1)^-0.6) eta), kbar already
# counts the attempt (reading c3).  With kbar + 1 = 1024 = 2^10: 2^-3 and 2^-6;
# with kbar + 1 = 32 = 2^5: 2^-1.5 and 2^-3.
NEXT_STEP = [
    ((0.5, 1.0, 1023), 0.5 * (1 + 2.0 ** -6)),          # min(0.875, 0.5078125)
    ((1.0, 0.5, 1023), 0.5 * (1 - 2.0 ** -3)),          # min(0.4375, 1.015625)
    ((1.0, 1.0, 31), 1.0 - 2.0 ** -1.5),                # min(0.6464466, 1.125)
    ((2.0, math.inf, 1023), 2.0 * (1 + 2.0 ** -6)),     # eta_bar = inf: growth cap
    ((3.0, 100.0, 3), 3.0 * (1 + 2.0 ** -1.2)),         # kbar + 1 = 4: 2^-0.6, 2^-1.2
]


def test_step_bound_table():
    assert _table_ok(OP.step_bound, STEP_BOUND)


def test_step_bound_rejects_planted_mistakes():
    def no_half(dx2, dy2, inter, omega):
        inter = abs(inter)
        return (omega * dx2 + dy2 / omega) / inter if inter > 0 else math.inf

    def omega_swapped(dx2, dy2, inter, omega):
        return OP.step_bound(dx2, dy2, inter, 1.0 / omega)

    assert not _table_ok(no_half, STEP_BOUND)
    assert not _table_ok(omega_swapped, STEP_BOUND)


def test_next_step_size_table():
    assert _table_ok(OP.next_step_size, NEXT_STEP)


def test_next_step_size_rejects_planted_mistakes():
    def exp_swapped(eta, eta_bar, kbar):
        return min((1.0 - (kbar + 1) ** -0.6) * eta_bar, (1.0 + (kbar + 1) ** -0.3) * eta)

    def kbar_not_shifted(eta, eta_bar, kbar):
        return min((1.0 - kbar ** -0.3) * eta_bar, (1.0 + kbar ** -0.6) * eta) if kbar else 0.0

    def max_not_min(eta, eta_bar, kbar):
        return max((1.0 - (kbar + 1) ** -0.3) * eta_bar, (1.0 + (kbar + 1) ** -0.6) * eta)

    for bad in (exp_swapped, kbar_not_shifted, max_not_min):
        assert not _table_ok(bad, NEXT_STEP), bad.__name__


# ------------------------------------------------- eq. adaptive_reflection
# beta = Proj_[0,1](-0.1 log10(maxErr) + 0.2)
REFLECTION = [
    ((1e-12,), 1.0),    # 1.2 + 0.2 = 1.4 -> clamped to 1
    ((1e-8,), 1.0),     # 0.8 + 0.2 = 1.0 exactly
    ((1e-6,), 0.8),     # 0.6 + 0.2
    ((1e-2,), 0.4),     # 0.2 + 0.2
    ((1.0,), 0.2),      # 0 + 0.2
    ((10.0,), 0.1),     # -0.1 + 0.2
    ((1e3,), 0.0),      # -0.3 + 0.2 = -0.1 -> clamped to 0
    ((0.0,), 1.0),      # log10(0) = -inf -> +inf -> 1
]


def test_reflection_table():
    assert _table_ok(OP.reflection, REFLECTION, tol=1e-14)


def test_reflection_rejects_planted_mistakes():
    def natural_log(e):
        return 1.0 if e <= 0 else float(min(1.0, max(0.0, -0.1 * np.log(e) + 0.2)))

    def wrong_offset(e):
        return 1.0 if e <= 0 else float(min(1.0, max(0.0, -0.1 * np.log10(e) + 0.1)))

    def no_upper_clamp(e):
        return 1.0 if e <= 0 else float(max(0.0, -0.1 * np.log10(e) + 0.2))

    def no_lower_clamp(e):
        return 1.0 if e <= 0 else float(min(1.0, -0.1 * np.log10(e) + 0.2))

    for bad in (natural_log, wrong_offset, no_upper_clamp, no_lower_clamp):
        assert not _table_ok(bad, REFLECTION), bad.__name__


# ------------------------------------------------- reflected Halpern step
# z' = (k+1)/(k+2) ((1+beta) zhat - beta z) + z0 / (k+2)
HALPERN = [
    ((2, 0.5, 4.0, 2.0, 8.0), 5.75),      # (3/4)(6 - 1) + 8/4
    ((0, 0.0, 1.0, 5.0, 3.0), 2.0),       # (1/2)(1) + 3/2
    ((1, 1.0, 2.0, 1.0, -3.0), 1.0),      # (2/3)(4 - 1) - 3/3
]


def test_halpern_step_table():
    assert _table_ok(OP.halpern_step, HALPERN)


def test_halpern_step_rejects_planted_mistakes():
    def anchor_weight_k1(k, beta, zh, z, z0):
        a = (k + 1.0) / (k + 2.0)
        return a * ((1.0 + beta) * zh - beta * z) + z0 / (k + 1.0)

    def reflect_sign(k, beta, zh, z, z0):
        a = (k + 1.0) / (k + 2.0)
        return a * ((1.0 + beta) * zh + beta * z) + z0 / (k + 2.0)

    for bad in (anchor_weight_k1, reflect_sign):
        assert not _table_ok(bad, HALPERN), bad.__name__


# --------------------------------------------------- restart conditions
# (sufficient: val <= 0.4 ref, necessary: val <= 0.8 ref and val > prev,
#  long loop: k >= 0.223 kbar); the first period has no reference (reading c8)
RESTART = [
    ((0.39, 1.0, None, 1, 1000), (True, False, False)),
    ((0.41, 1.0, None, 1, 1000), (False, False, False)),
    ((0.70, 1.0, 0.60, 1, 1000), (False, True, False)),   # no local progress
    ((0.70, 1.0, 0.75, 1, 1000), (False, False, False)),  # still improving
    ((0.85, 1.0, 0.60, 1, 1000), (False, False, False)),  # above 0.8 ref
    ((0.50, 1.0, None, 224, 1000), (False, False, True)),  # 224 >= 223
    ((0.50, 1.0, None, 222, 1000), (False, False, False)),
    ((0.01, None, None, 222, 1000), (False, False, False)),  # first period: only cond. 3
    ((0.01, None, None, 300, 1000), (False, False, True)),
]


def test_restart_conditions_table():
    assert _table_ok(OP.restart_conditions, RESTART)


def test_restart_conditions_reject_planted_mistakes():
    def swapped_thresholds(val, ref, prev, k, kbar):
        c3 = k >= 0.223 * kbar
        if ref is None:
            return False, False, c3
        return val <= 0.8 * ref, prev is not None and val <= 0.4 * ref and val > prev, c3

    def progress_flipped(val, ref, prev, k, kbar):
        c3 = k >= 0.223 * kbar
        if ref is None:
            return False, False, c3
        return val <= 0.4 * ref, prev is not None and val <= 0.8 * ref and val < prev, c3

    def artificial_on_k_only(val, ref, prev, k, kbar):
        c1, c2, _ = OP.restart_conditions(val, ref, prev, k, kbar)
        return c1, c2, k >= 0.223 * 1000.0 * 0.99

    for bad in (swapped_thresholds, progress_flipped, artificial_on_k_only):
        assert not _table_ok(bad, RESTART), bad.__name__


# ------------------------------------------------------------ Sec. 2.5
INIT_WEIGHT = [
    ((3.0, 4.0), 0.75),
    ((1e-11, 4.0), 1.0),    # ||c|| below the 1e-10 guard
    ((2.0, 0.0), 1.0),
]

# omega' = exp(0.5 log(dy/dx) + 0.5 log(omega)) = sqrt(omega dy / dx); reset
# to omega0 outside [1e-5, 1e5]; unchanged when dx or dy <= 1e-10
WEIGHT_UPDATE = [
    ((1.0, 4.0, 1.0, 7.0), 2.0),
    ((4.0, 1.0, 4.0, 7.0), 1.0),
    ((2.0, 8.0, 9.0, 7.0), 6.0),            # sqrt(9 * 4)
    ((1e-11, 1.0, 3.0, 7.0), 3.0),          # guard on dx
    ((1.0, 1e-11, 3.0, 7.0), 3.0),          # guard on dy
    ((1.0, 1e10, 10.0, 7.0), 7.0),          # sqrt(1e11) > 1e5 -> omega0
    ((1e3, 1e-9, 1e-3, 7.0), 7.0),          # sqrt(1e-15) < 1e-5 -> omega0
    ((1e-11, 1.0, 2e5, 7.0), 7.0),          # guard keeps 2e5, out of range -> omega0
    ((1.0, 1.0, 2e5, 7.0), math.sqrt(2e5)),  # sqrt(2e5 * 1) = 447.2: kept
]


def test_primal_weight_tables():
    assert _table_ok(OP.initialize_primal_weight, INIT_WEIGHT)
    assert _table_ok(OP.primal_weight_update, WEIGHT_UPDATE, tol=1e-12)


def test_primal_weight_rejects_planted_mistakes():
    def inverted_ratio(c, h):
        return h / c if (c > 1e-10 and h > 1e-10) else 1.0

    def theta_one(dx, dy, omega, omega0):
        if dx > 1e-10 and dy > 1e-10:
            omega = dy / dx
        return omega0 if (omega > 1e5 or omega < 1e-5) else omega

    def ratio_flipped(dx, dy, omega, omega0):
        return OP.primal_weight_update(dy, dx, omega, omega0)

    def no_reset(dx, dy, omega, omega0):
        if dx > 1e-10 and dy > 1e-10:
            omega = float(np.exp(0.5 * np.log(dy / dx) + 0.5 * np.log(omega)))
        return omega

    assert not _table_ok(inverted_ratio, INIT_WEIGHT)
    for bad in (theta_one, ratio_flipped, no_reset):
        assert not _table_ok(bad, WEIGHT_UPDATE, tol=1e-12), bad.__name__


# ---------------------------------------------------------- KKT_omega
# sqrt(omega^2 p^2 + d^2 / omega^2 + gap^2)
KKT_OMEGA = [
    ((2.0, 3.0, 4.0, 1.0), math.sqrt(41.0)),   # 4*9 + 16/4 + 1
    ((0.5, 2.0, 1.0, 0.0), math.sqrt(5.0)),    # 0.25*4 + 1/0.25
]


def _kkt(omega, p, d, g):
    return kkt_omega(dict(abs_p=p, abs_d=d, abs_gap=g), omega)


def test_kkt_omega_table():
    assert _table_ok(_kkt, KKT_OMEGA)


def test_kkt_omega_rejects_planted_mistake():
    def weights_swapped(omega, p, d, g):
        return math.sqrt(p * p / omega ** 2 + omega ** 2 * d * d + g * g)

    assert not _table_ok(weights_swapped, KKT_OMEGA)


# ----------------------------------------------- fixed step (reading c21)
def test_fixed_step_size_hand_value_and_bound():
    # |G| column sums (4, 3, 4), row sums (3, 8): eta = 1 / sqrt(4 * 8)
    G = sp.csr_matrix(np.array([[1.0, -2.0, 0.0], [3.0, 1.0, 4.0]]))
    assert abs(OP.fixed_step_size(G) - 1.0 / math.sqrt(32.0)) < 1e-15
    # the bound: eta ||G||_2 <= 1 on random matrices
    rng = np.random.default_rng(0)
    for _ in range(20):
        A = sp.random(7, 5, density=0.5, random_state=rng, data_rvs=rng.standard_normal)
        A = sp.csr_matrix(A)
        if A.nnz:
            assert OP.fixed_step_size(A) * np.linalg.norm(A.toarray(), 2) <= 1.0 + 1e-12
    # planted mistakes: the column sums alone, or the largest entry (the
    # adaptive method's eta^0), give other values
    for wrong in (1.0 / float(np.max(abs(G).sum(axis=0))), 1.0 / float(np.max(abs(G.data)))):
        assert abs(wrong - 1.0 / math.sqrt(32.0)) > 1e-3


# ------------------------------------------------- infeasibility (c19)
class _Eps:
    eps_primal_infeasible_low_acc = 1e-12
    eps_dual_infeasible_low_acc = 1e-12
    eps_primal_infeasible_high_acc = 1e-16
    eps_dual_infeasible_high_acc = 1e-16


UP = [1.0, 2.0, 3.0, 4.0]        # strictly rising over the last 3 checks
FLAT = [1.0, 2.0, 2.0, 4.0]


def test_infeasibility_exit_table():
    e = _Eps()
    f = OP.infeasibility_exit
    assert f((0.0, np.inf), FLAT, FLAT, e) == 3            # high accuracy needs no trend
    assert f((np.inf, 1e-17), FLAT, FLAT, e) == 5
    assert f((1e-13, np.inf), UP, FLAT, e) == 2            # low accuracy with the trend
    assert f((1e-13, np.inf), FLAT, FLAT, e) is None       # ... and not without it
    assert f((1e-13, np.inf), UP[1:], FLAT, e) is None     # fewer than 4 checks: no trend
    assert f((np.inf, 1e-13), FLAT, UP, e) == 4
    assert f((1e-11, 1e-11), UP, UP, e) is None            # above both thresholds
    assert f((1e-13, 1e-17), UP, UP, e) == 5               # dual high before primal low
    assert f((1e-17, 1e-17), UP, UP, e) == 3               # primal high first


def _lp(G, h, c, lo, hi, rows):
    return ConicProblem(sp.csr_matrix(np.asarray(G, float)), h, c, len(c), np.asarray(lo, float),
                        np.asarray(hi, float), rows, [])


def test_primal_infeasible_lp_is_detected():
    """x1 + x2 >= 2 and x1 + x2 <= 1 with x >= 0: y = (1, 1) is a Farkas
    certificate (G^T y = 0, h^T y = 1 > 0)."""
    from scipy.optimize import linprog
    G = [[1.0, 1.0], [-1.0, -1.0]]
    h = [2.0, -1.0]
    assert linprog([1, 1], A_ub=-np.asarray(G), b_ub=-np.asarray(h), bounds=[(0, None)] * 2).status == 2
    res = oracle.solve(_lp(G, h, [1.0, 1.0], [0, 0], [np.inf, np.inf], [(C.NONNEG, 2)]),
                       max_iter=20000)
    assert res["exit_code"] in (2, 3)


def test_dual_infeasible_lp_is_detected():
    """min -x1 s.t. x1 - x2 >= 0, x2 >= 0, x >= 0: x = (t, t) drives the
    objective to -inf."""
    from scipy.optimize import linprog
    G = [[1.0, -1.0], [0.0, 1.0]]
    assert linprog([-1, 0], A_ub=-np.asarray(G), b_ub=[0, 0], bounds=[(0, None)] * 2).status == 3
    res = oracle.solve(_lp(G, [0.0, 0.0], [-1.0, 0.0], [0, 0], [np.inf, np.inf], [(C.NONNEG, 2)]),
                       max_iter=20000)
    assert res["exit_code"] in (4, 5)


def test_feasible_box_lp_with_positive_objective_is_not_declared_infeasible():
    """All-finite bounds make lambda feasible for every y, so a test on the
    candidate itself (not its change) would call this feasible LP infeasible."""
    res = oracle.solve(_lp([[1.0, 1.0]], [1.0], [1.0, 2.0], [0, 0], [3, 3], [(C.NONNEG, 1)]),
                       max_iter=20000)
    assert res["exit_code"] == 0 and abs(res["pobj"] - 1.0) < 1e-5


# ------------------------------------- the loop uses the pinned functions
def _trace(monkeypatch=None, **patch):
    p = workloads.tiny_conic(seed=4, m_nonneg=10, soc_rows=(4,), nb=20, soc_cols=(3,), density=0.3)
    if monkeypatch is not None:
        for name, fn in patch.items():
            monkeypatch.setattr(OP, name, fn)
    tr = []
    oracle.solve(oracle.problem_from_dict(p), trace=tr, max_iter=80, check_freq=16)
    return tr


@pytest.mark.parametrize("name, bad", [
    ("next_step_size", lambda eta, eb, kb: min((1.0 - (kb + 1) ** -0.6) * eb, (1.0 + (kb + 1) ** -0.3) * eta)),
    ("reflection", lambda e: 0.5),
    ("halpern_step", lambda k, b, zh, z, z0: (k + 1.0) / (k + 2.0) * zh + z0 / (k + 2.0)),
    ("restart_conditions", lambda v, r, p, k, kb: (False, False, False)),
    ("primal_weight_update", lambda dx, dy, w, w0: 2.0 * w),
])
def test_solver_loop_goes_through_the_pinned_functions(monkeypatch, name, bad):
    good = _trace()
    assert any(r["restart"] for r in good)
    changed = _trace(monkeypatch, **{name: bad})
    keys = ("eta", "eta_hat", "beta", "omega", "max_err", "restart")
    assert any(any(g[k] != c[k] for k in keys) for g, c in zip(good, changed)), name
