"""Pins for the oracle's cone projections (CPU only).

Each projection is checked against something other than itself: textbook
closed forms, the Moreau decomposition with the two pieces computed by
independent routines, and a general-purpose library optimiser (SciPy SLSQP) on
small random inputs."""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import cones as C


def _rng(seed=0):
    return np.random.default_rng(seed)


# --------------------------------------------------------------------------- SOC
def test_soc_closed_form_special_cases():
    # inside: unchanged; polar: zero; boundary case: ((t+|w|)/2)(1, w/|w|)
    v = np.array([5.0, 3.0, 4.0])
    assert np.allclose(C.proj_soc(v), v)
    v = np.array([-5.0, 3.0, 4.0])
    assert np.allclose(C.proj_soc(v), 0.0)
    v = np.array([1.0, 3.0, 4.0])
    assert np.allclose(C.proj_soc(v), [3.0, 1.8, 2.4])


@pytest.mark.parametrize("seed", range(5))
def test_scaled_soc_reduces_to_standard_when_d_is_constant(seed):
    rng = _rng(seed)
    for _ in range(50):
        dim = rng.integers(2, 12)
        v = rng.standard_normal(dim) * rng.uniform(0.1, 10)
        alpha = rng.uniform(0.1, 10.0)
        a = C.proj_soc_scaled(v, np.full(dim, alpha))
        b = C.proj_soc(v)
        assert np.allclose(a, b, rtol=1e-12, atol=1e-12 * np.linalg.norm(v))


def _in_scaled_soc(w, d, tol):
    return np.linalg.norm(w[1:] / d[1:]) <= w[0] / d[0] + tol


@pytest.mark.parametrize("seed", range(5))
def test_scaled_soc_moreau_with_independent_pieces(seed):
    """P_{DK}(v) - P_{D^{-1}K}(-v) = v and the two pieces are orthogonal; the
    second piece comes from a separate root-find on the reciprocal scaling."""
    rng = _rng(100 + seed)
    for _ in range(100):
        dim = int(rng.integers(2, 30))
        v = rng.standard_normal(dim) * 3
        d = np.exp(rng.uniform(-2, 2, size=dim))
        p = C.proj_soc_scaled(v, d)
        q = C.proj_soc_scaled(-v, 1.0 / d)
        scale = 1 + np.linalg.norm(v)
        assert np.allclose(p - q, v, atol=1e-10 * scale)
        assert abs(p @ q) <= 1e-9 * scale ** 2
        assert _in_scaled_soc(p, d, 1e-10 * scale)
        assert _in_scaled_soc(q, 1.0 / d, 1e-10 * scale)


@pytest.mark.parametrize("seed", range(3))
def test_scaled_soc_matches_library_optimiser(seed):
    rng = _rng(200 + seed)
    for _ in range(15):
        dim = int(rng.integers(2, 6))
        v = rng.standard_normal(dim) * 2
        d = np.exp(rng.uniform(-1, 1, size=dim))
        p = C.proj_soc_scaled(v, d)
        cons = {"type": "ineq", "fun": lambda w: w[0] / d[0] - np.sqrt(np.sum((w[1:] / d[1:]) ** 2) + 1e-300)}
        best = None
        for start in (np.zeros(dim) + 1e-3, p + 0.1 * rng.standard_normal(dim), np.abs(v)):
            r = minimize(lambda w: np.sum((w - v) ** 2), start, constraints=[cons],
                         method="SLSQP", options=dict(ftol=1e-14, maxiter=500))
            if _in_scaled_soc(r.x, d, 1e-7) and (best is None or r.fun < best.fun):
                best = r
        assert best is not None
        # SLSQP may end slightly outside the cone, so allow a small slack.
        assert np.sum((p - v) ** 2) <= best.fun + 1e-6
        assert np.allclose(p, best.x, atol=1e-3)


def test_scaled_soc_v0_zero_branch():
    rng = _rng(7)
    for _ in range(20):
        dim = int(rng.integers(2, 8))
        v = rng.standard_normal(dim)
        v[0] = 0.0
        d = np.exp(rng.uniform(-1, 1, size=dim))
        p = C.proj_soc_scaled(v, d)
        q = C.proj_soc_scaled(-v, 1.0 / d)
        assert np.allclose(p - q, v, atol=1e-10)
        assert abs(p @ q) < 1e-10


# --------------------------------------------------------------------------- EXP
def test_exp_special_cases():
    # inside the cone: unchanged
    p = np.array([[0.0, 1.0, 2.0]])
    assert np.allclose(C.proj_exp_scaled(p, np.ones(3)), p)
    # in the polar -K_exp^*: zero
    p = np.array([[1.0, -1.0, -5.0]])  # -p = (-1, 1, 5) in K_exp^*
    assert C.in_exp_dual(-p)[0]
    assert np.allclose(C.proj_exp_scaled(p, np.ones(3)), 0.0)
    # x <= 0 and y <= 0: (x, 0, max(z, 0))
    p = np.array([[-2.0, -1.0, 3.0], [-1.0, -0.5, -2.0]])
    for d in (np.ones(3), np.array([0.3, 2.0, 5.0])):
        assert np.allclose(C.proj_exp_scaled(p, d), [[-2.0, 0.0, 3.0], [-1.0, 0.0, 0.0]])


def _random_points(rng, k, scale=2.0):
    return rng.standard_normal((k, 3)) * scale


@pytest.mark.parametrize("seed", range(3))
def test_exp_moreau_with_direct_dual(seed):
    """P_{DK}(v) - P_{D^{-1}K^*}(-v) = v with the dual piece projected directly
    onto the dual cone's own boundary parametrisation."""
    rng = _rng(300 + seed)
    p = _random_points(rng, 300)
    d = np.exp(rng.uniform(-1.5, 1.5, size=(300, 3)))
    a = C.proj_exp_scaled(p, d)
    b = C.proj_exp_dual_scaled_direct(-p, 1.0 / d)
    scale = 1 + np.linalg.norm(p, axis=1)
    assert np.all(np.abs(a - b - p).max(axis=1) <= 1e-9 * scale)
    assert np.all(np.abs(np.sum(a * b, axis=1)) <= 1e-9 * scale ** 2)


@pytest.mark.parametrize("seed", range(3))
def test_exp_standard_moreau(seed):
    rng = _rng(400 + seed)
    p = _random_points(rng, 300, 5.0)
    a = C.proj_exp_scaled(p, np.ones(3))
    b = C.proj_exp_dual_scaled_direct(-p, np.ones(3))
    assert np.allclose(a - b, p, atol=1e-9 * (1 + np.abs(p).max()))


def _slsqp_exp(p, d):
    """Nearest point of diag(d) K_exp to p by SLSQP on u with w = d o u,
    using the log form u_x <= u_y log(u_z / u_y), u_y, u_z > 0."""
    def f(u):
        return np.sum((d * u - p) ** 2)
    cons = {"type": "ineq", "fun": lambda u: u[1] * np.log(u[2] / u[1]) - u[0]}
    bounds = [(None, None), (1e-12, None), (1e-12, None)]
    best = None
    for start in ([-1.0, 1.0, 1.0], [0.0, 1.0, 2.0], [1.0, 0.5, 5.0], [-3.0, 2.0, 0.5]):
        r = minimize(f, np.array(start), bounds=bounds, constraints=[cons], method="SLSQP",
                     options=dict(ftol=1e-15, maxiter=1000))
        if r.x[1] * np.log(r.x[2] / r.x[1]) - r.x[0] >= -1e-7 and (best is None or r.fun < best.fun):
            best = r
    return d * best.x, best.fun


@pytest.mark.parametrize("seed", range(2))
def test_exp_matches_library_optimiser(seed):
    rng = _rng(500 + seed)
    checked = 0
    while checked < 12:
        p = _random_points(rng, 1)[0]
        d = np.exp(rng.uniform(-1, 1, size=3))
        if C.in_exp((p / d)[None])[0] or C.in_exp_dual((-d * p)[None])[0]:
            continue
        if p[0] <= 0 and p[1] <= 0:
            continue
        q = C.proj_exp_scaled(p[None], d[None])[0]
        w, fval = _slsqp_exp(p, d)
        assert np.sum((q - p) ** 2) <= fval + 1e-7
        assert np.allclose(q, w, atol=2e-4)
        checked += 1


def test_exp_dual_via_moreau_matches_direct():
    rng = _rng(600)
    p = _random_points(rng, 200)
    d = np.exp(rng.uniform(-1, 1, size=(200, 3)))
    a = C.proj_exp_dual_scaled(p, d)
    b = C.proj_exp_dual_scaled_direct(p, d)
    assert np.allclose(a, b, atol=1e-9 * (1 + np.abs(p).max()))


# ------------------------------------------------------------------ elementwise
def test_lambda_projection_table():
    lo = np.array([-np.inf, -np.inf, 0.0, 0.0])
    hi = np.array([np.inf, 1.0, np.inf, 1.0])
    kind = C.lambda_kind(lo, hi)
    assert list(kind) == [0, 1, 2, 3]
    lam = np.array([2.0, 2.0, -2.0, -2.0])
    assert np.allclose(C.proj_lambda(lam, kind), [0.0, 0.0, 0.0, -2.0])
    lam = -lam
    assert np.allclose(C.proj_lambda(lam, kind), [0.0, -2.0, 2.0, 2.0])


def test_product_projection_dual_flag_and_moreau():
    rng = _rng(700)
    cones = [(C.ZERO, 2), (C.NONNEG, 3), (C.SOC, 4), (C.EXP, 3), (C.DUAL_EXP, 3)]
    n = sum(dm for _, dm in cones)
    for _ in range(20):
        v = rng.standard_normal(n) * 2
        d = np.exp(rng.uniform(-1, 1, size=n))
        p = C.proj_cone_product(v, cones, d, dual=False)
        q = C.proj_cone_product(-v, cones, 1.0 / d, dual=True)
        assert np.allclose(p - q, v, atol=1e-9)
        assert abs(p @ q) < 1e-8


# ------------------------------------------------------- planted-mistake check
def test_pins_detect_a_planted_mistake(monkeypatch):
    """A wrong scaled-SOC formula (multiplier applied with the wrong sign on the
    head) must be caught by the Moreau pin."""
    good = C.proj_soc_scaled

    def bad(v, d):
        out = good(v, d)
        if not np.allclose(out, v) and not np.allclose(out, 0):
            out = out.copy()
            out[0] = out[0] * 1.001
        return out

    monkeypatch.setattr(C, "proj_soc_scaled", bad)
    rng = _rng(800)
    failures = 0
    for _ in range(50):
        v = rng.standard_normal(6)
        d = np.exp(rng.uniform(-1, 1, size=6))
        p = C.proj_soc_scaled(v, d)
        q = C.proj_soc_scaled(-v, 1.0 / d)
        if not np.allclose(p - q, v, atol=1e-10):
            failures += 1
    assert failures > 0
