"""Infeasibility detection (Sec. 3.2.3, exit codes 2-5) on the GPU against the
oracle, on primal- and dual-infeasible linear programs whose infeasibility is
established independently (scipy's LP solver); feasible problems are never
declared infeasible (every other GPU test ends with exit code 0).

Both sides detect at a check where a ratio crosses its threshold; the
trajectories separate under rounding over thousands of iterations, so the
two may cross at different checks and the comparison is on the kind of
infeasibility (primal: 2 / 3, dual: 4 / 5).  With the paper's default
thresholds (1e-12 / 1e-16) the random primal-infeasible programs are not
detected within 30,000 iterations (their ratio falls noisily to ~1e-9), so
they run with the low-accuracy threshold at 1e-6."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_15504_b300 as P
    return P


def _lp(G, h, c, nb=None):
    n = G.shape[1]
    return workloads._pack(sp.csr_matrix(G), h, c, n, np.zeros(n), np.full(n, np.inf),
                           [(workloads.NONNEG, G.shape[0])], [], dict(kind="lp"))


def _random_primal_infeasible(seed):
    """G x - h >= 0, x >= 0 feasible at x0, plus the row -a^T x + h_a - 1 >= 0
    contradicting row a (a^T x >= h_a): y = e_a + e_new certifies
    infeasibility (G^T y = 0, h^T y = 1)."""
    rng = np.random.default_rng(seed)
    m, n = 12, 16
    G = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.5)
    x0 = rng.uniform(0.5, 1.5, n)
    h = G @ x0 - rng.uniform(0.1, 1.0, m)
    G = np.vstack([G, -G[3]])
    h = np.concatenate([h, [1.0 - h[3]]])
    # c > 0 keeps the dual feasible (y = 0), so the problem is primal
    # infeasible only
    return _lp(G, h, np.abs(rng.standard_normal(n)) + 0.1)


def _random_dual_infeasible(seed):
    """Feasible LP whose first column is nonnegative with c_0 < 0: x0 + t e_0
    stays feasible and c^T x -> -inf."""
    rng = np.random.default_rng(seed)
    m, n = 12, 16
    G = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.5)
    G[:, 0] = np.abs(G[:, 0])
    x0 = rng.uniform(0.5, 1.5, n)
    h = G @ x0 - rng.uniform(0.1, 1.0, m)
    c = np.abs(rng.standard_normal(n))
    c[0] = -1.0
    return _lp(G, h, c)


def _scipy_status(prob):
    G = workloads.to_scipy(prob).toarray()
    return linprog(prob["c"], A_ub=-G, b_ub=-prob["h"], bounds=[(0, None)] * prob["n"]).status


PRIMAL, DUAL = (2, 3), (4, 5)


def _both(prob, kind, **opts):
    P = _gpu()
    ref = oracle.solve(oracle.problem_from_dict(prob), max_iter=50000, **opts)
    res = P.solve(prob, max_iter=50000, time_limit=60.0, **opts)
    assert ref["exit_code"] in kind, ref["exit_code"]
    assert res["exit_code"] in kind, (res["status"], ref["exit_code"])
    return res, ref


def test_two_variable_lps():
    """x1 + x2 >= 2 and x1 + x2 <= 1 on x >= 0 (primal infeasible); min -x1 with
    x1 - x2 >= 0, x2 >= 0 (unbounded): both found at the second check."""
    G = np.array([[1.0, 1.0], [-1.0, -1.0]])
    res, ref = _both(_lp(G, np.array([2.0, -1.0]), np.array([1.0, 1.0])), PRIMAL)
    assert res["exit_code"] == ref["exit_code"] == 3 and res["iters"] == ref["iters"]
    G = np.array([[1.0, -1.0], [0.0, 1.0]])
    res, ref = _both(_lp(G, np.zeros(2), np.array([-1.0, 0.0])), DUAL)
    assert res["exit_code"] == ref["exit_code"] == 5 and res["iters"] == ref["iters"]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_primal_infeasible_lp(seed):
    prob = _random_primal_infeasible(seed)
    assert _scipy_status(prob) == 2  # infeasible
    _both(prob, PRIMAL, eps_primal_infeasible_low_acc=1e-6)


@pytest.mark.parametrize("seed", [1, 2])
def test_dual_infeasible_lp(seed):
    prob = _random_dual_infeasible(seed)
    assert _scipy_status(prob) == 3  # unbounded
    _both(prob, DUAL)
