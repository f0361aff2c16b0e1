"""The step-size test (Function 1) needs (k+1)^-0.3 and (k+1)^-0.6 once per
attempt.  The CUDA path does not call an FP64 pow for them (a long chain of
FP64 operations on the part's scarce FP64 pipe): it takes an FP32 seed and
two Newton steps in FP64 on f(p) = K p^10 - 1, K = kb1^3, with 1/q expanded
to second order around 1 (step_powers in csrc/iterate.cuh).  This checks that
method's error bound on the host, in the same FP64 operations, against the
correctly rounded power, over the counts a solve reaches and for seeds off by
the worst FP32 error and more."""
import numpy as np


def _refine(kb1, seed):
    p = np.float64(seed)
    K = kb1 * kb1 * kb1
    for _ in range(2):
        p2 = p * p
        p4 = p2 * p2
        p8 = p4 * p4
        e = p8 * p2 * K - 1.0
        p = p - 0.1 * p * (e * (1.0 - e))
    return p, p * p


def test_newton_refined_powers_are_within_a_few_ulps():
    kb = np.unique(np.concatenate([np.arange(2, 5000), np.geomspace(5000, 2e7, 4000).round()]))
    worst3 = worst6 = 0.0
    for kb1 in kb.astype(np.float64):
        exact3, exact6 = kb1 ** -0.3, kb1 ** -0.6
        seed32 = np.float32(kb1) ** np.float32(-0.3)
        for rel in (0.0, 3e-7, -3e-7, 2e-6, -2e-6):  # FP32 seed error and beyond
            p3, p6 = _refine(kb1, np.float64(seed32) * (1.0 + rel))
            worst3 = max(worst3, abs(p3 - exact3) / exact3)
            worst6 = max(worst6, abs(p6 - exact6) / exact6)
    assert worst3 <= 6e-16, worst3  # a few units of 2^-53 (1.1e-16)
    assert worst6 <= 1.2e-15, worst6


def test_step_factors_keep_their_order():
    # 1 - kb1^-0.3 and 1 + kb1^-0.6 bracket the step as Function 1 needs:
    # increasing and decreasing in kb1 respectively
    kb = np.arange(2.0, 3000.0)
    p3 = np.array([_refine(k, np.float32(k) ** np.float32(-0.3))[0] for k in kb])
    p6 = p3 * p3
    assert np.all(np.diff(1.0 - p3) > 0.0)
    assert np.all(np.diff(1.0 + p6) < 0.0)
