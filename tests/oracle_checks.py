"""Helpers that judge a GPU result with the oracle (test infrastructure)."""
import numpy as np

import oracle
from oracle.kkt import unscaled_errors
from oracle.problem import apply_block_T


def oracle_kkt(prob, x, y):
    """The oracle's termination errors (Sec. 3.2.3, infinity norms) of the point
    (x, y) given in the problem's original variables, on the FP64 data."""
    o = oracle.Oracle(oracle.problem_from_dict(prob), oracle.Options(use_preconditioner=False))
    xt = apply_block_T(np.asarray(x, float), o.sp.col_T)
    yt = apply_block_T(np.asarray(y, float), o.sp.row_T)
    return unscaled_errors(o.sp, xt, yt)


def rel_dist(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(1.0, np.linalg.norm(b)))


def compare_with_oracle(prob, res, ref):
    """Relative distances of x, y and the objective of the GPU result res from
    the oracle's solution ref, and the oracle's KKT error of res's point."""
    e = oracle_kkt(prob, res["x"], res["y"])
    return dict(x=rel_dist(res["x"], ref["x"]), y=rel_dist(res["y"], ref["y"]),
                obj=abs(res["pobj"] - ref["pobj"]) / (1.0 + abs(ref["pobj"])), kkt=e["max_rel"])
