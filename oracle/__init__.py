"""Oracle: a plain, slow, FP64 CPU restatement of the restarted PDHG conic solver
described in the paper (PDCS technical note).  TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check of the package entry point and the benchmark's
CPU-baseline leg may import or run anything under this directory.  It shares no
code with the CUDA product path, and the product path never calls it.

Modules:
  cones    projections onto (rescaled) zero / nonnegative / box / SOC / exp cones
  problem  problem data, rotated-SOC reformulation, Ruiz + Pock-Chambolle scaling
  kkt      2-norm and infinity-norm KKT error measures
  pdcs     Algorithm 2 / Algorithm 1 loop with Function 1 and Algorithm 3
"""
from .cones import ZERO, NONNEG, SOC, RSOC, EXP, DUAL_EXP  # noqa: F401
from .problem import ConicProblem, ScaledProblem  # noqa: F401
from .pdcs import Oracle, Options, solve  # noqa: F401


def problem_from_dict(p):
    """ConicProblem from a workloads-style problem dict (CSR arrays)."""
    import scipy.sparse as sp
    G = sp.csr_matrix((p["val"], p["col_idx"], p["row_ptr"]), shape=(p["m"], p["n"]))
    return ConicProblem(G, p["h"], p["c"], p["nb"], p["lo"], p["hi"], p["row_cones"],
                        p["col_cones"])
