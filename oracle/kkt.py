"""Oracle KKT error measures (test infrastructure only; plain FP64 CPU code).

Two families, both from the paper:
  * 2-norm absolute errors err_abs,{p,d,gap} (Sec. 1.1, eq. tolerance-3) and their
    relative forms with 1-norm denominators (Sec. 2.2, eq. tolerance-2); maxErr
    (eq. tolerance) drives the reflection parameter and KKT_omega (Sec. 2.3)
    is the restart fallback.  Evaluated on the rescaled problem (reading c11).
  * infinity-norm termination errors (Sec. 3.2.3, eqs. PDCS_terminate_tolerance_abs
    and _rel), evaluated on the unscaled problem x = D2 xt, y = D1 yt with the
    standard cones.
"""
import numpy as np

from .cones import lambda_kind, proj_lambda, proj_cone_product


def dual_objective(h, y, lo, hi, lam1):
    """y^T h + l^T lam1^+ - u^T lam1^-; infinite bounds contribute nothing
    (reading c14)."""
    lp = np.maximum(lam1, 0.0)
    lm = np.maximum(-lam1, 0.0)
    fl = np.isfinite(lo)
    fu = np.isfinite(hi)
    return float(h @ y + np.sum(lo[fl] * lp[fl]) - np.sum(hi[fu] * lm[fu]))


def residual_pieces(h, c, nb, lo, hi, row_cones, col_cones, d_row, d_lam, x, y, Gx, GTy):
    """Primal residual vector, its projection, and the dual residual vectors.

    Gx - h must lie in the row cone diag(d_row) K_r; lambda_2 (the cone part of
    c - G^T y) must lie in diag(d_lam) K_p^*.  For the rescaled problem the
    column cone is D2^{-1} K_p, whose dual is D2 K_p^*, so d_lam = D2 there."""
    u = Gx - h
    pu = proj_cone_product(u, row_cones, d_row, dual=False)
    rp = u - pu
    lam = c - GTy
    lam1 = lam[:nb]
    lam2 = lam[nb:]
    kind = lambda_kind(lo, hi)
    rd1 = lam1 - proj_lambda(lam1, kind)
    rd2 = lam2 - proj_cone_product(lam2, col_cones, d_lam[nb:], dual=True)
    pobj = float(c @ x)
    dobj = dual_objective(h, y, lo, hi, lam1)
    return rp, pu, rd1, rd2, pobj, dobj


def scaled_errors(sp_, x, y):
    """2-norm absolute and relative errors of (x, y) for the rescaled problem.

    Returns dict with abs_p, abs_d, abs_gap, rel_p, rel_d, rel_gap, max_err,
    pobj, dobj.  Gx and G^T y are recomputed directly."""
    Gx = sp_.G @ x
    GTy = sp_.GT @ y
    rp, _, rd1, rd2, pobj, dobj = residual_pieces(
        sp_.h, sp_.c, sp_.nb, sp_.lo, sp_.hi, sp_.row_cones, sp_.col_cones,
        sp_.d1, sp_.d2, x, y, Gx, GTy)
    abs_p = float(np.linalg.norm(rp))
    abs_d = float(np.sqrt(rd1 @ rd1 + rd2 @ rd2))
    abs_gap = abs(pobj - dobj)
    rel_p = abs_p / (1.0 + np.sum(np.abs(sp_.h)))
    rel_d = abs_d / (1.0 + np.sum(np.abs(sp_.c)))
    rel_gap = abs_gap / (1.0 + abs(pobj) + abs(dobj))
    return dict(abs_p=abs_p, abs_d=abs_d, abs_gap=abs_gap, rel_p=rel_p, rel_d=rel_d,
                rel_gap=rel_gap, max_err=max(rel_p, rel_d, rel_gap), pobj=pobj, dobj=dobj)


def kkt_omega(err, omega):
    """Weighted KKT error of Sec. 2.3 from the absolute 2-norm errors."""
    return float(np.sqrt(omega ** 2 * err["abs_p"] ** 2 + err["abs_d"] ** 2 / omega ** 2
                         + err["abs_gap"] ** 2))


def unscaled_errors(sp_, xt, yt):
    """Infinity-norm termination errors (Sec. 3.2.3) of the unscaled point
    x = D2 xt, y = D1 yt on the SOC-reformulated problem with standard cones."""
    base = sp_.base
    x = sp_.d2 * xt
    y = sp_.d1 * yt
    Gx = base.G @ x
    GTy = base.G.T @ y
    ones_r = np.ones(base.m)
    ones_c = np.ones(base.n)
    rp, pu, rd1, rd2, pobj, dobj = residual_pieces(
        base.h, base.c, base.nb, base.lo, base.hi, base.row_cones, base.col_cones,
        ones_r, ones_c, x, y, Gx, GTy)
    inf = lambda v: float(np.max(np.abs(v))) if v.size else 0.0
    abs_p = inf(rp)
    abs_d = max(inf(rd1), inf(rd2))
    abs_gap = abs(pobj - dobj)
    rel_p = abs_p / (1.0 + max(inf(base.h), inf(Gx), inf(pu)))
    rel_d = abs_d / (1.0 + max(inf(base.c), inf(GTy)))
    rel_gap = abs_gap / (1.0 + max(abs(pobj), abs(dobj)))
    return dict(abs_p=abs_p, abs_d=abs_d, abs_gap=abs_gap, rel_p=rel_p, rel_d=rel_d,
                rel_gap=rel_gap, max_rel=max(rel_p, rel_d, rel_gap), pobj=pobj, dobj=dobj,
                x=x, y=y, Gx=Gx)
