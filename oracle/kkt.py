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


def _proj_recession_box(v, lo, hi):
    """Projection onto the recession cone of the box [lo, hi]: {0} where both
    bounds are finite, R_+ (R_-) where only lo (hi) is finite, R otherwise."""
    out = v.copy()
    lf, uf = np.isfinite(lo), np.isfinite(hi)
    out[lf & uf] = 0.0
    m = lf & ~uf
    out[m] = np.maximum(v[m], 0.0)
    m = ~lf & uf
    out[m] = np.minimum(v[m], 0.0)
    return out


def infeasibility_ratios(sp_, dxt, dyt):
    """Ratios of the infeasibility tests of Sec. 3.2.3 (reading c19) for the
    direction (dxt, dyt) in the solver's scaled variables (the change of the
    restart candidate between two checks), evaluated on the unscaled
    SOC-reformulated problem after x = D2 dxt, y = D1 dyt.

    Primal infeasibility (a Farkas ray y): the dual error of eq.
    PDCS_terminate_tolerance_abs for the homogeneous problem (c = 0, so
    lambda = -G^T y), together with the distance of y from the dual row cone,
    over the dual objective y^T h + l^T lambda_1^+ - u^T lambda_1^- (finite
    bounds); +inf unless that objective is positive.
    Dual infeasibility (a ray x): the relative primal error of eq.
    PDCS_terminate_tolerance_rel for the homogeneous problem (h = 0), together
    with the distance of x from the recession cone of [l, u] x K_p, over
    -c^T x; +inf unless -c^T x is positive.
    Returns (primal_ratio, dual_ratio)."""
    base = sp_.base
    nb = base.nb
    x = sp_.d2 * dxt
    y = sp_.d1 * dyt
    inf = lambda v: float(np.max(np.abs(v))) if v.size else 0.0
    lam = -(base.G.T @ y)
    lam1 = lam[:nb]
    ed1 = lam1 - proj_lambda(lam1, lambda_kind(base.lo, base.hi))
    ed2 = lam[nb:] - proj_cone_product(lam[nb:], base.col_cones, np.ones(base.n - nb), dual=True)
    ey = y - proj_cone_product(y, base.row_cones, np.ones(base.m), dual=True)
    dobj = dual_objective(base.h, y, base.lo, base.hi, lam1)
    num_p = max(inf(ed1), inf(ed2), inf(ey))
    gx = base.G @ x
    pg = proj_cone_product(gx, base.row_cones, np.ones(base.m), dual=False)
    rel_p = inf(gx - pg) / (1.0 + max(inf(gx), inf(pg)))
    ex1 = x[:nb] - _proj_recession_box(x[:nb], base.lo, base.hi)
    ex2 = x[nb:] - proj_cone_product(x[nb:], base.col_cones, np.ones(base.n - nb), dual=False)
    num_d = max(rel_p, inf(ex1), inf(ex2))
    mpobj = -float(base.c @ x)
    return (num_p / dobj if dobj > 0 else np.inf), (num_d / mpobj if mpobj > 0 else np.inf)
