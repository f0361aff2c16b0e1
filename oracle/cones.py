"""Oracle cone projections (plain, slow, FP64 CPU code; test infrastructure only).

Every function here is an obviously-correct restatement of a Euclidean projection
that the restarted PDHG method of the paper needs: onto the zero cone, the
nonnegative orthant, boxes, the second-order cone K_soc, the exponential cone
K_exp and its dual K_exp^*, each possibly rescaled by a positive diagonal matrix D
(Sec. 2.6: the rescaled cones D_1 K_d^* and D_2^{-1} K_p are "non-standard" and
their projections reduce to root finding; the paper gives no formula, so the
derivations below are this project's own).

Conventions (Sec. 3.2.3 cone list, MOI ordering):
  K_soc  = {(t, w) : ||w||_2 <= t}
  K_exp  = cl{(x, y, z) : y > 0, y exp(x / y) <= z}
  K_exp* = cl{(u, v, w) : u < 0, -u exp(v / u) <= e w}
Scaled cone D K = {D k : k in K} for a positive vector d (D = diag(d)).
(D K)^* = D^{-1} K^*.  Moreau: v = P_C(v) + P_{C°}(v), C° = -C^*, hence
P_{C^*}(v) = v + P_C(-v).

Nothing here is imported by the CUDA product path.
"""
import numpy as np

ZERO, NONNEG, SOC, RSOC, EXP, DUAL_EXP = 0, 1, 2, 3, 4, 5


# ----------------------------------------------------------------------------
# Elementwise cones
# ----------------------------------------------------------------------------
def proj_nonneg(v):
    """Projection onto R_+^d: max(v, 0)."""
    return np.maximum(v, 0.0)


def proj_box(v, lo, hi):
    """Projection onto the box [lo, hi] (entries may be +-inf): clamp."""
    return np.minimum(np.maximum(v, lo), hi)


def lambda_kind(lo, hi):
    """Sec. 1.1, definition of Lambda_i from the finiteness of (l_i, u_i).

    Returns an int array: 0 -> {0} (both infinite), 1 -> R^- (only u finite),
    2 -> R^+ (only l finite), 3 -> R (both finite)."""
    lf = np.isfinite(lo)
    uf = np.isfinite(hi)
    kind = np.zeros(lo.shape, dtype=np.int64)
    kind[~lf & uf] = 1
    kind[lf & ~uf] = 2
    kind[lf & uf] = 3
    return kind


def proj_lambda(lam, kind):
    """Projection onto Lambda = prod_i Lambda_i (Sec. 1.1)."""
    out = lam.copy()
    out[kind == 0] = 0.0
    m1 = kind == 1
    out[m1] = np.minimum(lam[m1], 0.0)
    m2 = kind == 2
    out[m2] = np.maximum(lam[m2], 0.0)
    return out


# ----------------------------------------------------------------------------
# Second-order cone
# ----------------------------------------------------------------------------
def proj_soc(v):
    """Projection onto the standard K_soc (textbook closed form, e.g. Parikh &
    Boyd, Proximal Algorithms, Sec. 6.3.2)."""
    t = v[0]
    w = v[1:]
    nw = np.linalg.norm(w)
    if nw <= t:
        return v.copy()
    if nw <= -t:
        return np.zeros_like(v)
    a = 0.5 * (t + nw)
    out = np.empty_like(v)
    out[0] = a
    out[1:] = (a / nw) * w
    return out


def _bisect(fun, lo, hi, increasing, max_iter=400):
    """Bisection for the sign change of a monotone scalar function on (lo, hi)."""
    for _ in range(max_iter):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        f = fun(mid)
        if (f > 0) == increasing:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def proj_soc_scaled(v, d):
    """Projection onto diag(d) K_soc, d > 0 (a rescaled second-order cone).

    Derivation (own, from the KKT conditions of min 1/2||w - v||^2 subject to
    ||dbar^{-1} o wbar||^2 <= (w0 / d0)^2, w0 >= 0):
      (i)   ||vbar / dbar|| <= v0 / d0            -> v is in the cone, return v;
      (ii)  ||dbar o vbar|| <= -d0 v0            -> v in the polar -D^{-1}K, return 0;
      (iii) otherwise w lies on the boundary with
            wbar_i = vbar_i dbar_i^2 / (dbar_i^2 + 2 mu),
            w0     = v0 d0^2 / (d0^2 - 2 mu),
            for the unique mu > 0 solving ||dbar^{-1} o wbar(mu)|| = w0(mu) / d0,
            on (0, d0^2/2) when v0 > 0 and on (d0^2/2, inf) when v0 < 0;
            when v0 = 0, mu = d0^2/2 and w0 = d0 ||dbar^{-1} o wbar||.
    The root is found by plain bisection on the monotone residual
    psi(mu) = ||dbar^{-1} wbar(mu)|| - w0(mu)/d0 (decreasing for v0 > 0;
    2 mu psi(mu) increasing for v0 < 0)."""
    v = np.asarray(v, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    v0, vb = v[0], v[1:]
    d0, db = d[0], d[1:]
    if np.linalg.norm(vb / db) <= v0 / d0:
        return v.copy()
    if np.linalg.norm(vb * db) <= -d0 * v0:
        return np.zeros_like(v)
    db2 = db * db
    d02 = d0 * d0

    def wbar(mu):
        return vb * db2 / (db2 + 2.0 * mu)

    out = np.empty_like(v)
    if v0 == 0.0:
        mu = 0.5 * d02
        wb = wbar(mu)
        out[0] = d0 * np.linalg.norm(wb / db)
        out[1:] = wb
        return out

    def psi(mu):
        wb = wbar(mu)
        return np.linalg.norm(wb / db) - (v0 * d0 / (d02 - 2.0 * mu))

    if v0 > 0:
        mu = _bisect(psi, 0.0, 0.5 * d02, increasing=False)
    else:
        lo = 0.5 * d02
        hi = d02
        while psi(hi) <= 0:
            hi *= 2.0
        mu = _bisect(psi, lo, hi, increasing=True)
    out[0] = v0 * d02 / (d02 - 2.0 * mu)
    out[1:] = wbar(mu)
    return out


# ----------------------------------------------------------------------------
# Exponential cone and its dual (vectorised over cones: arrays of shape (k, 3))
# ----------------------------------------------------------------------------
def in_exp(u):
    """Membership in K_exp for rows of u (closed set)."""
    x, y, z = u[:, 0], u[:, 1], u[:, 2]
    with np.errstate(over="ignore", divide="ignore", invalid="ignore"):
        pos = (y > 0) & (y * np.exp(x / np.where(y > 0, y, 1.0)) <= z)
    face = (y == 0) & (x <= 0) & (z >= 0)
    return pos | face


def in_exp_dual(u):
    """Membership in K_exp^* for rows of u (closed set)."""
    a, b, c = u[:, 0], u[:, 1], u[:, 2]
    with np.errstate(over="ignore", divide="ignore", invalid="ignore"):
        neg = (a < 0) & (-a * np.exp(b / np.where(a < 0, a, -1.0)) <= np.e * c)
    face = (a == 0) & (b >= 0) & (c >= 0)
    return neg | face


# Grid of ray parameters used to locate the best boundary ray before the local
# refinement (sinh spacing: dense near 0, reaching |r| ~ 6e5; beyond that the
# ray directions are indistinguishable in FP64 from the limit rays).
_RGRID = np.sinh(np.linspace(-14.0, 14.0, 3001))


def _best_ray(p, d, ray, dray, chunk=1024):
    """Nearest point to p (rows) on the smooth boundary surface {s * D a(r): s >= 0}.

    The distance from p to the ray through D a(r) is ||p||^2 - phi(r)^2 with
    phi(r) = <p, D a(r)> / ||D a(r)|| (when positive), so the nearest surface
    point maximises phi.  phi is scanned on a fixed grid, then the bracket around
    the best grid point is refined by bisection on the sign of dphi/dr.
    Returns (q, dist2); dist2 = +inf where no ray has phi > 0."""
    k = p.shape[0]
    q = np.zeros_like(p)
    dist2 = np.full(k, np.inf)
    for s in range(0, k, chunk):
        pp = p[s:s + chunk]
        dd = d[s:s + chunk]
        A = ray(_RGRID[None, :, None]) * dd[:, None, :]          # (c, G, 3)
        num = np.einsum("cgj,cj->cg", A, pp)
        den = np.sqrt(np.einsum("cgj,cgj->cg", A, A))
        phi = num / den
        j = np.argmax(phi, axis=1)
        ok = phi[np.arange(len(j)), j] > 0
        lo = _RGRID[np.maximum(j - 1, 0)].copy()
        hi = _RGRID[np.minimum(j + 1, len(_RGRID) - 1)].copy()

        def dphi_sign(r):
            a = ray(r[:, None]) * dd
            da = dray(r[:, None]) * dd
            pa = np.sum(pp * a, axis=1)
            pda = np.sum(pp * da, axis=1)
            aa = np.sum(a * a, axis=1)
            ada = np.sum(a * da, axis=1)
            return pda * aa - pa * ada

        for _ in range(200):
            mid = 0.5 * (lo + hi)
            g = dphi_sign(mid)
            up = g > 0
            lo = np.where(up, mid, lo)
            hi = np.where(up, hi, mid)
        r = 0.5 * (lo + hi)
        a = ray(r[:, None]) * dd
        y = np.sum(pp * a, axis=1) / np.sum(a * a, axis=1)
        qq = np.where(ok[:, None], np.maximum(y, 0.0)[:, None] * a, 0.0)
        q[s:s + chunk] = qq
        dd2 = np.sum((pp - qq) ** 2, axis=1)
        dist2[s:s + chunk] = np.where(ok, dd2, np.inf)
    return q, dist2


# Ray directions and their r-derivatives.  Only the direction matters (phi and
# the sign of dphi/dr are unchanged when a(r) and a'(r) share a positive
# factor), so both are multiplied by exp(-max(0, exponent)) to avoid overflow.
def _exp_ray(r):
    """Direction of the boundary ray {(s r, s, s e^r)} of K_exp."""
    g = np.exp(-np.maximum(r, 0.0))
    return np.concatenate(np.broadcast_arrays(r * g, g, np.exp(r - np.maximum(r, 0.0))), axis=-1)


def _exp_dray(r):
    g = np.exp(-np.maximum(r, 0.0))
    return np.concatenate(np.broadcast_arrays(g, np.zeros_like(r), np.exp(r - np.maximum(r, 0.0))), axis=-1)


def _expd_ray(r):
    """Direction of the boundary ray {s (-1, r, e^{-r-1})} of K_exp^*."""
    e = -r - 1.0
    g = np.exp(-np.maximum(e, 0.0))
    return np.concatenate(np.broadcast_arrays(-g, r * g, np.exp(e - np.maximum(e, 0.0))), axis=-1)


def _expd_dray(r):
    e = -r - 1.0
    g = np.exp(-np.maximum(e, 0.0))
    return np.concatenate(np.broadcast_arrays(np.zeros_like(r), g, -np.exp(e - np.maximum(e, 0.0))), axis=-1)


def _nearest_of(p, cands):
    """Pick, per row, the candidate with the smallest distance to p."""
    best = None
    bestd = None
    for q, dist2 in cands:
        if best is None:
            best, bestd = q.copy(), dist2.copy()
        else:
            m = dist2 < bestd
            best[m] = q[m]
            bestd[m] = dist2[m]
    return best


def proj_exp_scaled(p, d):
    """Projection onto diag(d) K_exp for each row of p (shape (k, 3)).

    The boundary of D K_exp is the smooth surface {s D (r, 1, e^r) : s > 0, r real}
    together with the flat face D F = F = {(x, 0, z) : x <= 0, z >= 0}.  The
    projection is therefore the nearest of: p itself (if D^{-1} p is in K_exp),
    the origin, the projection onto the face F (a closed form, since F is an
    orthant-like polyhedral cone), and the nearest point of the smooth surface."""
    p = np.atleast_2d(np.asarray(p, dtype=np.float64))
    d = np.broadcast_to(np.asarray(d, dtype=np.float64), p.shape)
    k = p.shape[0]
    inside = in_exp(p / d)
    zero = (np.zeros_like(p), np.sum(p * p, axis=1))
    face_q = np.stack([np.minimum(p[:, 0], 0.0), np.zeros(k), np.maximum(p[:, 2], 0.0)], axis=1)
    face = (face_q, np.sum((p - face_q) ** 2, axis=1))
    surf = _best_ray(p, d, _exp_ray, _exp_dray)
    out = _nearest_of(p, [zero, face, surf])
    out[inside] = p[inside]
    return out


def proj_exp_dual_scaled_direct(p, d):
    """Projection onto diag(d) K_exp^*, computed directly from the boundary of the
    dual cone (used to pin proj_exp_scaled through the Moreau identity).

    Boundary of D K_exp^*: the surface {s D (-1, r, e^{-r-1}) : s > 0} and the
    face {(0, v, w) : v >= 0, w >= 0}."""
    p = np.atleast_2d(np.asarray(p, dtype=np.float64))
    d = np.broadcast_to(np.asarray(d, dtype=np.float64), p.shape)
    k = p.shape[0]
    inside = in_exp_dual(p / d)
    zero = (np.zeros_like(p), np.sum(p * p, axis=1))
    face_q = np.stack([np.zeros(k), np.maximum(p[:, 1], 0.0), np.maximum(p[:, 2], 0.0)], axis=1)
    face = (face_q, np.sum((p - face_q) ** 2, axis=1))
    surf = _best_ray(p, d, _expd_ray, _expd_dray)
    out = _nearest_of(p, [zero, face, surf])
    out[inside] = p[inside]
    return out


def proj_exp_dual_scaled(p, d):
    """Projection onto diag(d) K_exp^* = (diag(1/d) K_exp)^* via Moreau:
    P_{C^*}(v) = v + P_C(-v) with C = diag(1/d) K_exp."""
    p = np.atleast_2d(np.asarray(p, dtype=np.float64))
    d = np.broadcast_to(np.asarray(d, dtype=np.float64), p.shape)
    return p + proj_exp_scaled(-p, 1.0 / d)


# ----------------------------------------------------------------------------
# Products of cones
# ----------------------------------------------------------------------------
def cone_offsets(cones):
    """Start offset of each block of an ordered cone list [(type, dim), ...]."""
    off = [0]
    for _, dim in cones:
        off.append(off[-1] + int(dim))
    return off


def proj_cone_product(v, cones, d, dual=False):
    """Projection of v onto the product prod_b diag(d_b) K_b (or onto the product
    of the dual cones diag(d_b) K_b^* when dual=True).  ZERO/NONNEG/SOC/EXP/
    DUAL_EXP blocks; RSOC blocks must have been reformulated already."""
    v = np.asarray(v, dtype=np.float64)
    out = np.empty_like(v)
    off = cone_offsets(cones)
    exp_idx = []
    expd_idx = []
    for b, (typ, dim) in enumerate(cones):
        s, e = off[b], off[b + 1]
        if typ == ZERO:
            out[s:e] = v[s:e] if dual else 0.0
        elif typ == NONNEG:
            out[s:e] = proj_nonneg(v[s:e])
        elif typ == SOC:
            out[s:e] = proj_soc_scaled(v[s:e], d[s:e])
        elif typ == EXP:
            (expd_idx if dual else exp_idx).append(s)
        elif typ == DUAL_EXP:
            (exp_idx if dual else expd_idx).append(s)
        else:
            raise ValueError("unsupported cone type %r in projection" % (typ,))
    if exp_idx:
        ix = np.asarray(exp_idx)[:, None] + np.arange(3)[None, :]
        out[ix] = proj_exp_scaled(v[ix], d[ix])
    if expd_idx:
        ix = np.asarray(expd_idx)[:, None] + np.arange(3)[None, :]
        out[ix] = proj_exp_dual_scaled(v[ix], d[ix])
    return out
