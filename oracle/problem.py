"""Oracle problem set-up: conic problem data, rotated-SOC reformulation and
diagonal rescaling (test infrastructure only; plain FP64 CPU code).

Problem (Sec. 1.1, eq. prob_cp):
    min c^T x  s.t.  G x - h in K_r,  l <= x_[0:nb] <= u,  x_[nb:n] in K_p,
where K_r (the row cone, written K_d^* in the paper) and K_p are ordered products
of ZERO / NONNEG / SOC / RSOC / EXP / DUAL_EXP blocks (Sec. 3.2.3 cone list).

Rescaled problem (Sec. 2.6, eq. rescaled_prob and Algorithm 2):
    Ghat = D1 G D2, chat = D2 c, hhat = D1 h, lhat = l / D2, uhat = u / D2,
    row cone D1 K_r, column cone D2^{-1} K_p; solution x = D2 xt, y = D1 yt.
How D1, D2 are chosen is not stated in the paper; the reading used here is
10 Ruiz equilibration passes (row / column infinity norms) followed by one
Pock-Chambolle pass with alpha = 1 (row / column 1-norms), per element.
"""
import numpy as np
import scipy.sparse as sp

from .cones import ZERO, NONNEG, SOC, RSOC, EXP, DUAL_EXP, cone_offsets

SQRT_HALF = np.sqrt(0.5)


class ConicProblem:
    """Data of one conic program (the paper's problem statement, Sec. 1.1)."""

    def __init__(self, G, h, c, nb, lo, hi, row_cones, col_cones):
        self.G = sp.csr_matrix(G, dtype=np.float64)
        self.m, self.n = self.G.shape
        self.h = np.asarray(h, dtype=np.float64).copy()
        self.c = np.asarray(c, dtype=np.float64).copy()
        self.nb = int(nb)
        self.lo = np.asarray(lo, dtype=np.float64).copy()
        self.hi = np.asarray(hi, dtype=np.float64).copy()
        self.row_cones = [(int(t), int(dm)) for t, dm in row_cones]
        self.col_cones = [(int(t), int(dm)) for t, dm in col_cones]
        if sum(dm for _, dm in self.row_cones) != self.m:
            raise ValueError("row cone dims must sum to m")
        if sum(dm for _, dm in self.col_cones) != self.n - self.nb:
            raise ValueError("column cone dims must sum to n - nb")
        for t, dm in self.row_cones + self.col_cones:
            if t in (EXP, DUAL_EXP) and dm != 3:
                raise ValueError("exponential cone blocks have dimension 3")
            if t in (SOC,) and dm < 1:
                raise ValueError("SOC blocks need dimension >= 1")
            if t == RSOC and dm < 2:
                raise ValueError("RSOC blocks need dimension >= 2")


def reformulate_rsoc(prob):
    """Return (problem with every RSOC block rewritten as SOC, row_T, col_T).

    Sec. 3: rotated SOCs are handled by reformulation as standard SOCs.  The
    symmetric orthogonal map T (T = T^T = T^{-1}) acts on the first two entries of
    a block, (p, q, r) -> ((p+q)/sqrt2, (p-q)/sqrt2, r), and takes the rotated
    cone {2 p q >= ||r||^2, p, q >= 0} onto the standard SOC.  row_T / col_T list
    the start offsets of the transformed blocks, so y_original = T y_solver and
    x_original = T x_solver on those blocks."""
    G = prob.G.copy()
    h = prob.h.copy()
    c = prob.c.copy()
    row_T = []
    col_T = []
    roff = cone_offsets(prob.row_cones)
    new_rows = []
    for b, (t, dm) in enumerate(prob.row_cones):
        if t == RSOC:
            row_T.append(roff[b])
            new_rows.append((SOC, dm))
        else:
            new_rows.append((t, dm))
    coff = cone_offsets(prob.col_cones)
    new_cols = []
    for b, (t, dm) in enumerate(prob.col_cones):
        if t == RSOC:
            col_T.append(prob.nb + coff[b])
            new_cols.append((SOC, dm))
        else:
            new_cols.append((t, dm))
    if row_T:
        T = sp.identity(prob.m, format="lil")
        for s in row_T:
            T[s, s] = SQRT_HALF
            T[s, s + 1] = SQRT_HALF
            T[s + 1, s] = SQRT_HALF
            T[s + 1, s + 1] = -SQRT_HALF
        T = T.tocsr()
        G = (T @ G).tocsr()
        h = T @ h
    if col_T:
        T = sp.identity(prob.n, format="lil")
        for s in col_T:
            T[s, s] = SQRT_HALF
            T[s, s + 1] = SQRT_HALF
            T[s + 1, s] = SQRT_HALF
            T[s + 1, s + 1] = -SQRT_HALF
        T = T.tocsr()
        G = (G @ T).tocsr()
        c = T @ c
    G.eliminate_zeros()
    G.sort_indices()
    out = ConicProblem(G, h, c, prob.nb, prob.lo, prob.hi, new_rows, new_cols)
    return out, row_T, col_T


def apply_block_T(v, starts):
    """Apply the RSOC rotation to the first two entries of each listed block."""
    v = v.copy()
    for s in starts:
        a, b = v[s], v[s + 1]
        v[s] = SQRT_HALF * (a + b)
        v[s + 1] = SQRT_HALF * (a - b)
    return v


def _safe_inv_sqrt(norms):
    out = np.ones_like(norms)
    nz = norms > 0
    out[nz] = 1.0 / np.sqrt(norms[nz])
    return out


def compute_scaling(G, ruiz_iters=10, pc_alpha=1.0):
    """Diagonal rescaling D1 (rows), D2 (columns) of G (Sec. 2.6; reading c1).

    Ruiz: each pass divides row i by sqrt(max_j |Ghat_ij|) and column j by
    sqrt(max_i |Ghat_ij|) (a zero norm leaves the row/column unchanged).
    Pock-Chambolle (alpha): rows by sqrt(sum_j |Ghat_ij|^alpha), columns by
    sqrt(sum_i |Ghat_ij|^(2-alpha)).  pc_alpha < 0 skips the PC pass."""
    m, n = G.shape
    d1 = np.ones(m)
    d2 = np.ones(n)
    A = abs(sp.csr_matrix(G))
    for _ in range(ruiz_iters):
        S = sp.diags(d1) @ A @ sp.diags(d2)
        S = sp.csr_matrix(S)
        rn = np.zeros(m)
        cn = np.zeros(n)
        if S.nnz:
            rn = np.asarray(S.max(axis=1).todense()).ravel()
            cn = np.asarray(S.max(axis=0).todense()).ravel()
        d1 = d1 * _safe_inv_sqrt(rn)
        d2 = d2 * _safe_inv_sqrt(cn)
    if pc_alpha >= 0:
        S = sp.csr_matrix(sp.diags(d1) @ A @ sp.diags(d2))
        rn = np.asarray(S.power(pc_alpha).sum(axis=1)).ravel() if S.nnz else np.zeros(m)
        cn = np.asarray(S.power(2.0 - pc_alpha).sum(axis=0)).ravel() if S.nnz else np.zeros(n)
        d1 = d1 * _safe_inv_sqrt(rn)
        d2 = d2 * _safe_inv_sqrt(cn)
    return d1, d2


class ScaledProblem:
    """The rescaled problem of Sec. 2.6 plus the data the solver loop needs."""

    def __init__(self, prob, use_preconditioner=True, ruiz_iters=10, pc_alpha=1.0):
        self.orig = prob
        rp, self.row_T, self.col_T = reformulate_rsoc(prob)
        self.base = rp                      # SOC-only problem, unscaled
        if use_preconditioner:
            d1, d2 = compute_scaling(rp.G, ruiz_iters, pc_alpha)
        else:
            d1, d2 = np.ones(rp.m), np.ones(rp.n)
        self.d1, self.d2 = d1, d2
        self.G = sp.csr_matrix(sp.diags(d1) @ rp.G @ sp.diags(d2))
        self.GT = sp.csr_matrix(self.G.T)
        self.h = d1 * rp.h
        self.c = d2 * rp.c
        nb = rp.nb
        self.nb = nb
        self.lo = rp.lo / d2[:nb]
        self.hi = rp.hi / d2[:nb]
        self.m, self.n = rp.m, rp.n
        self.row_cones = rp.row_cones
        self.col_cones = rp.col_cones
