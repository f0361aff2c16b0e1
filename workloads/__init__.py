"""Seeded synthetic conic programs shared by the tests, the benchmark and the
oracle comparisons.  This module only draws random data and assembles CSR
arrays; it contains none of the solver's arithmetic.

A problem is a dict with keys
    m, n           rows / columns of G
    row_ptr        int64 [m+1]     CSR of G
    col_idx        int32 [nnz]     (sorted within rows, no duplicates)
    val            float64 [nnz]
    h, c           float64 [m], [n]
    nb             number of leading box-bounded columns
    lo, hi         float64 [nb]    (+-inf allowed)
    row_cones      list of (type, dim); Gx - h lies in the product, in order
    col_cones      list of (type, dim); x[nb:] lies in the product, in order
    meta           dict describing the instance (sizes, seed, planted optimum...)
Cone type codes: 0 zero, 1 nonnegative, 2 second-order, 3 rotated second-order,
4 exponential (x, y, z) with y exp(x / y) <= z, 5 dual exponential.
"""
import numpy as np
import scipy.sparse as sp

ZERO, NONNEG, SOC, RSOC, EXP, DUAL_EXP = 0, 1, 2, 3, 4, 5


def _pack(G, h, c, nb, lo, hi, row_cones, col_cones, meta):
    G = sp.csr_matrix(G, dtype=np.float64)
    if not G.has_canonical_format:
        G.sum_duplicates()
        G.sort_indices()
    m, n = G.shape
    return dict(m=int(m), n=int(n), row_ptr=G.indptr.astype(np.int64),
                col_idx=G.indices.astype(np.int32), val=G.data.astype(np.float64),
                h=np.asarray(h, np.float64), c=np.asarray(c, np.float64), nb=int(nb),
                lo=np.asarray(lo, np.float64), hi=np.asarray(hi, np.float64),
                row_cones=[(int(t), int(d)) for t, d in row_cones],
                col_cones=[(int(t), int(d)) for t, d in col_cones], meta=meta)


def to_scipy(prob):
    """CSR matrix of a problem dict."""
    return sp.csr_matrix((prob["val"], prob["col_idx"], prob["row_ptr"]),
                         shape=(prob["m"], prob["n"]))


def _sparse_normal(rng, rows, cols, density):
    """rows x cols matrix, each entry nonzero independently with the given
    probability, nonzeros N(0, 1)."""
    nnz_expected = rows * cols * density
    if nnz_expected > 5e7:
        raise ValueError("matrix too large for the Bernoulli sampler")
    mask = rng.random((rows, cols)) < density if rows * cols <= 4e7 else None
    if mask is not None:
        r, cidx = np.nonzero(mask)
    else:
        k = rng.binomial(rows * cols, density)
        flat = np.unique(rng.integers(0, rows * cols, size=int(k * 1.05) + 16))[:k]
        r, cidx = np.divmod(flat, cols)
    v = rng.standard_normal(len(r))
    return sp.csr_matrix((v, (r, cidx)), shape=(rows, cols))


def _boundary_soc_pair(rng, dim):
    """Complementary boundary pair s = a (1, u), y = b (1, -u), ||u|| = 1."""
    u = rng.standard_normal(dim - 1)
    u /= np.linalg.norm(u)
    a, b = rng.uniform(0.5, 1.5, size=2)
    s = a * np.concatenate([[1.0], u])
    y = b * np.concatenate([[1.0], -u])
    return s, y


def _boundary_exp_pair(rng):
    """Complementary boundary pair of the exponential cone and its dual:
    p = a (r, 1, e^r) on the boundary of K_exp, q = b (-e^r, e^r (r - 1), 1) on
    the boundary of K_exp^* (-q_0 exp(q_1 / q_0) = b e = e q_2), p^T q = 0."""
    r = rng.uniform(-1.0, 1.0)
    a, b = rng.uniform(0.5, 1.5, size=2)
    er = np.exp(r)
    return a * np.array([r, 1.0, er]), b * np.array([-er, er * (r - 1.0), 1.0])


def tiny_conic(seed=20260101, m_nonneg=60, soc_rows=(10, 10, 10, 10), nb=150,
               soc_cols=(10, 10, 10, 10, 10), density=0.05, exp_rows=0, dexp_rows=0,
               exp_cols=0, dexp_cols=0):
    """Random conic program with a planted primal-dual optimum.

    G has N(0,1) entries with the given density.  Rows: m_nonneg nonnegative
    rows, SOC blocks, then exp_rows exponential and dexp_rows dual-exponential
    blocks; columns: nb box [0, inf), SOC blocks, then exp_cols exponential and
    dexp_cols dual-exponential blocks.  A strictly complementary
    (x*, s*, y*, lambda*) is drawn (boundary pairs for the cone blocks) and
    h = G x* - s*, c = G^T y* + lambda*, so the optimal value is
    c^T x* = h^T y*."""
    rng = np.random.default_rng(seed)
    m = m_nonneg + sum(soc_rows) + 3 * (exp_rows + dexp_rows)
    n = nb + sum(soc_cols) + 3 * (exp_cols + dexp_cols)
    G = _sparse_normal(rng, m, n, density)
    s = np.zeros(m)
    y = np.zeros(m)
    half = m_nonneg // 2
    mags = rng.uniform(0.5, 1.5, size=m_nonneg)
    perm = rng.permutation(m_nonneg)
    s[perm[:half]] = mags[perm[:half]]
    y[perm[half:]] = mags[perm[half:]]
    off = m_nonneg
    for dim in soc_rows:
        s[off:off + dim], y[off:off + dim] = _boundary_soc_pair(rng, dim)
        off += dim
    for b in range(exp_rows + dexp_rows):
        p_, q_ = _boundary_exp_pair(rng)
        # exp rows: s in K_exp, y in K_exp^*; dual-exp rows the other way round
        s[off:off + 3], y[off:off + 3] = (p_, q_) if b < exp_rows else (q_, p_)
        off += 3
    x = np.zeros(n)
    lam = np.zeros(n)
    halfc = nb // 2
    magc = rng.uniform(0.5, 1.5, size=nb)
    permc = rng.permutation(nb)
    x[permc[:halfc]] = magc[permc[:halfc]]
    lam[permc[halfc:]] = magc[permc[halfc:]]
    off = nb
    for dim in soc_cols:
        x[off:off + dim], lam[off:off + dim] = _boundary_soc_pair(rng, dim)
        off += dim
    for b in range(exp_cols + dexp_cols):
        p_, q_ = _boundary_exp_pair(rng)
        x[off:off + 3], lam[off:off + 3] = (p_, q_) if b < exp_cols else (q_, p_)
        off += 3
    h = G @ x - s
    c = G.T @ y + lam
    row_cones = ([(NONNEG, m_nonneg)] + [(SOC, d) for d in soc_rows] +
                 [(EXP, 3)] * exp_rows + [(DUAL_EXP, 3)] * dexp_rows)
    col_cones = ([(SOC, d) for d in soc_cols] + [(EXP, 3)] * exp_cols +
                 [(DUAL_EXP, 3)] * dexp_cols)
    meta = dict(kind="tiny_conic", seed=seed, x_star=x, y_star=y, s_star=s, lam_star=lam,
                opt=float(c @ x))
    return _pack(G, h, c, nb, np.zeros(nb), np.full(nb, np.inf), row_cones, col_cones, meta)


def portfolio(n=200_000, k=200, n_limits=1000, limit_density=1e-3, limit_nnz_min=1,
              gamma=1.0, seed=20260102, mu=None, F=None, d=None, limits=None):
    """Factor-model portfolio SOCP.

    Variables x in R^n (box [0, inf)) and t >= 0 (box [0, inf)); minimise
    -mu^T x + gamma t subject to
      1^T x = 1                                      (one zero-cone row)
      u_j - a_j^T x >= 0, j < n_limits               (nonnegative rows)
      (t, 1/2, F^T x, sqrt(d) o x) in RSOC^{k+n+2}  (2 t / 2 >= x^T (F F^T + D) x)
    F ~ N(0, 0.1^2) (n x k, stored as sparse rows of G), d ~ U(0.01, 0.1),
    mu ~ N(0.05, 0.02^2), a_j sparse N(0,1) with the given density (at least
    limit_nnz_min entries), u_j = a_j^T (1/n) + U(0,1)/n (feasible at x = 1/n).
    mu, F, d and limits may be passed in to share them across a family."""
    rng = np.random.default_rng(seed)
    if F is None:
        F = 0.1 * rng.standard_normal((n, k))
    if d is None:
        d = rng.uniform(0.01, 0.1, size=n)
    if mu is None:
        mu = 0.05 + 0.02 * rng.standard_normal(n)
    if limits is None:
        rows, cols, vals = [], [], []
        for j in range(n_limits):
            cnt = max(limit_nnz_min, rng.binomial(n, limit_density))
            cidx = np.sort(rng.choice(n, size=min(cnt, n), replace=False))
            rows.append(np.full(len(cidx), j))
            cols.append(cidx)
            vals.append(rng.standard_normal(len(cidx)))
        A = sp.csr_matrix((np.concatenate(vals) if vals else np.zeros(0),
                           (np.concatenate(rows) if rows else np.zeros(0, int),
                            np.concatenate(cols) if cols else np.zeros(0, int))),
                          shape=(n_limits, n))
        ub = A @ np.full(n, 1.0 / n) + rng.uniform(0.0, 1.0, size=n_limits) / n
        limits = (A, ub)
    A, ub = limits
    A = sp.csr_matrix(A)
    A.sort_indices()
    nv = n + 1                                   # x then t
    k = F.shape[1]
    L = A.shape[0]
    # Rows, assembled directly in CSR form: the budget row 1^T x = 1 (zero
    # cone); the limits u_j - a_j^T x >= 0 (G row -a_j, h = -u_j); the RSOC
    # block (t, 1/2, F^T x, sqrt(d) o x) as rows (e_t; 0 with h = -1/2; F^T; diag(sqrt d)).
    lens = [np.array([n]), np.diff(A.indptr), np.array([1, 0]), np.full(k, n),
            np.ones(n, dtype=np.int64)]
    idx = [np.arange(n), A.indices, np.array([n]), np.tile(np.arange(n), k), np.arange(n)]
    val = [np.ones(n), -A.data, np.array([1.0]), np.ascontiguousarray(F.T).ravel(), np.sqrt(d)]
    indptr = np.concatenate([[0], np.cumsum(np.concatenate(lens))]).astype(np.int64)
    G = sp.csr_matrix((np.concatenate(val), np.concatenate(idx).astype(np.int32), indptr),
                      shape=(1 + L + 2 + k + n, nv))
    h = np.concatenate([[1.0], -ub, [0.0, -0.5], np.zeros(k), np.zeros(n)])
    c = np.concatenate([-mu, [gamma]])
    row_cones = [(ZERO, 1)] + ([(NONNEG, L)] if L else []) + [(RSOC, F.shape[1] + n + 2)]
    meta = dict(kind="portfolio", seed=seed, n_assets=n, k=F.shape[1], n_limits=L, gamma=gamma)
    return _pack(G, h, c, nv, np.zeros(nv), np.full(nv, np.inf), row_cones, [], meta)


def portfolio_small_instance(n, seed):
    """One instance of the batched serving workload: the portfolio generator
    with k = max(1, n // 20) factors and ceil(n / 200) limits of
    max(2, ceil(1e-3 n)) nonzeros each."""
    k = max(1, n // 20)
    L = int(np.ceil(n / 200))
    nnz_l = max(2, int(np.ceil(1e-3 * n)))
    return portfolio(n=n, k=k, n_limits=L, limit_density=0.0, limit_nnz_min=nnz_l, seed=seed)


def portfolio_batch(count=4096, n_lo=50, n_hi=2000, seed=20260104):
    """count independent small portfolio SOCPs with n ~ U{n_lo..n_hi}."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    return [portfolio_small_instance(int(nn), seed + 1 + i) for i, nn in enumerate(ns)]


def logistic_l1(N=100_000, p=2000, density=0.005, support=50, flip=0.05, seed=20260103,
                reg_frac=0.1):
    """L1-regularised logistic regression in exponential-cone form.

    A (N x p) sparse N(0,1); planted w* with `support` nonzeros; labels
    sign(a_i^T w*) (ties by a fair coin), then a fraction `flip` flipped.
    Variables (all free, box (-inf, inf)): w (p), s (p), t (N), u (N), v (N).
    min sum t_i + lam sum s_j  subject to
      s_j - w_j >= 0, s_j + w_j >= 0                     (2p nonnegative rows)
      1 - u_i - v_i >= 0                                 (N nonnegative rows)
      (-y_i a_i^T w - t_i, 1, u_i) in K_exp,  (-t_i, 1, v_i) in K_exp
    lam = reg_frac * 0.5 * ||A^T y||_inf (the smallest lam with w = 0 optimal,
    scaled by reg_frac)."""
    rng = np.random.default_rng(seed)
    A = _sparse_normal(rng, N, p, density)
    w = np.zeros(p)
    sup = rng.choice(p, size=min(support, p), replace=False)
    w[sup] = rng.standard_normal(len(sup))
    z = A @ w
    lab = np.sign(z)
    ties = lab == 0
    lab[ties] = rng.choice([-1.0, 1.0], size=int(ties.sum()))
    fl = rng.random(N) < flip
    lab[fl] = -lab[fl]
    lam = reg_frac * 0.5 * np.max(np.abs(A.T @ lab))
    iw, is_, it, iu, iv = 0, p, 2 * p, 2 * p + N, 2 * p + 2 * N
    n = 2 * p + 3 * N
    rows, cols, vals, hs = [], [], [], []
    r = 0
    # s_j - w_j >= 0 ; s_j + w_j >= 0
    j = np.arange(p)
    rows += [r + j, r + j]; cols += [is_ + j, iw + j]; vals += [np.ones(p), -np.ones(p)]
    r += p
    rows += [r + j, r + j]; cols += [is_ + j, iw + j]; vals += [np.ones(p), np.ones(p)]
    r += p
    hs.append(np.zeros(2 * p))
    # 1 - u_i - v_i >= 0  ->  G row (-1 on u_i, -1 on v_i), h = -1
    i = np.arange(N)
    rows += [r + i, r + i]; cols += [iu + i, iv + i]; vals += [-np.ones(N), -np.ones(N)]
    r += N
    hs.append(-np.ones(N))
    # exp cones, 6 rows per sample
    base = r + 6 * i
    Ac = A.tocoo()
    rows += [base[Ac.row]]; cols += [iw + Ac.col]; vals += [-lab[Ac.row] * Ac.data]
    rows += [base]; cols += [it + i]; vals += [-np.ones(N)]
    rows += [base + 2]; cols += [iu + i]; vals += [np.ones(N)]
    rows += [base + 3]; cols += [it + i]; vals += [-np.ones(N)]
    rows += [base + 5]; cols += [iv + i]; vals += [np.ones(N)]
    he = np.zeros(6 * N)
    he[1::6] = -1.0
    he[4::6] = -1.0
    hs.append(he)
    m = r + 6 * N
    G = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(m, n))
    h = np.concatenate(hs)
    c = np.zeros(n)
    c[it:it + N] = 1.0
    c[is_:is_ + p] = lam
    row_cones = [(NONNEG, 2 * p + N)] + [(EXP, 3)] * (2 * N)
    meta = dict(kind="logistic_l1", seed=seed, N=N, p=p, lam=lam, w_star=w)
    return _pack(G, h, c, n, np.full(n, -np.inf), np.full(n, np.inf), row_cones, [], meta)


def portfolio_family(n=20_000, k=100, n_limits=100, seed=20260105):
    """Shared data (F, d, limits) of the parameterised portfolio family; each
    instance draws mu ~ N(0.05, 0.02^2) and gamma log-uniform on [0.1, 10]."""
    rng = np.random.default_rng(seed)
    F = 0.1 * rng.standard_normal((n, k))
    d = rng.uniform(0.01, 0.1, size=n)
    base = portfolio(n=n, k=k, n_limits=n_limits, seed=seed + 7, F=F, d=d,
                     mu=np.zeros(n))
    A_rows = to_scipy(base)[1:1 + n_limits, :n]
    ub = -base["h"][1:1 + n_limits]
    return dict(n=n, k=k, F=F, d=d, limits=(-A_rows, ub), seed=seed)


def portfolio_family_instance(fam, idx, split_seed=0):
    """Instance idx of a family: returns (problem, params) with params the
    concatenation (mu, gamma)."""
    rng = np.random.default_rng([fam["seed"], split_seed, idx])
    mu = 0.05 + 0.02 * rng.standard_normal(fam["n"])
    gamma = float(np.exp(rng.uniform(np.log(0.1), np.log(10.0))))
    prob = portfolio(n=fam["n"], k=fam["k"], F=fam["F"], d=fam["d"], limits=fam["limits"],
                     mu=mu, gamma=gamma, seed=fam["seed"])
    return prob, np.concatenate([mu, [gamma]])
