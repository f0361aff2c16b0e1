// Device kernels of one restarted-PDHG solve (PDCS note, Algorithm 1 on the
// rescaled problem of Sec. 2.6).  All scalars live in one device struct (Ctl)
// so the loop runs from captured CUDA graphs without host round trips:
//   attempt   Function 1: primal step, G xhat, dual step, step-size test,
//             then (accepted) G^T yhat, maxErr(zhat) -> beta (eq.
//             adaptive_reflection), reflected Halpern step and weighted average
//             (Algorithm 1);
//   check     every check_freq accepted iterations: average candidate, KKT
//             statistics of both candidates, normalized duality gaps by the
//             bisection of Algorithm 3, restart candidate / conditions / KKT_omega
//             fallback (Sec. 2.3), primal weight (Sec. 2.5), termination (Sec.
//             3.2.3).
// Grid-level sums use a fixed-order two-stage reduction (per-CTA partials, the
// last CTA to finish adds them in CTA order), so every run is deterministic.
#pragma once
#include "common.cuh"
#include "cones.cuh"
#include "spmv.cuh"

namespace pdcs {

enum : int { kRunning = -1 };
// Row kinds (the cone G x - h belongs to) and column kinds.
enum : uint8_t { RK_FREE = 0, RK_NONNEG = 1, RK_SOC = 2, RK_EXP = 3, RK_DEXP = 4 };
enum : uint8_t { CK_BOX = 0, CK_ZERO = 1, CK_NONNEG = 2, CK_SOC = 3, CK_EXP = 4, CK_DEXP = 5 };
enum : int { BS_DONE = 0, BS_EXP = 1, BS_BISECT = 2 };
enum : int { CNT_STEP = 0, CNT_STATS0 = 1, CNT_HALPERN = 5, CNT_PROBE = 6, CNT_INFEAS = 7, CNT_NUM = 8 };
constexpr int kTraceF = 13;  // trace row: the fields listed with pdcs_get_trace
constexpr int kHist = 4;     // checks kept for the infeasibility trend (3 rises)
constexpr int kEwThreads = 256;
constexpr int kStatSums = 8, kStatMax = 5, kStatK = kStatSums + kStatMax;

struct PointStats {
  double abs_p, abs_d, pobj, dobj, gap, rel_p, rel_d, rel_gap, max_err;
  double u2, lam2, dx2, dy2;
  double inf_abs_p, inf_abs_d, inf_rel_p, inf_rel_d, inf_rel_gap, inf_max;
};

struct Bisect {
  int phase, k, nb, active;
  double t, tl, tr, r, tau, sigma, result, last_dot;
};

struct Ctl {
  double eta, eta_hat, eta_acc, omega, omega0, eta0, beta, wsum;
  long long kbar, iter, k, period, restarts;
  int status, accepted, period_done, cand;
  int have_cand, has_ref, has_prev, pad0;
  double ref_rho, ref_ep, ref_ed, ref_eg;
  double prev_rho, prev_ep, prev_ed, prev_eg;
  double h1, c1, hinf, cinf;
  double rel_tol, abs_tol, bisect_tol, pad1;
  long long check_freq, max_iter;
  int method, adaptive_restart, require_abs, trace_cap;
  int guard, guard_cap, probes, probe_cap;
  int g_attempt, g_accept, g_check, g_restart;
  long long bodies_a, bodies_b;  // executions of the attempt / probe loop bodies
  // options of Sec. 3.2.3: fixed step, restart criteria, infeasibility tests
  int adaptive_step, gap_restart, kkt_restart, infeas_on;
  long long kkt_freq;
  double eta_fixed;
  double eps_pl, eps_dl, eps_ph, eps_dh;
  // the current check: rho^N computed (gap criterion), KKT criterion, KKT_omega used
  int chk_gap, chk_kkt, chk_fb, n_hist;
  double hist_d[kHist], hist_p[kHist];  // candidates' dual objective / -c^T x, newest last
  double infeas[2][2];  // per candidate: (primal, dual) ratio of its change since the last one
  int infeas_gate[2];   // the infeasibility statistics run for candidate 0 / 1
  PointStats st[4];  // 0 zhat (attempt), 1 z, 2 zbar (check), 3 returned point
  Bisect bs[2];
  unsigned int cnt[CNT_NUM];
};

template <typename T>
struct Prob {
  int64_t m, n, nb;
  const T* h;
  const T* c;
  const double* lo;
  const double* hi;
  const double* d1;
  const double* d2;
  const uint8_t* rk;
  const uint8_t* ck;
  KTimer* tm;  // timer slots (NULL: not profiling)
};

template <typename T>
struct PointRef {
  const T* x;
  const T* y;
  const T* gx;
  const T* gty;
};

struct TmpRef {
  double* tm;  // scaled projection of u = G x - h on cone rows
  double* tn;  // scaled projection of lambda = c - G^T y on cone columns
  double* um;  // unscaled projection of u / d1 on cone rows
  double* un;  // unscaled projection of lambda / d2 on cone columns
};

#define PDCS_GRID_LOOP(i, N) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (N); i += (int64_t)gridDim.x * blockDim.x)

// ---------------------------------------------------------------- attempt
// xhat = Proj_X(x - tau (c - G^T y)), tau = eta / omega (eq. PDHG); cone columns
// are projected afterwards by the cone kernels.
template <typename T>
PDCS_DEV void primal_elem(const Prob<T>& p, double tau, const T* __restrict__ x,
                          const T* __restrict__ gty, T* __restrict__ xh, int64_t j) {
  double v = (double)x[j] - tau * ((double)p.c[j] - (double)gty[j]);
  const uint8_t kd = p.ck[j];
  if (kd == CK_BOX) v = fmin(fmax(v, p.lo[j]), p.hi[j]);
  else if (kd == CK_ZERO) v = 0.0;
  else if (kd == CK_NONNEG) v = fmax(v, 0.0);
  xh[j] = (T)v;
}

// sx (FP32-value mode without column cones, else NULL): also the FP32
// (hi, lo) shadow of xhat that the product G xhat gathers.
template <typename T>
__global__ void __launch_bounds__(kEwThreads) k_primal(Prob<T> p, const Ctl* __restrict__ ctl,
                                                       const T* __restrict__ x,
                                                       const T* __restrict__ gty,
                                                       T* __restrict__ xh, float2* __restrict__ sx) {
  pdl_wait();
  pdl_trigger();
  if (!ctl->g_attempt) return;
  ktimer_begin(tslot(p.tm, TM_PRIMAL));
  const double tau = ctl->eta / ctl->omega;
  PDCS_GRID_LOOP(j, p.n) {
    primal_elem(p, tau, x, gty, xh, j);
    if (sx != nullptr) sx[j] = split_ff((double)xh[j]);
  }
  ktimer_end(tslot(p.tm, TM_PRIMAL));
}

// yhat = Proj_Y(y + sigma (h - G (2 xhat - x))), sigma = eta omega.
template <typename T>
PDCS_DEV void dual_elem(const Prob<T>& p, double sigma, const T* __restrict__ y,
                        const T* __restrict__ gxh, const T* __restrict__ gx, T* __restrict__ yh,
                        int64_t i) {
  double v = (double)y[i] + sigma * ((double)p.h[i] - 2.0 * (double)gxh[i] + (double)gx[i]);
  if (p.rk[i] == RK_NONNEG) v = fmax(v, 0.0);
  yh[i] = (T)v;
}

// The dual step of row i as the epilogue of the product G xhat (the product
// hands each row's value to this functor): stores (G xhat)_i, the dual update
// of dual_elem, and, when res is non-NULL, u = G xhat - h on the cone rows
// (the primal residual's argument, as res_prep_row), so the cone projections
// of yhat and of u can run as one launch.  sigma = eta omega of the attempt.
template <typename T>
struct DualOut {
  static constexpr int kMinBlocks = 6;  // resident CTAs per SM of the product (40 registers)
  Prob<T> p;
  const Ctl* ctl;
  const T* y;
  const T* gx;
  T* gxh;
  T* yh;
  double* res;
  struct Pre {
    double y, gx, h, sigma;
    uint8_t rk;
  };
  PDCS_DEV Pre pre(int64_t i) const {
    return Pre{(double)__ldg(y + i), (double)__ldg(gx + i), (double)__ldg(p.h + i),
               ctl->eta * ctl->omega, __ldg(p.rk + i)};
  }
  PDCS_DEV void operator()(int64_t i, double v, const Pre& q) const {
    const T g = (T)v;
    gxh[i] = g;
    double w = q.y + q.sigma * (q.h - 2.0 * (double)g + q.gx);
    if (q.rk == RK_NONNEG) w = fmax(w, 0.0);
    yh[i] = (T)w;
    if (res != nullptr && q.rk >= RK_SOC) res[i] = (double)g - q.h;
  }
};

// Dual step as a kernel of its own (products with short rows, where the
// product's epilogue would cost it occupancy); res as in DualOut.
template <typename T>
__global__ void __launch_bounds__(kEwThreads) k_dual(Prob<T> p, const Ctl* __restrict__ ctl,
                                                     const T* __restrict__ y,
                                                     const T* __restrict__ gxh,
                                                     const T* __restrict__ gx,
                                                     T* __restrict__ yh, double* __restrict__ res) {
  pdl_wait();
  pdl_trigger();
  if (!ctl->g_attempt) return;
  ktimer_begin(tslot(p.tm, TM_DUAL));
  const double sigma = ctl->eta * ctl->omega;
  PDCS_GRID_LOOP(i, p.m) {
    dual_elem(p, sigma, y, gxh, gx, yh, i);
    if (res != nullptr && p.rk[i] >= RK_SOC) res[i] = (double)gxh[i] - (double)p.h[i];
  }
  ktimer_end(tslot(p.tm, TM_DUAL));
}

// (kb1)^-0.3 and (kb1)^-0.6 for a count kb1 >= 2 (the exponents of Function
// 1).  A library FP64 pow is a long dependent chain of FP64 operations, and
// on this part every dependent FP64 operation of a thread costs ~64 cycles
// (the pair of pows took ~5.7 us of the step's critical path).  Instead: an
// FP32 seed (relative error ~1e-7), then two Newton steps in FP64 on
// f(p) = kb1^3 p^10 - 1, p <- p - p (q - 1) / (10 q) with q = kb1^3 p^10 and
// 1 / q expanded to second order around 1 (|q - 1| is a few 1e-6), which
// square the error twice: the result is within a few units in the last place
// of the exact power; (kb1)^-0.6 is its square.
PDCS_DEV void step_powers(double kb1, double& p3, double& p6) {
  double p = (double)powf((float)kb1, -0.3f);
  const double K = kb1 * kb1 * kb1;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double p2 = p * p, p4 = p2 * p2, p8 = p4 * p4;
    const double e = p8 * p2 * K - 1.0;
    p = p - 0.1 * p * (e * (1.0 - e));
  }
  p3 = p;
  p6 = p * p;
}

// Step-size test of Function 1 (eq. adaptive_step_size) from the reduced
// ||dx||^2, ||dy||^2 and dy^T G dx.  kbar counts every attempt and is
// incremented before the exponents use (kbar + 1).  (Thread-0 logic shared by
// the grid-wide and the per-instance batched engines.)
PDCS_DEV void ctl_step_finalize(Ctl& c, double dx2, double dy2, double inter) {
  if (!c.adaptive_step) {
    // fixed step (use_adaptive_step_size_weight = 0): every attempt accepted
    c.kbar += 1;
    c.accepted = 1;
    c.eta = c.eta_hat = c.eta_acc = c.eta_fixed;
    c.g_accept = 1;
    return;
  }
  inter = fabs(inter);
  const double omega = c.omega, eta = c.eta;
  c.kbar += 1;
  const double kb1 = (double)(c.kbar + 1);
  const double num = 0.5 * (omega * dx2 + dy2 / omega);
  const double eta_bar = inter > 0.0 ? num / inter : INFINITY;
  double p3, p6;
  step_powers(kb1, p3, p6);
  const double eta_p = fmin((1.0 - p3) * eta_bar, (1.0 + p6) * eta);
  const int acc = eta < eta_bar ? 1 : 0;
  c.accepted = acc;
  if (acc) {
    c.eta_acc = eta;
    c.eta_hat = eta_p;
  }
  c.eta = eta_p;
  c.g_accept = acc;
  if (!(eta_p > 0.0) || !isfinite(eta_p)) {
    c.status = 8;  // numerical error
    c.g_accept = 0;
    c.g_attempt = 0;
  }
}

template <typename T>
__global__ void __launch_bounds__(kEwThreads) k_step(Prob<T> p, Ctl* __restrict__ ctl,
                                                     const T* __restrict__ x,
                                                     const T* __restrict__ xh,
                                                     const T* __restrict__ y,
                                                     const T* __restrict__ yh,
                                                     const T* __restrict__ gxh,
                                                     const T* __restrict__ gx,
                                                     double* __restrict__ part,
                                                     float2* __restrict__ sy) {
  pdl_wait();
  pdl_trigger();
  if (!ctl->g_attempt) return;
  ktimer_begin(tslot(p.tm, TM_STEP));
  __shared__ double sh[3 * kEwThreads + 3];
  double s[3] = {0.0, 0.0, 0.0};
  PDCS_GRID_LOOP(j, p.n) {
    const double d = (double)xh[j] - (double)x[j];
    s[0] += d * d;
  }
  PDCS_GRID_LOOP(i, p.m) {
    const double yv = (double)yh[i];
    const double d = yv - (double)y[i];
    s[1] += d * d;
    s[2] += d * ((double)gxh[i] - (double)gx[i]);
    if (sy != nullptr) sy[i] = split_ff(yv);  // shadow of yhat for G^T yhat (FP32 values)
  }
  block_sum<3>(s, sh);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) part[blockIdx.x * 3 + k] = s[k];
  }
  ktimer_end(tslot(p.tm, TM_STEP));
  if (!last_block_done(&ctl->cnt[CNT_STEP])) return;
  double S3[3];
  cta_reduce_sums<3>(part, gridDim.x, 3, S3, sh);
  if (threadIdx.x != 0) return;
  ctl->cnt[CNT_STEP] = 0u;
  ctl_step_finalize(*ctl, S3[0], S3[1], S3[2]);
}

// ------------------------------------------------------------- cone kernels
PDCS_DEV double cone_scale(const double* d, int64_t i, int inv) {
  if (d == nullptr) return 1.0;
  return inv ? 1.0 / d[i] : d[i];
}

// e = d or 1/d (inv) or 1 (d == NULL) for the 3-block at s, and ie = 1 / e;
// dinv, when given, holds the reciprocals 1 / d (else one division per element).
PDCS_DEV void cone_scale_pair(const double* d, const double* dinv, int64_t s, int inv,
                              double (&e)[3], double (&ie)[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (d == nullptr) { e[k] = ie[k] = 1.0; continue; }
    const double di = d[s + k], r = dinv ? dinv[s + k] : 1.0 / di;
    e[k] = inv ? r : di;
    ie[k] = inv ? di : r;
  }
}

// Exponential-cone blocks: one thread per 3-vector.  Target cone diag(e) K' with
// e = d or 1/d (inv) and K' = K_exp or K_exp^* (is_dual_exp[b] xor dual).
// blockIdx.y selects one of two vectors (each with its own gate).
PDCS_DEV bool gate_on(const int* g) { return g == nullptr || *g != 0; }

// Exponential-cone blocks, one thread per block.  flip1: vector 1 is
// projected onto the other family member (1 - dual) under the inverse scales
// (1 - inv), as for a dual iterate and a primal residual in one launch.
template <typename B>
__global__ void __launch_bounds__(128, 6) k_cone_exp(B* v0, B* v1, const int64_t* __restrict__ starts,
                           const uint8_t* __restrict__ isd, int64_t count,
                           const double* __restrict__ d, const double* __restrict__ dinv, int inv,
                           int dual, int flip1,
                           const int* __restrict__ gate0, const int* __restrict__ gate1,
                           KTimer* tm) {
  pdl_wait();
  pdl_trigger();
  B* v = blockIdx.y == 0 ? v0 : v1;
  if (flip1 && blockIdx.y == 1) {
    inv = 1 - inv;
    dual = 1 - dual;
  }
  const bool on = gate_on(blockIdx.y == 0 ? gate0 : gate1);
  if (!gate_on(gate0) && (gridDim.y == 1 || !gate_on(gate1))) return;  // whole launch idle
  ktimer_begin(tm);
  __shared__ float grid[kExpGrid];  // the scan abscissae, once per CTA
  for (int i = threadIdx.x; i < kExpGrid; i += blockDim.x) grid[i] = exp_grid_r(i);
  __syncthreads();
  if (on) PDCS_GRID_LOOP(b, count) {
    const int64_t s = starts[b];
    const double in[3] = {(double)v[s], (double)v[s + 1], (double)v[s + 2]};
    double e[3], ie[3];
    cone_scale_pair(d, dinv, s, inv, e, ie);
    double out[3];
    proj_exp_family(in, e, ie, (isd[b] != 0) != (dual != 0), out, grid);
    v[s] = (B)out[0];
    v[s + 1] = (B)out[1];
    v[s + 2] = (B)out[2];
  }
  ktimer_end(tm);
}

// Second-order-cone blocks: one CTA per block (dims <= NT * EPT); target cone
// diag(e) K_soc (self-dual, so the same routine serves both modes); flip1:
// vector 1 takes the inverse scales.
template <typename B, int NT, int EPT>
__global__ void __launch_bounds__(NT) k_cone_soc(B* v0, B* v1, const int64_t* __restrict__ starts,
                                                 const int32_t* __restrict__ dims,
                                                 const double* __restrict__ d, int inv, int flip1,
                                                 const int* __restrict__ gate0,
                                                 const int* __restrict__ gate1, KTimer* tm) {
  pdl_wait();
  pdl_trigger();
  B* v = blockIdx.y == 0 ? v0 : v1;
  if (flip1 && blockIdx.y == 1) inv = 1 - inv;
  if (!gate_on(gate0) && (gridDim.y == 1 || !gate_on(gate1))) return;  // whole launch idle
  ktimer_begin(tm);
  if (!gate_on(blockIdx.y == 0 ? gate0 : gate1)) {
    ktimer_end(tm);
    return;
  }
  __shared__ double sh[8 + 3 * NT + 3];
  const int64_t s = starts[blockIdx.x];
  const int dim = dims[blockIdx.x];
  double vv[EPT], ee[EPT];
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int i = threadIdx.x + k * NT;
    vv[k] = i < dim ? (double)v[s + i] : 0.0;
    ee[k] = i < dim ? cone_scale(d, s + i, inv) : 1.0;
  }
  soc_proj_cta<NT, EPT>(vv, ee, dim, sh);
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int i = threadIdx.x + k * NT;
    if (i < dim) v[s + i] = (B)vv[k];
  }
  ktimer_end(tm);
}

// --------------------------------------------------------- KKT statistics
// Copy u = G x - h (cone rows) and lambda = c - G^T y (cone columns) into the
// projection buffers, scaled and (optionally) unscaled.  blockIdx.y selects the
// point when two are processed together.
template <typename T>
PDCS_DEV void res_prep_row(const Prob<T>& p, const PointRef<T>& pt, const TmpRef& tr, int64_t i) {
  if (tr.tm != nullptr && p.rk[i] >= RK_SOC) {
    const double u = (double)pt.gx[i] - (double)p.h[i];
    tr.tm[i] = u;
    if (tr.um) tr.um[i] = u / p.d1[i];
  }
}

template <typename T>
PDCS_DEV void res_prep_col(const Prob<T>& p, const PointRef<T>& pt, const TmpRef& tr, int64_t j) {
  if (p.ck[j] >= CK_SOC) {
    const double l = (double)p.c[j] - (double)pt.gty[j];
    tr.tn[j] = l;
    if (tr.un) tr.un[j] = l / p.d2[j];
  }
}

template <typename T>
__global__ void __launch_bounds__(kEwThreads) k_res_prep(Prob<T> p, const int* __restrict__ gate,
                                                         PointRef<T> a, PointRef<T> b,
                                                         TmpRef ta, TmpRef tb) {
  pdl_wait();
  pdl_trigger();
  if (gate != nullptr && *gate == 0) return;
  ktimer_begin(tslot(p.tm, TM_RES_PREP));
  const PointRef<T> pt = blockIdx.y == 0 ? a : b;
  const TmpRef tr = blockIdx.y == 0 ? ta : tb;
  PDCS_GRID_LOOP(i, p.m) res_prep_row(p, pt, tr, i);
  PDCS_GRID_LOOP(j, p.n) res_prep_col(p, pt, tr, j);
  ktimer_end(tslot(p.tm, TM_RES_PREP));
}

// Projection onto Lambda_j (Sec. 1.1): {0}, R^-, R^+ or R by bound finiteness.
PDCS_DEV double proj_lambda(double lam, double lo, double hi) {
  const bool lf = isfinite(lo), uf = isfinite(hi);
  if (!lf && !uf) return 0.0;
  if (!lf) return fmin(lam, 0.0);
  if (!uf) return fmax(lam, 0.0);
  return lam;
}

// The square roots and quotients of the statistics, in six independent
// groups (k = 0..5) so that one point's groups can run on separate warps:
// q[0..1] abs_p, rel_p; q[2..3] abs_d, rel_d; q[4] rel_gap; q[5] inf_rel_p;
// q[6] inf_rel_d; q[7] inf_rel_gap.
constexpr int kStatGroups = 6;
PDCS_DEV void stats_quotients(const Ctl* ctl, int k, const double* s, const double* mx,
                              double* q) {
  switch (k) {
    case 0: q[0] = sqrt(s[0]); q[1] = q[0] / (1.0 + ctl->h1); break;
    case 1: q[2] = sqrt(s[1]); q[3] = q[2] / (1.0 + ctl->c1); break;
    case 2: q[4] = fabs(s[2] - s[3]) / (1.0 + fabs(s[2]) + fabs(s[3])); break;
    case 3: q[5] = mx[0] / (1.0 + fmax(ctl->hinf, fmax(mx[1], mx[2]))); break;
    case 4: q[6] = mx[3] / (1.0 + fmax(ctl->cinf, mx[4])); break;
    case 5: q[7] = fabs(s[2] - s[3]) / (1.0 + fmax(fabs(s[2]), fabs(s[3]))); break;
    default: break;
  }
}
static_assert(kEwThreads / 32 >= kStatGroups, "one warp per quotient group");

PDCS_DEV void finish_stats_q(PointStats& st, const double* s, const double* mx, const double* q) {
  st.abs_p = q[0];
  st.abs_d = q[2];
  st.pobj = s[2];
  st.dobj = s[3];
  st.u2 = s[4];
  st.lam2 = s[5];
  st.dx2 = s[6];
  st.dy2 = s[7];
  st.gap = fabs(st.pobj - st.dobj);
  st.rel_p = q[1];
  st.rel_d = q[3];
  st.rel_gap = q[4];
  st.max_err = fmax(st.rel_p, fmax(st.rel_d, st.rel_gap));
  st.inf_abs_p = mx[0];
  st.inf_abs_d = mx[3];
  st.inf_rel_p = q[5];
  st.inf_rel_d = q[6];
  st.inf_rel_gap = q[7];
  st.inf_max = fmax(st.inf_rel_p, fmax(st.inf_rel_d, st.inf_rel_gap));
}

PDCS_DEV void finish_stats(const Ctl* ctl, PointStats& st, const double* s, const double* mx) {
  double q[8];
  for (int k = 0; k < kStatGroups; ++k) stats_quotients(ctl, k, s, mx, q);
  finish_stats_q(st, s, mx, q);
}

// Reflection parameter beta (eq. adaptive_reflection) from maxErr.
PDCS_DEV void ctl_set_beta(Ctl& c) {
  const double me = c.st[0].max_err;
  double beta = me > 0.0 ? -0.1 * log10(me) + 0.2 : 1.0;
  beta = fmin(1.0, fmax(0.0, beta));
  if (isnan(me)) beta = 0.0;
  c.beta = beta;
}

// Statistics of one point from its reduced sums / maxima; slot 0 also sets the
// reflection parameter beta (eq. adaptive_reflection) from maxErr.
PDCS_DEV void ctl_stats_finalize(Ctl& c, int slot, const double* S, const double* M) {
  finish_stats(&c, c.st[slot], S, M);
  if (slot == 0) ctl_set_beta(c);
}

// Per-element contributions to the point statistics (row i / column j).
template <typename T, bool FULL>
PDCS_DEV void stats_row(const Prob<T>& p, const PointRef<T>& pt, const T* __restrict__ y0,
                        const TmpRef& tr, int64_t i, double (&s)[kStatSums],
                        double (&mx)[kStatMax]) {
  const double gx = (double)pt.gx[i], h = (double)p.h[i], y = (double)pt.y[i];
  const double u = gx - h;
  const uint8_t kd = p.rk[i];
  double P;
  if (kd == RK_FREE) P = 0.0;
  else if (kd == RK_NONNEG) P = fmax(u, 0.0);
  else P = tr.tm[i];
  const double r = u - P;
  s[0] += r * r;
  s[3] += h * y;
  s[4] += u * u;
  if (FULL) {
    const double d1 = p.d1[i];
    const double uu = u / d1;
    double Pu;
    if (kd == RK_FREE) Pu = 0.0;
    else if (kd == RK_NONNEG) Pu = fmax(uu, 0.0);
    else Pu = tr.um[i];
    mx[0] = fmax(mx[0], fabs(uu - Pu));
    mx[1] = fmax(mx[1], fabs(gx / d1));
    mx[2] = fmax(mx[2], fabs(Pu));
    if (y0) {
      const double dy = y - (double)y0[i];
      s[7] += dy * dy;
    }
  }
}

template <typename T, bool FULL>
PDCS_DEV void stats_col(const Prob<T>& p, const PointRef<T>& pt, const T* __restrict__ x0,
                        const TmpRef& tr, int64_t j, double (&s)[kStatSums],
                        double (&mx)[kStatMax]) {
  const double gty = (double)pt.gty[j], c = (double)p.c[j], x = (double)pt.x[j];
  const double lam = c - gty;
  const uint8_t kd = p.ck[j];
  double res;
  if (kd == CK_BOX) {
    const double lo = p.lo[j], hi = p.hi[j];
    res = lam - proj_lambda(lam, lo, hi);
    if (isfinite(lo)) s[3] += lo * fmax(lam, 0.0);
    if (isfinite(hi)) s[3] -= hi * fmax(-lam, 0.0);
  } else if (kd == CK_ZERO) {
    res = 0.0;
  } else if (kd == CK_NONNEG) {
    res = fmin(lam, 0.0);
  } else {
    res = lam - tr.tn[j];
  }
  s[1] += res * res;
  s[2] += c * x;
  s[5] += lam * lam;
  if (FULL) {
    const double d2 = p.d2[j];
    const double resu = kd >= CK_SOC ? lam / d2 - tr.un[j] : res / d2;
    mx[3] = fmax(mx[3], fabs(resu));
    mx[4] = fmax(mx[4], fabs(gty / d2));
    if (x0) {
      const double dx = x - (double)x0[j];
      s[6] += dx * dx;
    }
  }
}

// Residual norms (eqs. tolerance-3 / tolerance-2 on the rescaled problem and
// eq. PDCS_terminate_tolerance_rel on the unscaled one), objectives, and the
// norms needed by Algorithm 3 and Sec. 2.5, for one point.  slot 0 also sets
// the reflection parameter beta (eq. adaptive_reflection).
template <typename T, bool FULL>
__global__ void __launch_bounds__(kEwThreads) k_point_stats(Prob<T> p, Ctl* __restrict__ ctl,
                                                            const int* __restrict__ gate, int slot,
                                                            PointRef<T> pt, const T* __restrict__ x0,
                                                            const T* __restrict__ y0, TmpRef tr,
                                                            double* __restrict__ part) {
  pdl_wait();
  pdl_trigger();
  if (gate != nullptr && *gate == 0) return;
  KTimer* tmr = tslot(p.tm, slot == 0 ? TM_STATS_ATTEMPT : TM_STATS_CHECK);
  ktimer_begin(tmr);
  __shared__ double sh[kStatSums * kEwThreads + kStatSums];
  double s[kStatSums];
  double mx[kStatMax];
#pragma unroll
  for (int k = 0; k < kStatSums; ++k) s[k] = 0.0;
#pragma unroll
  for (int k = 0; k < kStatMax; ++k) mx[k] = 0.0;
  PDCS_GRID_LOOP(i, p.m) stats_row<T, FULL>(p, pt, y0, tr, i, s, mx);
  PDCS_GRID_LOOP(j, p.n) stats_col<T, FULL>(p, pt, x0, tr, j, s, mx);
  block_sum<kStatSums>(s, sh);
  block_max<kStatMax>(mx, sh);
  if (threadIdx.x == 0) {
    for (int k = 0; k < kStatSums; ++k) part[blockIdx.x * kStatK + k] = s[k];
    for (int k = 0; k < kStatMax; ++k) part[blockIdx.x * kStatK + kStatSums + k] = mx[k];
  }
  ktimer_end(tmr);
  if (!last_block_done(&ctl->cnt[CNT_STATS0 + slot])) return;
  double S[kStatSums], M[kStatMax];
  cta_reduce_parts<kStatSums, kStatMax>(part, gridDim.x, kStatK, S, M, sh);
  // the quotient groups on separate warps (schedulers), then thread 0
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0 && w < kStatGroups) stats_quotients(ctl, w, S, M, sh);
  __syncthreads();
  if (threadIdx.x != 0) return;
  ctl->cnt[CNT_STATS0 + slot] = 0u;
  finish_stats_q(ctl->st[slot], S, M, sh);
  if (slot == 0) ctl_set_beta(*ctl);
}

// ------------------------------------------------------- Halpern + average
// One coordinate of the reflected Halpern step for a vector v and its
// maintained product q (x with G^T y, or y with G x), plus the FP64 average
// sum, in the order of operations of Algorithm 1, a ((1 + beta) vh - beta v) +
// b v0: folding the scalars into two coefficients saves an FP64 operation but
// rounds differently, enough to move a free-running trajectory by ~1e-9
// within 40 iterations (the method amplifies rounding differences).
struct HalpernCoefs {
  double a, b, beta;
};

PDCS_HD HalpernCoefs halpern_coefs(double k, double beta) {
  return HalpernCoefs{(k + 1.0) / (k + 2.0), 1.0 / (k + 2.0), beta};
}

template <typename T>
PDCS_DEV void halpern_elem(const HalpernCoefs& hc, double eta, T* __restrict__ v,
                           T* __restrict__ q, const T* __restrict__ vh, const T* __restrict__ qh,
                           const T* __restrict__ v0, const T* __restrict__ q0,
                           double* __restrict__ vs, int64_t i) {
  const double a = hc.a, b = hc.b, beta = hc.beta;
  const T vn = (T)(a * ((1.0 + beta) * (double)vh[i] - beta * (double)v[i]) + b * (double)v0[i]);
  v[i] = vn;
  vs[i] += eta * (double)vn;
  q[i] = (T)(a * ((1.0 + beta) * (double)qh[i] - beta * (double)q[i]) + b * (double)q0[i]);
}

// Counters after an accepted step; sets the check / stop flags.
PDCS_DEV void ctl_halpern_finalize(Ctl& c, double eta, double beta, double* trace) {
  c.k += 1;
  c.iter += 1;
  c.wsum += eta;
  const long long it = c.iter;
  if (trace != nullptr && it <= c.trace_cap) {
    double* r = trace + (it - 1) * kTraceF;
    r[0] = (double)it; r[1] = (double)c.kbar; r[2] = (double)c.period; r[3] = eta;
    r[4] = c.eta_hat; r[5] = beta; r[6] = c.omega; r[7] = c.st[0].max_err;
    r[8] = 0.0; r[9] = -1.0; r[10] = 0.0; r[11] = NAN; r[12] = 0.0;
  }
  const bool kkt_due = c.kkt_restart && it % c.kkt_freq == 0;
  if (!isfinite(c.st[0].max_err)) {
    c.status = 8;
    c.g_attempt = 0;
  } else if (it % c.check_freq == 0 || kkt_due) {
    c.period_done = 1;
    c.g_attempt = 0;
    c.g_check = 1;
    c.chk_gap = c.gap_restart && it % c.check_freq == 0;
    c.chk_kkt = kkt_due;
    // infeasibility statistics need the previous check's candidate
    c.infeas_gate[0] = c.infeas_on && c.have_cand;
    c.infeas_gate[1] = c.infeas_on && c.have_cand && c.method == 0;
  } else if (it >= c.max_iter) {
    c.status = 1;
    c.g_attempt = 0;
  }
}

// Body terminator of the attempt loop: continue while the period needs more
// accepted iterations (bounded by guard_cap bodies per graph launch).
// (use_cond = 0: launched eagerly from the host, which reads g_attempt itself.)
PDCS_DEV int ctl_loop_ctl(Ctl& c) {
  c.guard += 1;
  c.bodies_a += 1;
  const int go = (c.status == kRunning && !c.period_done && c.guard < c.guard_cap);
  c.g_attempt = go;
  return go;
}

PDCS_DEV int ctl_period_begin(Ctl& c) {
  c.guard = 0;
  const int go = (c.status == kRunning && !c.period_done);
  c.g_attempt = go;
  c.g_accept = 0;
  return go;
}

// The loop decision and, inside a graph, the WHILE node's condition.
PDCS_DEV void loop_ctl(Ctl& c, cudaGraphConditionalHandle h, int use_cond) {
  const int go = ctl_loop_ctl(c);
  if (use_cond) cudaGraphSetConditional(h, go ? 1u : 0u);
}

// z^{t,k+1} = (k+1)/(k+2) ((1+beta) zhat - beta z) + z^{t,0}/(k+2) (Algorithm
// 1), applied to (x, y) and, by linearity, to the maintained products G x and
// G^T y; the average accumulators add eta * z^{t,k+1} in FP64.  The kernel
// ends the attempt body: after the step (or at once for a rejected attempt)
// one thread takes the loop decision.
template <typename T>
__global__ void __launch_bounds__(kEwThreads) k_halpern(
    Prob<T> p, Ctl* __restrict__ ctl, T* __restrict__ x, T* __restrict__ y, T* __restrict__ gx,
    T* __restrict__ gty, const T* __restrict__ xh, const T* __restrict__ yh,
    const T* __restrict__ gxh, const T* __restrict__ gtyh, const T* __restrict__ x0,
    const T* __restrict__ y0, const T* __restrict__ gx0, const T* __restrict__ gty0,
    double* __restrict__ xs, double* __restrict__ ys, double* __restrict__ trace,
    cudaGraphConditionalHandle h, int use_cond) {
  pdl_wait();
  pdl_trigger();
  if (!ctl->g_accept) {
    // rejected attempt: only the loop decision
    if (blockIdx.x == 0 && threadIdx.x == 0) loop_ctl(*ctl, h, use_cond);
    return;
  }
  ktimer_begin(tslot(p.tm, TM_HALPERN));
  const double beta = ctl->beta, eta = ctl->eta_acc;
  const HalpernCoefs hc = halpern_coefs((double)ctl->k, beta);
  PDCS_GRID_LOOP(j, p.n) halpern_elem(hc, eta, x, gty, xh, gtyh, x0, gty0, xs, j);
  PDCS_GRID_LOOP(i, p.m) halpern_elem(hc, eta, y, gx, yh, gxh, y0, gx0, ys, i);
  ktimer_end(tslot(p.tm, TM_HALPERN));
  if (!last_block_done(&ctl->cnt[CNT_HALPERN])) return;
  if (threadIdx.x != 0) return;
  ctl->cnt[CNT_HALPERN] = 0u;
  ctl_halpern_finalize(*ctl, eta, beta, trace);
  loop_ctl(*ctl, h, use_cond);
}

__global__ void k_period_begin(Ctl* ctl, cudaGraphConditionalHandle h, int use_cond) {
  pdl_wait();
  pdl_trigger();
  const int go = ctl_period_begin(*ctl);
  if (use_cond) cudaGraphSetConditional(h, go ? 1u : 0u);
}

// ------------------------------------------------------------------ check
template <typename T>
__global__ void __launch_bounds__(kEwThreads) k_average(int64_t n, int64_t m, const Ctl* __restrict__ ctl,
                                                        const double* __restrict__ xs,
                                                        const double* __restrict__ ys,
                                                        T* __restrict__ xb, T* __restrict__ yb,
                                                        KTimer* tm) {
  pdl_wait();
  pdl_trigger();
  if (!ctl->g_check) return;
  ktimer_begin(tm);
  const double w = ctl->wsum;
  PDCS_GRID_LOOP(j, n) xb[j] = (T)(xs[j] / w);
  PDCS_GRID_LOOP(i, m) yb[i] = (T)(ys[i] / w);
  ktimer_end(tm);
}

// Algorithm 3 set-up for both candidates: r = ||z_c - z^{t,0}||_N, and the first
// trial t0 = r / sqrt(tau ||b1||^2 + sigma ||b2||^2) (the unconstrained step that
// reaches radius r).
PDCS_DEV int ctl_bisect_init(Ctl& cl) {
  int any = 0;
  const double tau = cl.eta_acc / cl.omega, sigma = cl.eta_acc * cl.omega;
  for (int c = 0; c < 2; ++c) {
    Bisect& b = cl.bs[c];
    b.phase = BS_DONE;
    b.active = 0;
    b.result = c == 0 ? 0.0 : INFINITY;
    b.k = 0;
    b.nb = 0;
    b.tau = tau;
    b.sigma = sigma;
    b.last_dot = 0.0;
    if (!cl.g_check) continue;
    if (c == 1 && cl.method != 0) continue;
    if (!cl.chk_gap) {
      b.result = NAN;  // KKT-criterion or termination-only check: no gap
      continue;
    }
    const PointStats& st = cl.st[1 + c];
    const double r = sqrt(st.dx2 / tau + st.dy2 / sigma);
    const double scale = sqrt(tau * st.lam2 + sigma * st.u2);
    b.r = r;
    b.result = 0.0;
    if (!(r > 0.0) || !(scale > 0.0)) continue;
    b.t = r / scale;
    b.tl = 0.0;
    b.tr = b.t;
    b.phase = BS_EXP;
    b.active = 1;
    any = 1;
  }
  cl.probes = 0;
  return any;
}

__global__ void k_bisect_init(Ctl* ctl, cudaGraphConditionalHandle h, int use_cond) {
  pdl_wait();
  pdl_trigger();
  const int any = ctl_bisect_init(*ctl);
  if (use_cond) cudaGraphSetConditional(h, any ? 1u : 0u);
}

PDCS_DEV double probe_t(const Bisect& b) { return b.phase == BS_EXP ? b.t : 0.5 * (b.tl + b.tr); }

template <typename T>
PDCS_DEV void probe_prep_col(const Prob<T>& p, const PointRef<T>& pt, double tt,
                             double* __restrict__ px, int64_t j) {
  const double b1 = (double)pt.gty[j] - (double)p.c[j];
  double v = (double)pt.x[j] + tt * b1;
  const uint8_t kd = p.ck[j];
  if (kd == CK_BOX) v = fmin(fmax(v, p.lo[j]), p.hi[j]);
  else if (kd == CK_ZERO) v = 0.0;
  else if (kd == CK_NONNEG) v = fmax(v, 0.0);
  px[j] = v;
}

template <typename T>
PDCS_DEV void probe_prep_row(const Prob<T>& p, const PointRef<T>& pt, double ts,
                             double* __restrict__ py, int64_t i) {
  const double b2 = (double)p.h[i] - (double)pt.gx[i];
  double v = (double)pt.y[i] + ts * b2;
  if (p.rk[i] == RK_NONNEG) v = fmax(v, 0.0);
  py[i] = v;
}

// Accumulates ||dx||^2, b1^T dx (column j) and ||dy||^2, b2^T dy (row i).
template <typename T>
PDCS_DEV void probe_sum_col(const Prob<T>& p, const PointRef<T>& pt, const double* __restrict__ px,
                            int64_t j, double (&s)[4]) {
  const double dx = px[j] - (double)pt.x[j];
  s[0] += dx * dx;
  s[2] += ((double)pt.gty[j] - (double)p.c[j]) * dx;
}

template <typename T>
PDCS_DEV void probe_sum_row(const Prob<T>& p, const PointRef<T>& pt, const double* __restrict__ py,
                            int64_t i, double (&s)[4]) {
  const double dy = py[i] - (double)pt.y[i];
  s[1] += dy * dy;
  s[3] += ((double)p.h[i] - (double)pt.gx[i]) * dy;
}

// z(t) = (Proj_X(x + t tau b1), Proj_Y(y + t sigma b2)), b = (G^T y - c, h - G x)
// (eq. compute_zt_2), elementwise part; blockIdx.y = candidate.
template <typename T>
__global__ void __launch_bounds__(kEwThreads) k_probe_prep(Prob<T> p, const Ctl* __restrict__ ctl,
                                                           PointRef<T> a, PointRef<T> bpt,
                                                           double* __restrict__ px0,
                                                           double* __restrict__ py0,
                                                           double* __restrict__ px1,
                                                           double* __restrict__ py1) {
  pdl_wait();
  pdl_trigger();
  const int c = blockIdx.y;
  const Bisect& bs = ctl->bs[c];
  if (!ctl->bs[0].active && !ctl->bs[1].active) return;  // whole launch idle
  KTimer* tm = tslot(p.tm, TM_PROBE_PREP);
  ktimer_begin(tm);
  if (!bs.active) {
    ktimer_end(tm);
    return;
  }
  const PointRef<T> pt = c == 0 ? a : bpt;
  double* px = c == 0 ? px0 : px1;
  double* py = c == 0 ? py0 : py1;
  const double t = probe_t(bs);
  const double tt = t * bs.tau, ts = t * bs.sigma;
  PDCS_GRID_LOOP(j, p.n) probe_prep_col(p, pt, tt, px, j);
  PDCS_GRID_LOOP(i, p.m) probe_prep_row(p, pt, ts, py, i);
  ktimer_end(tm);
}

// Advances the exponential search / bisection state machines of Algorithm 3
// for both candidates from the reduced sums SS[c] = (||dx||^2, ||dy||^2,
// b1^T dx, b2^T dy); returns whether any candidate still needs probes.
PDCS_DEV int ctl_probe_finalize(Ctl& c, const double (&SS)[2][4]) {
  int any = 0;
  for (int cc = 0; cc < 2; ++cc) {
    Bisect& b = c.bs[cc];
    if (!b.active) continue;
    const double* S = SS[cc];
    const double dist = sqrt(S[0] / b.tau + S[1] / b.sigma);
    b.last_dot = S[2] + S[3];
    if (b.phase == BS_EXP) {
      if (dist > b.r) {
        if (b.k == 0) { b.tl = 0.0; b.tr = b.t; }
        else { b.tl = 0.5 * b.t; b.tr = b.t; }
        b.phase = BS_BISECT;
      } else {
        b.t *= 2.0;
        b.k += 1;
        b.tl = 0.5 * b.t;
        b.tr = b.t;
        if (b.k >= 64) b.phase = BS_BISECT;
      }
    } else {
      const double tm = 0.5 * (b.tl + b.tr);
      if (dist < b.r) b.tl = tm; else b.tr = tm;
      b.nb += 1;
    }
    if (b.phase == BS_BISECT && (b.tr - b.tl <= c.bisect_tol * b.tr || b.nb >= 64)) {
      b.phase = BS_DONE;
      b.active = 0;
      b.result = b.last_dot / b.r;
    }
    any |= b.active;
  }
  c.probes += 1;
  c.bodies_b += 1;
  if (c.probes >= c.probe_cap) {
    for (int cc = 0; cc < 2; ++cc) {
      Bisect& b = c.bs[cc];
      if (b.active) { b.active = 0; b.phase = BS_DONE; b.result = b.last_dot / b.r; }
    }
    any = 0;
  }
  return any;
}


// ||z(t) - z||_N and b^T (z(t) - z) for both candidates; the last CTA advances
// the exponential search / bisection state machines of Algorithm 3.
template <typename T>
__global__ void __launch_bounds__(kEwThreads) k_probe_reduce(Prob<T> p, Ctl* __restrict__ ctl,
                                                             PointRef<T> a, PointRef<T> bpt,
                                                             const double* __restrict__ px0,
                                                             const double* __restrict__ py0,
                                                             const double* __restrict__ px1,
                                                             const double* __restrict__ py1,
                                                             double* __restrict__ part,
                                                             cudaGraphConditionalHandle h,
                                                             int use_cond) {
  pdl_wait();
  pdl_trigger();
  const int c = blockIdx.y;
  const Bisect& bs = ctl->bs[c];
  ktimer_begin(tslot(p.tm, TM_PROBE_REDUCE));
  __shared__ double sh[4 * kEwThreads + 4];
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  if (bs.active) {
    const PointRef<T> pt = c == 0 ? a : bpt;
    const double* px = c == 0 ? px0 : px1;
    const double* py = c == 0 ? py0 : py1;
    PDCS_GRID_LOOP(j, p.n) probe_sum_col(p, pt, px, j, s);
    PDCS_GRID_LOOP(i, p.m) probe_sum_row(p, pt, py, i, s);
  }
  block_sum<4>(s, sh);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) part[(blockIdx.y * gridDim.x + blockIdx.x) * 4 + k] = s[k];
  }
  ktimer_end(tslot(p.tm, TM_PROBE_REDUCE));
  if (!last_block_done(&ctl->cnt[CNT_PROBE])) return;
  double SS[2][4];
  for (int cc = 0; cc < 2; ++cc) {
    double S4[4];
    cta_reduce_sums<4>(part + (size_t)cc * gridDim.x * 4, gridDim.x, 4, S4, sh);
    for (int k = 0; k < 4; ++k) SS[cc][k] = S4[k];
  }
  if (threadIdx.x != 0) return;
  ctl->cnt[CNT_PROBE] = 0u;
  const int any = ctl_probe_finalize(*ctl, SS);
  if (use_cond) cudaGraphSetConditional(h, any ? 1u : 0u);
}

PDCS_DEV double kkt_w(double ep, double ed, double eg, double w) {
  return sqrt(w * w * ep * ep + ed * ed / (w * w) + eg * eg);
}

// Infeasibility tests of Sec. 3.2.3 on the candidate's (primal, dual) ratios:
// high accuracy on the ratio alone (3 / 5), low accuracy with the candidates'
// dual objective (resp. -c^T x) rising at each of the last kHist - 1 checks
// (2 / 4); 0 when no test fires.
PDCS_DEV bool hist_rising(const double* h, int n) {
  if (n < kHist) return false;
  for (int q = 1; q < kHist; ++q)
    if (!(h[q] > h[q - 1])) return false;
  return true;
}

PDCS_DEV int infeasibility_code(const Ctl& c, double pr, double dr) {
  if (pr < c.eps_ph) return 3;
  if (dr < c.eps_dh) return 5;
  if (pr < c.eps_pl && hist_rising(c.hist_d, c.n_hist)) return 2;
  if (dr < c.eps_dl && hist_rising(c.hist_p, c.n_hist)) return 4;
  return 0;
}

// GetRestartCandidate, termination, restart conditions, KKT_omega fallback,
// primal-weight update (Secs. 2.3, 2.5, 3.2.3).
PDCS_DEV void ctl_check_decide(Ctl& c, double* trace) {
  if (!c.g_check) return;
  const bool avg = c.method == 0;
  const double rho_h = c.bs[0].result;
  const double rho_a = avg ? c.bs[1].result : INFINITY;
  const double w = c.omega;
  // KKT_omega replaces every gap when one of them is negative or was not
  // computed (a KKT-criterion check)
  const bool fb = !(rho_h >= 0.0) || (avg && !(rho_a >= 0.0)) || (c.has_ref && !(c.ref_rho >= 0.0)) ||
                  (c.has_prev && !(c.prev_rho >= 0.0));
  const PointStats& s1 = c.st[1];
  const PointStats& s2 = c.st[2];
  const double m_h = fb ? kkt_w(s1.abs_p, s1.abs_d, s1.gap, w) : rho_h;
  const double m_a = avg ? (fb ? kkt_w(s2.abs_p, s2.abs_d, s2.gap, w) : rho_a) : INFINITY;
  const int cand = (m_h <= m_a) ? 0 : 1;
  const double val = cand ? m_a : m_h;
  const double rho_c = cand ? rho_a : rho_h;
  const PointStats& sc = c.st[1 + cand];
  const bool had_cand = c.have_cand != 0;
  c.cand = cand;
  c.have_cand = 1;
  c.chk_fb = fb ? 1 : 0;
  const long long it = c.iter;
  if (trace != nullptr && it >= 1 && it <= c.trace_cap) {
    double* r = trace + (it - 1) * kTraceF;
    r[8] = 1.0; r[9] = (double)cand; r[11] = val; r[12] = fb ? 1.0 : 0.0;
  }
  // objectives of the candidates of the last checks (infeasibility trend)
  if (c.n_hist == kHist) {
    for (int q = 0; q + 1 < kHist; ++q) { c.hist_d[q] = c.hist_d[q + 1]; c.hist_p[q] = c.hist_p[q + 1]; }
    c.n_hist -= 1;
  }
  c.hist_d[c.n_hist] = sc.dobj;
  c.hist_p[c.n_hist] = -sc.pobj;
  c.n_hist += 1;
  bool done = sc.inf_max <= c.rel_tol;
  if (c.require_abs) done = done && fmax(sc.inf_abs_p, fmax(sc.inf_abs_d, sc.gap)) <= c.abs_tol;
  c.g_restart = 0;
  if (done) { c.status = 0; return; }
  if (!isfinite(sc.inf_max)) { c.status = 8; return; }
  if (c.infeas_on && had_cand) {
    const int code = infeasibility_code(c, c.infeas[cand][0], c.infeas[cand][1]);
    if (code) { c.status = code; return; }
  }
  bool restart = false;
  if (c.adaptive_restart) {
    const bool cond3 = (double)c.k >= 0.223 * (double)c.kbar;
    if (!c.has_ref) {
      restart = cond3;
    } else {
      const double ref = fb ? kkt_w(c.ref_ep, c.ref_ed, c.ref_eg, w) : c.ref_rho;
      const bool crit = c.chk_gap || c.chk_kkt;  // conditions 1 and 2 need a criterion
      const bool c1 = crit && val <= 0.4 * ref;
      bool c2 = false;
      if (c.has_prev && crit) {
        const double pv = fb ? kkt_w(c.prev_ep, c.prev_ed, c.prev_eg, w) : c.prev_rho;
        c2 = val <= 0.8 * ref && val > pv;
      }
      restart = c1 || c2 || cond3;
    }
  }
  if (restart) {
    if (trace != nullptr && it >= 1 && it <= c.trace_cap) trace[(it - 1) * kTraceF + 10] = 1.0;
    const double dx = sqrt(sc.dx2), dy = sqrt(sc.dy2);
    double om = c.omega;
    if (dx > 1e-10 && dy > 1e-10) om = exp(0.5 * log(dy / dx) + 0.5 * log(om));
    if (om > 1e5 || om < 1e-5) om = c.omega0;
    c.omega = om;
    c.has_ref = 1;
    c.ref_rho = rho_c;
    c.ref_ep = sc.abs_p; c.ref_ed = sc.abs_d; c.ref_eg = sc.gap;
    c.has_prev = 0;
    c.period += 1;
    c.restarts += 1;
    c.k = 0;
    c.wsum = 0.0;
    c.g_restart = 1;
  } else {
    c.has_prev = 1;
    c.prev_rho = rho_c;
    c.prev_ep = sc.abs_p; c.prev_ed = sc.abs_d; c.prev_eg = sc.gap;
  }
}

__global__ void k_check_decide(Ctl* ctl, double* trace) {
  pdl_wait();
  pdl_trigger(); ctl_check_decide(*ctl, trace); }

// Keep the chosen candidate (the returned point) and, on restart, make it the
// new anchor and current iterate and clear the average.
// sx / sy (FP32-value mode, else NULL): on restart also the FP32 shadows of
// the new anchor for its products.
template <typename T>
__global__ void __launch_bounds__(kEwThreads) k_cand_copy(int64_t n, int64_t m, const Ctl* __restrict__ ctl,
                                                          PointRef<T> z, PointRef<T> zb, T* xc, T* yc,
                                                          T* gxc, T* gtyc, T* x0, T* y0, T* x, T* y,
                                                          double* xs, double* ys, float2* sx,
                                                          float2* sy, KTimer* tm) {
  pdl_wait();
  pdl_trigger();
  if (!ctl->g_check) return;
  ktimer_begin(tm);
  const PointRef<T> s = ctl->cand ? zb : z;
  const bool rs = ctl->g_restart != 0;
  PDCS_GRID_LOOP(j, n) {
    const T v = s.x[j];
    gtyc[j] = s.gty[j];
    xc[j] = v;
    if (rs) {
      x0[j] = v; x[j] = v; xs[j] = 0.0;
      if (sx != nullptr) sx[j] = split_ff((double)v);
    }
  }
  PDCS_GRID_LOOP(i, m) {
    const T v = s.y[i];
    gxc[i] = s.gx[i];
    yc[i] = v;
    if (rs) {
      y0[i] = v; y[i] = v; ys[i] = 0.0;
      if (sy != nullptr) sy[i] = split_ff((double)v);
    }
  }
  ktimer_end(tm);
}

template <typename T>
__global__ void __launch_bounds__(kEwThreads) k_copy_products(int64_t n, int64_t m, const int* __restrict__ gate,
                                                              const T* gx0, const T* gty0, T* gx, T* gty,
                                                              KTimer* tm) {
  pdl_wait();
  pdl_trigger();
  if (!*gate) return;
  ktimer_begin(tm);
  PDCS_GRID_LOOP(j, n) gty[j] = gty0[j];
  PDCS_GRID_LOOP(i, m) gx[i] = gx0[i];
  ktimer_end(tm);
}

PDCS_DEV void ctl_check_end(Ctl& c) {
  if (!c.g_check) return;
  c.period_done = 0;
  c.g_restart = 0;
  c.g_check = 0;
  c.infeas_gate[0] = c.infeas_gate[1] = 0;
  if (c.status == kRunning && c.iter >= c.max_iter) c.status = 1;
  c.g_attempt = c.status == kRunning;
}

__global__ void k_check_end(Ctl* ctl) {
  pdl_wait();
  pdl_trigger(); ctl_check_end(*ctl); }

// ------------------------------------------------ infeasibility statistics
// Sec. 3.2.3 infeasibility ratios for the change of restart candidate cidx
// (0: z, 1: zbar; blockIdx.y) since the previous check's candidate pc, in the
// unscaled variables: dx = D2 (x_c - x_pc), dy = D1 (y_c - y_pc), and by
// linearity of the carried products G dx = (Ghat dx~) / D1 and, for the
// homogeneous problem (c = 0), lambda = -G^T dy = -(Ghat^T dy~) / D2.
// The prep pass stores the parts that need cone projections onto the standard
// cones (done by the cone kernels in place): tm <- G dx (onto K_r), um <- dy
// (onto K_r^*) on cone rows; tn <- lambda (onto K_p^*), un <- dx (onto K_p)
// on cone columns.
template <typename T>
__global__ void __launch_bounds__(kEwThreads) k_infeas_prep(Prob<T> p, const Ctl* __restrict__ ctl,
                                                            PointRef<T> z, PointRef<T> zb,
                                                            PointRef<T> pc, TmpRef ta, TmpRef tb) {
  pdl_wait();
  pdl_trigger();
  const int cidx = blockIdx.y;
  if (!ctl->infeas_gate[cidx]) return;
  const PointRef<T> a = cidx == 0 ? z : zb;
  const TmpRef t = cidx == 0 ? ta : tb;
  PDCS_GRID_LOOP(i, p.m) {
    if (p.rk[i] < RK_SOC) continue;
    const double d1 = p.d1[i];
    t.tm[i] = ((double)a.gx[i] - (double)pc.gx[i]) / d1;
    t.um[i] = d1 * ((double)a.y[i] - (double)pc.y[i]);
  }
  PDCS_GRID_LOOP(j, p.n) {
    if (p.ck[j] < CK_SOC) continue;
    const double d2 = p.d2[j];
    t.tn[j] = -((double)a.gty[j] - (double)pc.gty[j]) / d2;
    t.un[j] = d2 * ((double)a.x[j] - (double)pc.x[j]);
  }
}

// Projection onto the recession cone of [lo, hi] (by bound finiteness).
PDCS_DEV double proj_recession(double v, double lo, double hi) {
  const bool lf = isfinite(lo), uf = isfinite(hi);
  if (lf && uf) return 0.0;
  if (lf) return fmax(v, 0.0);
  if (uf) return fmin(v, 0.0);
  return v;
}

constexpr int kInfS = 2, kInfM = 5, kInfK = kInfS + kInfM;

// Ratios of both candidates (after the cone projections of k_infeas_prep's
// vectors): primal = max(dual error of lambda, dual-cone violation of dy) /
// (h^T dy + l^T lambda_1^+ - u^T lambda_1^-), dual = max(|G dx - P(G dx)| /
// (1 + max(|G dx|, |P(G dx)|)), recession-cone violation of dx) / (-c^T dx),
// infinity norms; +inf when the denominator is not positive.
template <typename T>
__global__ void __launch_bounds__(kEwThreads) k_infeas_reduce(Prob<T> p, Ctl* __restrict__ ctl,
                                                              PointRef<T> z, PointRef<T> zb,
                                                              PointRef<T> pc, TmpRef ta, TmpRef tb,
                                                              double* __restrict__ part) {
  pdl_wait();
  pdl_trigger();
  if (!ctl->infeas_gate[0] && !ctl->infeas_gate[1]) return;  // uniform over the grid
  const int cidx = blockIdx.y;
  __shared__ double sh[kInfM * kEwThreads + kInfM];
  // sums: dual objective of dy, -c^T dx; maxima: dual-side violation,
  // |G dx - P(G dx)|, |G dx|, |P(G dx)|, recession violation of dx
  double s[kInfS] = {0.0, 0.0};
  double mx[kInfM] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (ctl->infeas_gate[cidx]) {
    const PointRef<T> a = cidx == 0 ? z : zb;
    const TmpRef t = cidx == 0 ? ta : tb;
    PDCS_GRID_LOOP(i, p.m) {
      const double d1 = p.d1[i];
      const double dyt = (double)a.y[i] - (double)pc.y[i];
      const double g = ((double)a.gx[i] - (double)pc.gx[i]) / d1;
      const double dy = d1 * dyt;
      const uint8_t kd = p.rk[i];
      double pg, ey;
      if (kd == RK_FREE) { pg = 0.0; ey = 0.0; }                 // {0} and its dual R
      else if (kd == RK_NONNEG) { pg = fmax(g, 0.0); ey = fmin(dy, 0.0); }
      else { pg = t.tm[i]; ey = dy - t.um[i]; }
      mx[0] = fmax(mx[0], fabs(ey));
      mx[1] = fmax(mx[1], fabs(g - pg));
      mx[2] = fmax(mx[2], fabs(g));
      mx[3] = fmax(mx[3], fabs(pg));
      s[0] += (double)p.h[i] * dyt;  // h^T dy = hhat^T dy~
    }
    PDCS_GRID_LOOP(j, p.n) {
      const double d2 = p.d2[j];
      const double dxt = (double)a.x[j] - (double)pc.x[j];
      const double lam = -((double)a.gty[j] - (double)pc.gty[j]) / d2;
      const double dx = d2 * dxt;
      const uint8_t kd = p.ck[j];
      double el, ex;
      if (kd == CK_BOX) {
        const double lo = p.lo[j] * d2, hi = p.hi[j] * d2;  // unscaled bounds
        el = lam - proj_lambda(lam, lo, hi);
        ex = dx - proj_recession(dx, lo, hi);
        if (isfinite(lo)) s[0] += lo * fmax(lam, 0.0);
        if (isfinite(hi)) s[0] -= hi * fmax(-lam, 0.0);
      } else if (kd == CK_ZERO) {
        el = 0.0;
        ex = dx;
      } else if (kd == CK_NONNEG) {
        el = fmin(lam, 0.0);
        ex = fmin(dx, 0.0);
      } else {
        el = lam - t.tn[j];
        ex = dx - t.un[j];
      }
      mx[0] = fmax(mx[0], fabs(el));
      mx[4] = fmax(mx[4], fabs(ex));
      s[1] -= (double)p.c[j] * dxt;  // -c^T dx = -chat^T dx~
    }
  }
  block_sum<kInfS>(s, sh);
  block_max<kInfM>(mx, sh);
  if (threadIdx.x == 0) {
    double* q = part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * kInfK;
    for (int k = 0; k < kInfS; ++k) q[k] = s[k];
    for (int k = 0; k < kInfM; ++k) q[kInfS + k] = mx[k];
  }
  if (!last_block_done(&ctl->cnt[CNT_INFEAS])) return;
  double R[2][2];
  for (int cc = 0; cc < 2; ++cc) {
    double S[kInfS], M[kInfM];
    cta_reduce_parts<kInfS, kInfM>(part + (size_t)cc * gridDim.x * kInfK, gridDim.x, kInfK, S, M, sh);
    const double num_d = fmax(M[1] / (1.0 + fmax(M[2], M[3])), M[4]);
    R[cc][0] = S[0] > 0.0 ? M[0] / S[0] : INFINITY;
    R[cc][1] = S[1] > 0.0 ? num_d / S[1] : INFINITY;
  }
  if (threadIdx.x != 0) return;
  ctl->cnt[CNT_INFEAS] = 0u;
  for (int cc = 0; cc < 2; ++cc) {
    ctl->infeas[cc][0] = ctl->infeas_gate[cc] ? R[cc][0] : INFINITY;
    ctl->infeas[cc][1] = ctl->infeas_gate[cc] ? R[cc][1] : INFINITY;
  }
}

// ----------------------------------------------------------- init / output
template <typename T>
__global__ void k_fill(T* v, int64_t n, double val) {
  PDCS_GRID_LOOP(i, n) v[i] = (T)val;
}

template <typename S, typename D>
__global__ void k_convert(const S* in, D* out, int64_t n) {
  PDCS_GRID_LOOP(i, n) out[i] = (D)in[i];
}

// Warm start (original variables, RSOC rotation already undone) -> solver
// variables: divide by the scaling (Algorithm 2).
template <typename T>
__global__ void k_warm(T* out, const double* in, const double* d, int64_t n) {
  PDCS_GRID_LOOP(i, n) out[i] = (T)(in[i] / d[i]);
}

// Unscale the returned point: x = D2 xt, y = D1 yt, s = (G xt - hhat) / D1.
template <typename T>
__global__ void k_unscale(Prob<T> p, const T* xt, const T* yt, const T* gxt, double* x, double* y,
                          double* s) {
  PDCS_GRID_LOOP(j, p.n) x[j] = p.d2[j] * (double)xt[j];
  PDCS_GRID_LOOP(i, p.m) {
    y[i] = p.d1[i] * (double)yt[i];
    s[i] = ((double)gxt[i] - (double)p.h[i]) / p.d1[i];
  }
}

}  // namespace pdcs

namespace pdcs {

// Largest grid of the cooperative kernels (partials are read in one sweep).
constexpr int kMaxGridParts = 512;

// ------------------------------------------------- grid-wide SOC projection
// For second-order-cone blocks too large for one CTA (e.g. the single block of
// dimension k + n + 2 of a factor-model portfolio), the same root-finding as
// soc_proj_cta runs over the whole grid: each Newton step is a grid-wide sum
// (per-CTA partials, a grid barrier, then every CTA adds the partials in the
// same fixed order, so all CTAs take identical decisions).  The kernel is
// launched cooperatively, so all CTAs are resident; each barrier wait is still
// bounded and, if it ever gives up, sets *err and lets the kernel finish.
struct GridSync {
  // arrival counter, zeroed once at set-up and never reset: a barrier is the
  // next multiple of gridDim.x arrivals (every launch using the counter has
  // the same grid size, so arrivals fall into whole generations)
  unsigned long long* count;
  int* err;
};

PDCS_DEV void grid_sync(const GridSync& gs) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long g = gridDim.x;
    const unsigned long long target = (atomicAdd(gs.count, 1ull) / g + 1) * g;
    unsigned long long spins = 0;
    while (true) {
      unsigned long long v;
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(gs.count) : "memory");
      if (v >= target) break;
      __nanosleep(64);
      if (++spins > (1ull << 24)) { atomicExch(gs.err, 1); break; }
    }
    __threadfence();
  }
  __syncthreads();
}

// Grid-wide reductions of the cooperative SOC kernel.  Each pass stages its
// values per CTA in a partial buffer, crosses one grid barrier, and then the
// CTA adds the partials of all CTAs in a fixed order (so every CTA obtains
// bit-identical totals and takes identical decisions).
//
// Buffer layout (G = gridDim.x): two alternating halves of kSgHalf * G
// doubles (a CTA that runs ahead never overwrites partials another CTA is
// still reading); each half holds 8 FP64 slots x G, slot-major (so the reads
// after the barrier coalesce), followed by kSgF32Slots FP32 slots x G.  FP64
// slots < KS are sums, the others maxima of non-negative values (integer
// bit-pattern maxima).
constexpr int kSgProbes = 8;                     // probe points of pass 0 per vector
constexpr int kSgF32Slots = 3 * kSgProbes * 2;   // FP32 slots (up to two vectors)
constexpr int kSgHalf = 8 + kSgF32Slots / 2;     // doubles per CTA per half

struct GridPart {
  double* d;
  float* f;
};

PDCS_DEV GridPart grid_part(double* base, int flip) {
  double* h = base + (size_t)flip * kSgHalf * gridDim.x;
  return GridPart{h, reinterpret_cast<float*>(h + 8 * (size_t)gridDim.x)};
}

// CTA partials of K FP64 values: staged in shared memory, warp k adds value k.
template <int K>
PDCS_DEV void cta_rows_f64(const double (&v)[K], int KS, unsigned mask, double* red, GridPart p) {
  const int nt = blockDim.x;
#pragma unroll
  for (int k = 0; k < K; ++k) red[k * nt + threadIdx.x] = v[k];
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w < K && ((mask >> w) & 1u)) {
    const double* r = red + w * nt;
    if (w < KS) {
      double s = 0.0;
      for (int t = lane; t < nt; t += 32) s += r[t];
      s = warp_sum(s);
      if (lane == 0) p.d[(size_t)w * gridDim.x + blockIdx.x] = s;
    } else {
      long long s = 0;
      for (int t = lane; t < nt; t += 32) s = max(s, __double_as_longlong(r[t]));
      s = warp_max_bits(s);
      if (lane == 0) p.d[(size_t)w * gridDim.x + blockIdx.x] = __longlong_as_double(s);
    }
  }
}

PDCS_DEV float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// CTA partials of K FP32 sums (warp butterflies, then warp k adds the warps'
// value k); redf holds 32 * K floats.
template <int K>
PDCS_DEV void cta_rows_f32(const float (&v)[K], unsigned mask, float* redf, GridPart p) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (!((mask >> k) & 1u)) continue;
    const float s = warp_sum_f(v[k]);
    if (lane == 0) redf[w * K + k] = s;
  }
  __syncthreads();
  if (w < K && ((mask >> w) & 1u)) {
    float s = lane < nw ? redf[lane * K + w] : 0.0f;
    s = warp_sum_f(s);
    if (lane == 0) p.f[(size_t)w * gridDim.x + blockIdx.x] = s;
  }
}

// After the barrier: warp k < K totals slot k (lane l takes CTAs l, l + 32,
// ... with all loads issued together, then a fixed butterfly).  FP64 totals go
// to out, FP32 ones (slots in f32mask) to outf, not widened (the FP64 pipe is
// scarce).
PDCS_DEV void grid_totals(GridPart p, int K, int KS, unsigned f32mask, double* out, float* outf) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned G = gridDim.x;
  if (w < K) {
    if ((f32mask >> w) & 1u) {
      const float* src = p.f + (size_t)w * G;
      float buf[kMaxGridParts / 32];
#pragma unroll
      for (int j = 0; j < kMaxGridParts / 32; ++j) {
        const unsigned b = lane + 32u * j;
        buf[j] = b < G ? __ldcg(src + b) : 0.0f;
      }
      float s = 0.0f;
#pragma unroll
      for (int j = 0; j < kMaxGridParts / 32; ++j) s += buf[j];
      s = warp_sum_f(s);
      if (lane == 0) outf[w] = s;
    } else {
      const double* src = p.d + (size_t)w * G;
      if (w >= KS) {
        long long buf[kMaxGridParts / 32];
#pragma unroll
        for (int j = 0; j < kMaxGridParts / 32; ++j) {
          const unsigned b = lane + 32u * j;
          buf[j] = b < G ? __double_as_longlong(__ldcg(src + b)) : 0ll;
        }
        long long s = 0;
#pragma unroll
        for (int j = 0; j < kMaxGridParts / 32; ++j) s = max(s, buf[j]);
        s = warp_max_bits(s);
        if (lane == 0) out[w] = __longlong_as_double(s);
      } else {
        double buf[kMaxGridParts / 32];
#pragma unroll
        for (int j = 0; j < kMaxGridParts / 32; ++j) {
          const unsigned b = lane + 32u * j;
          buf[j] = b < G ? __ldcg(src + b) : 0.0;
        }
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < kMaxGridParts / 32; ++j) s += buf[j];
        s = warp_sum(s);
        if (lane == 0) out[w] = s;
      }
    }
  }
  __syncthreads();
}

// After the pass-0 barrier: the FP32 totals of the S probe slots, warp w
// taking slots w, w + nwarps, ... (at most kSgSlotsPerWarp; lane l adds CTAs
// l, l + 32, ... and a fixed butterfly follows, as grid_totals), with the
// loads of all its slots issued before the first add, so that one L2 round
// trip serves them; then the FP64 totals (warps < K64, grid_totals).
constexpr int kSgSlotsPerWarp = 3;
static_assert(kSgSlotsPerWarp * (512 / 32) >= kSgF32Slots, "probe slots per warp");
PDCS_DEV void grid_totals_pass0(GridPart p, int K64, int KS, int S, double* out, float* outp) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const unsigned G = gridDim.x;
  float acc[kSgSlotsPerWarp];
#pragma unroll
  for (int r = 0; r < kSgSlotsPerWarp; ++r) {
    const int sl = w + r * nw;
    float a = 0.0f;
    if (sl < S) {
      const float* src = p.f + (size_t)sl * G;
#pragma unroll
      for (int j = 0; j < kMaxGridParts / 32; ++j) {
        const unsigned bb = lane + 32u * j;
        if (bb < G) a += __ldcg(src + bb);
      }
    }
    acc[r] = a;
  }
#pragma unroll
  for (int r = 0; r < kSgSlotsPerWarp; ++r) {
    const int sl = w + r * nw;
    const float sm = warp_sum_f(acc[r]);
    if (lane == 0 && sl < S) outp[sl] = sm;
  }
  grid_totals(p, K64, KS, 0u, out, nullptr);  // ends with __syncthreads
}

// One element's terms of the FP64 phase (the sums soc_secular_terms forms,
// for a = vv^2 b): f0 and f1 in FP64; f2 in FP32, since it only enters the
// second-order term of a Halley step, multiplied by F, which vanishes at the
// root (an FP32 f2 changes a step of size d by ~1e-7 |F F''| / F'^2 of d).
// vv is the normalised tail element and b its squared scale.  a r^2 is
// formed as (vv r)^2 b, and the FP32 copies come from the integer pipes:
// 10 FP64 operations per element instead of 14 (the phase is bound by them).
PDCS_DEV void soc_terms_f64(bool pos, double vv, double b, double x, double& f0, double& f1,
                            float& f2) {
  const double r = pos ? rcp_nr(fma(2.0, x, b)) : rcp_nr(fma(b, x, 1.0));
  const double tv = vv * r;
  const double ar2 = tv * tv * b;
  f0 += ar2;
  const float rf = f32_trunc(r), af = f32_trunc(ar2);
  if (pos) {
    f1 = fma(ar2, r, f1);
    f2 = fmaf(af * rf, rf, f2);
  } else {
    const float bf = f32_trunc(b);
    f1 = fma(ar2 * b, r, f1);
    f2 = fmaf(af * bf * bf * rf, rf, f2);
  }
}

// Per-vector scalar state of the grid-wide SOC root-finding.  Warp 0 of every
// CTA updates it from the same grid totals, so all copies agree; the other
// threads only read it (xf, pos and esh spare them FP64 instructions).
struct SocGridVec {
  double x, lo, hi, top, sc, c0, e02, v0h, w, mu2;  // FP64 phase and writes
  float xf, lof, hif, topf, c0f, e02f;              // probes and FP32 phase
  int pos, esh, mode, it;
};
enum : int {
  SG_DONE = 0,      // nothing (left) to do for this vector
  SG_ZERO_HEAD,     // v0 == 0: one pass for the norm of the new tail
  SG_F32,           // root-finding, per-element terms in FP32
  SG_F64,           // root-finding, per-element terms in FP64 (polish)
  SG_WRITE_ZERO,    // write: polar case
  SG_WRITE_ZH,      // write: v0 == 0 case
  SG_WRITE          // write: general case
};

// Thresholds of the two phases: the FP32 phase hands over once a Halley step
// is below kSgF32Tol times the distance of x to the ends of its interval (or
// after kSgF32Max passes); the FP64 phase stops after a step below kSgF64Tol
// of that distance: Halley's cubic convergence leaves an error of order
// (1e-4)^3 of the distance after such a step, far below what the FP64 sums
// resolve.  The FP32 phase only has to bring x within reach of that: after an
// FP32 step below 5e-2 of the distance the error is of order 1e-4 of it, and
// further FP32 steps mostly chase the rounding of the FP32 sums.  Measured
// on the portfolio (passes per two-vector launch, FP32 + FP64): 1e-5 gave
// 4.7 + 2.2, 1e-2 gave 1.2 + 1.7, 5e-2 gives 1.1 + 1.2.
constexpr double kSgF32Tol = 5e-2;
constexpr int kSgF32Max = 40;
constexpr double kSgF64Tol = 1e-4;
constexpr int kSgF64Max = 200;
// Elements per thread held in registers across passes (the rest re-read; the
// pass-0 probes need every element of the CTA in a slot).
constexpr int kSgSlots = 2;
// Probe abscissae: x_j = top / (1 + exp(-u_j)), u_j evenly spaced in
// [-kSgProbeU, kSgProbeU] (logit scale, so both ends of (0, top) are covered).
constexpr float kSgProbeU = 12.0f;

// Probe j of an interval (0, topf), in FP32 (every thread computes it the same way).
PDCS_DEV float sg_probe_x(float topf, int j) {
  const float u = -kSgProbeU + 2.0f * kSgProbeU * ((float)j + 0.5f) / (float)kSgProbes;
  return topf / (1.0f + expf(-u));
}

// Projection of the blocks (starts[b], dims[b]) of NV vectors onto
// diag(e) K_soc, given the squared scales b_i = e_i^2 of each block (head
// included) and their reciprocals (bq, bqi at offs[b]; NULL: e = 1).  With
// FLIP1 the second vector is projected onto diag(1/e) K_soc instead (its
// squared scales are bqi and their reciprocals bq), so a dual iterate and a
// primal residual share one launch and its barriers.  part
// needs 2 * kSgHalf * gridDim.x doubles.  CTA c owns the tail elements 1 + c * chunk ... of each block.
//
// Root-finding (the secular equation and Halley steps of soc_proj_cta):
//  * pass 0 adds, besides the norms that decide inside / polar, the FP32
//    element sums at kSgProbes fixed abscissae of (0, top); their signs
//    bracket the root and the best of their Halley steps starts
//  * an FP32 phase whose per-element terms, CTA sums and grid sums are all
//    FP32 narrows it down
//  * an FP64 phase (bracket reset to the whole interval) polishes it.
// The tail is normalised by 2^-E, E the binary exponent of max |v| (exact, and
// free in the integer conversions).  The NV vectors advance through the same
// passes, so they share the barriers.
// Squared scales of vector q: slot k (FP64, FP32) and element i from memory.
#define SG_BD(q, k) ((FLIP1 && (q) == 1) ? bc1[FLIP1 ? (k) : 0] : bc[k])
#define SG_BF(q, k) ((FLIP1 && (q) == 1) ? bfc1[FLIP1 ? (k) : 0] : bfc[k])
#define SG_BM(q, i) (((FLIP1 && (q) == 1) ? bbi : bb) ? ((FLIP1 && (q) == 1) ? bbi : bb)[i] : 1.0)
template <typename B, int NV, bool FLIP1>
__global__ void __launch_bounds__(512, 2) k_cone_soc_grid(
    B* v0, B* v1, const int64_t* __restrict__ starts, const int64_t* __restrict__ dims,
    const int64_t* __restrict__ offs, int nblocks, const double* __restrict__ bq,
    const double* __restrict__ bqi, const int* __restrict__ gate0,
    const int* __restrict__ gate1, double* __restrict__ part, GridSync gs, KTimer* tm) {
  pdl_wait();
  pdl_trigger();
  constexpr int K = 3 * NV;
  constexpr int RC = kSgSlots;
  constexpr int PS = 3 * kSgProbes;  // probe sums per vector
  __shared__ double red[K * 512];
  __shared__ float redf[32 * K];
  __shared__ float pa[RC * 512], pb[RC * 512];
  __shared__ float pred[16 * PS];
  __shared__ float ptot[NV * PS];
  __shared__ double tot[8];
  __shared__ float totf[8];
  __shared__ SocGridVec sv[NV];
  // the first block's table entries load together with the gates
  int64_t s = starts[0], dim = dims[0], o = offs[0];
  bool act[NV];
  act[0] = gate_on(gate0);
  if (NV > 1) act[NV - 1] = gate_on(gate1);
  bool any_act = false;
#pragma unroll
  for (int q = 0; q < NV; ++q) any_act |= act[q];
  if (!any_act) return;  // whole launch idle (gates are uniform)
  ktimer_begin(tm);
  B* vp[NV];
  vp[0] = v0;
  if (NV > 1) vp[NV - 1] = v1;
  int flip = 0;
  const int t = threadIdx.x, nt = blockDim.x, w = t >> 5, lane = t & 31;
  for (int blk = 0; blk < nblocks; ++blk) {
    if (blk > 0) {
      s = starts[blk];
      dim = dims[blk];
      o = offs[blk];
    }
    const double* bb = bq ? bq + o : nullptr;
    const double* bbi = bqi ? bqi + o : nullptr;
    const int64_t chunk = (dim - 1 + gridDim.x - 1) / gridDim.x;
    const int64_t cbeg = 1 + (int64_t)blockIdx.x * chunk;
    const int64_t cend = min(dim, cbeg + chunk);
    const bool probes_ok = chunk <= (int64_t)RC * nt;  // every element in a slot
    // ---- pass 0: sum (v/e)^2, sum (e v)^2 and max |v| of each tail (FP64),
    // and the FP32 probe sums; the slots' v and b stay in registers
    double bc[RC];
    float bfc[RC];
    double bc1[FLIP1 ? RC : 1];  // vector 1's b_i (FLIP1: 1 / vector 0's)
    float bfc1[FLIP1 ? RC : 1];
    double vc[NV][RC];
    float afc[NV][RC];
    double v0h[NV];
    double acc[2 * NV];
    long long amx[NV];
    const double b0 = bb ? bb[0] : 1.0;  // the head's squared scale
    const double b0i = FLIP1 ? (bbi ? bbi[0] : 1.0) : b0;  // vector 1's, FLIP1
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      acc[2 * q] = 0.0;
      acc[2 * q + 1] = 0.0;
      v0h[q] = act[q] ? (double)vp[q][s] : 0.0;
      amx[q] = __double_as_longlong(v0h[q]) & 0x7fffffffffffffffll;
    }
#pragma unroll
    for (int k = 0; k < RC; ++k) {
      const int64_t i = cbeg + t + k * nt;
      const bool in = i < cend;
      const double b = in && bb ? bb[i] : 1.0, bi = in && bbi ? bbi[i] : 1.0;
      if (FLIP1) {
        bc1[k] = bi;
        bfc1[k] = f32_trunc(bi);
      }
      bc[k] = b;
      bfc[k] = f32_trunc(b);
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const double vi = in && act[q] ? (double)vp[q][s + i] : 0.0;
        vc[q][k] = vi;
        const double v2 = vi * vi;
        const bool fl = FLIP1 && q == 1;
        acc[2 * q] = fma(v2, fl ? b : bi, acc[2 * q]);
        acc[2 * q + 1] = fma(v2, fl ? bi : b, acc[2 * q + 1]);
        amx[q] = max(amx[q], __double_as_longlong(vi) & 0x7fffffffffffffffll);
      }
    }
    for (int64_t i = cbeg + t + RC * nt; i < cend; i += nt) {
      const double b = bb ? bb[i] : 1.0, bi = bbi ? bbi[i] : 1.0;
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        if (!act[q]) continue;
        const double vi = (double)vp[q][s + i], v2 = vi * vi;
        const bool fl = FLIP1 && q == 1;
        acc[2 * q] = fma(v2, fl ? b : bi, acc[2 * q]);
        acc[2 * q + 1] = fma(v2, fl ? bi : b, acc[2 * q + 1]);
        amx[q] = max(amx[q], __double_as_longlong(vi) & 0x7fffffffffffffffll);
      }
    }
    const GridPart gp0 = grid_part(part, flip);
    // probes: thread t evaluates probe t % kSgProbes over elements
    // t / kSgProbes, + nt / kSgProbes, ... of the CTA (unnormalised FP32
    // terms; the root does not depend on the scale)
    const float b0f = f32_trunc(b0), b0f1 = FLIP1 ? f32_trunc(b0i) : b0f;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      if (!act[q] || !probes_ok) continue;  // uniform
      const bool posq = __double_as_longlong(v0h[q]) > 0ll;
      const float hf = (FLIP1 && q == 1) ? b0f1 : b0f;
      const float topf = posq ? 0.5f * hf : __frcp_rn(hf);
#pragma unroll
      for (int k = 0; k < RC; ++k) {
        const float vf = f32_trunc(vc[q][k]);
        pa[t + k * nt] = vf * vf * SG_BF(q, k);
        pb[t + k * nt] = SG_BF(q, k);
      }
      __syncthreads();
      const int j = t % kSgProbes;
      const float xj = sg_probe_x(topf, j);
      float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f;
      const int nel = (int)(cend - cbeg);
      for (int e = t / kSgProbes; e < nel; e += nt / kSgProbes) {
        const float b = pb[e], a = pa[e];
        const float r = posq ? __frcp_rn(fmaf(2.0f, xj, b)) : __frcp_rn(fmaf(b, xj, 1.0f));
        const float ar2 = a * r * r;
        p0 += ar2;
        p1 += posq ? ar2 * r : ar2 * b * r;
        p2 += posq ? ar2 * r * r : ar2 * b * b * r * r;
      }
      // lanes with equal t % kSgProbes: butterflies over the other lane bits
#pragma unroll
      for (int off = kSgProbes; off < 32; off <<= 1) {
        p0 += __shfl_xor_sync(0xffffffffu, p0, off);
        p1 += __shfl_xor_sync(0xffffffffu, p1, off);
        p2 += __shfl_xor_sync(0xffffffffu, p2, off);
      }
      if (lane < kSgProbes) {
        pred[w * PS + 3 * lane] = p0;
        pred[w * PS + 3 * lane + 1] = p1;
        pred[w * PS + 3 * lane + 2] = p2;
      }
      __syncthreads();
      if (t < PS) {
        float a = 0.0f;
        for (int ww = 0; ww < (nt >> 5); ++ww) a += pred[ww * PS + t];
        gp0.f[(size_t)(q * PS + t) * gridDim.x + blockIdx.x] = a;
      }
    }
    {
      double r0[K];
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        r0[2 * q] = acc[2 * q];
        r0[2 * q + 1] = acc[2 * q + 1];
        r0[2 * NV + q] = __longlong_as_double(amx[q]);
      }
      cta_rows_f64<K>(r0, 2 * NV, (1u << K) - 1u, red, gp0);
      grid_sync(gs);
      grid_totals_pass0(gp0, K, 2 * NV, probes_ok ? NV * PS : 0, tot, ptot);
      flip ^= 1;
    }
    // one warp per vector, so that the vectors' scalar work runs on separate
    // schedulers (the same code one warp would run for each in turn)
    if (w < NV) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        if (q != w) continue;  // warp-uniform
        SocGridVec& g = sv[q];
        // e0^2 is the head's precomputed squared scale (exactly e0 * e0)
        const double e02 = (FLIP1 && q == 1) ? b0i : b0;
        if (lane == 0) {
          g.mode = SG_DONE;
          g.it = 0;
          g.esh = 0;
          g.xf = 0.0f;
          g.w = 0.0;
          g.mu2 = 0.0;
          g.e02 = e02;
          g.v0h = v0h[q];
          g.pos = v0h[q] > 0.0;
          if (act[q]) {
            // the tests of soc_proj_cta without roots or divisions:
            // inside ||tail/e|| <= v0/e0, polar ||e tail|| <= -e0 v0
            const double s0 = tot[2 * q], s1 = tot[2 * q + 1], mx = tot[2 * NV + q];
            const double v2 = v0h[q] * v0h[q];
            if (v0h[q] >= 0.0 && s0 * e02 <= v2) {
              // inside
            } else if (v0h[q] <= 0.0 && s1 <= e02 * v2) {
              g.mode = SG_WRITE_ZERO;  // polar: zero
            } else if (v0h[q] == 0.0) {
              g.mode = SG_ZERO_HEAD;
            } else {
              // 2^-E with E the binary exponent of max |v| (mx > 0 here)
              const int E = ((__double2hiint(mx) >> 20) & 0x7ff) - 1023;
              g.esh = E;
              g.sc = __hiloint2double((1023 - E) << 20, 0);
              g.c0 = (v0h[q] * g.sc) * (v0h[q] * g.sc) * e02;
              g.top = g.pos ? 0.5 * e02 : rcp_nr(e02);
              g.lo = 0.0;
              g.hi = g.top;
              g.c0f = (float)g.c0;
              g.e02f = (float)e02;
              g.topf = (float)g.top;
              g.lof = 0.0f;
              g.hif = g.topf;
              g.xf = -1.0f;  // no start yet
              g.mode = SG_F32;
            }
          }
        }
        __syncwarp();
        // probe selection in FP32 (lanes < kSgProbes, one probe each; the
        // unnormalised probe sums are rescaled by 2^-2E, so |v| must lie
        // within 2^+-40 for them to neither overflow nor underflow)
        if (g.mode == SG_F32 && probes_ok && g.esh >= -40 && g.esh <= 40) {
          const bool pos = g.pos != 0;
          const float hf = (FLIP1 && q == 1) ? b0f1 : b0f;
          const float topf = pos ? 0.5f * hf : __frcp_rn(hf);  // as the probe abscissae
          const float s2 = __uint_as_float((unsigned)(127 - 2 * g.esh) << 23);  // 2^-2E
          const float c0 = g.c0f, e02f = g.e02f, top = g.topf;
          int lo_b = 0, hi_b = __float_as_int(top);
          int key = 0x7f800000;  // +inf: no candidate
          float cand = 0.0f;
          bool finite = true;
          if (lane < kSgProbes) {
            const float xj = sg_probe_x(topf, lane);
            const float f[3] = {ptot[q * PS + 3 * lane] * s2, ptot[q * PS + 3 * lane + 1] * s2,
                                ptot[q * PS + 3 * lane + 2] * s2};
            float F, dF, d2F;
            soc_fderiv(pos, f, c0, e02f, xj, F, dF, d2F);
            finite = fabsf(F) < INFINITY && fabsf(dF) < INFINITY && fabsf(d2F) < INFINITY &&
                     f[0] > 0.0f;
            if (F > 0.0f) lo_b = __float_as_int(xj); else hi_b = __float_as_int(xj);
            const float step = soc_halley(F, dF, d2F);
            cand = xj + step;
            const float rel = fabsf(step) / fminf(xj, top - xj);
            if (rel < INFINITY) key = __float_as_int(rel);
          }
          // bracket: largest probe with F > 0, smallest with F <= 0
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) {
            lo_b = max(lo_b, __shfl_xor_sync(0xffffffffu, lo_b, off));
            hi_b = min(hi_b, __shfl_xor_sync(0xffffffffu, hi_b, off));
          }
          const float plo = __int_as_float(lo_b), phi = __int_as_float(hi_b);
          if (!(cand > plo && cand < phi)) key = 0x7f800000;
          // best candidate: smallest relative step, ties to the lowest lane
          int kb = key;
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) kb = min(kb, __shfl_xor_sync(0xffffffffu, kb, off));
          const unsigned hit = __ballot_sync(0xffffffffu, key == kb);
          const float best = __shfl_sync(0xffffffffu, cand, __ffs(hit) - 1);
          const bool all_finite = __all_sync(0xffffffffu, finite);
          if (lane == 0 && all_finite && plo < phi) {
            g.lof = plo;
            g.hif = phi;
            g.xf = kb < 0x7f800000 ? best : 0.5f * (plo + phi);
          }
        }
        __syncwarp();
        if (lane == 0 && g.mode == SG_F32 && !(g.xf > g.lof && g.xf < g.hif)) {
          // no probe start: the closed-form one (e0 = sqrt(e0^2))
          const double x0 = soc_initial_guess(tot[2 * q], tot[2 * q + 1], v0h[q], sqrt(e02));
          g.xf = (float)x0;
          if (!(g.xf > g.lof && g.xf < g.hif)) g.xf = 0.5f * (g.lof + g.hif);
        }
        __syncwarp();
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int esh = sv[q].esh;
      const bool f32 = sv[q].mode == SG_F32;
#pragma unroll
      for (int k = 0; k < RC; ++k) {
        const float vf = f32 ? f32_trunc(vc[q][k], esh) : 0.0f;
        afc[q][k] = vf * vf * SG_BF(q, k);
      }
    }
    // ---- passes until every vector is written
    for (;;) {
      int mode[NV];
      bool work = false;
      unsigned m32 = 0u, m64 = 0u;
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        mode[q] = sv[q].mode;
        const SocGridVec& g = sv[q];
        if (mode[q] >= SG_WRITE_ZERO) {
          // write pass (each vector once: warp 0 retires the mode below,
          // after a barrier every thread crosses first)
          const double e02 = g.e02, mu2 = g.mu2;
#pragma unroll
          for (int k = 0; k < RC; ++k) {
            const int64_t i = cbeg + t + k * nt;
            if (i >= cend) continue;
            const double b = SG_BD(q, k);
            double out = 0.0;
            if (mode[q] == SG_WRITE_ZH) out = vc[q][k] * b / (b + e02);
            else if (mode[q] == SG_WRITE) out = vc[q][k] * (b * rcp_nr(b + mu2));
            vp[q][s + i] = (B)out;
          }
          for (int64_t i = cbeg + t + RC * nt; i < cend; i += nt) {
            const double b = SG_BM(q, i), vi = (double)vp[q][s + i];
            double out = 0.0;
            if (mode[q] == SG_WRITE_ZH) out = vi * b / (b + e02);
            else if (mode[q] == SG_WRITE) out = vi * (b * rcp_nr(b + mu2));
            vp[q][s + i] = (B)out;
          }
          if (blockIdx.x == 0 && t == 0) {
            double h = 0.0;
            if (mode[q] == SG_WRITE_ZH) h = sqrt(e02) * sqrt(g.w);
            else if (mode[q] == SG_WRITE)
              h = g.pos ? g.v0h * e02 / (e02 - mu2) : g.v0h * e02 * g.x / (e02 * g.x - 1.0);
            vp[q][s] = (B)h;
          }
        } else if (mode[q] == SG_F32) {
          work = true;
          m32 |= 7u << (3 * q);
        } else if (mode[q] == SG_F64) {
          // f0, f1 in FP64; f2 (see soc_terms_f64) in FP32
          work = true;
          m64 |= 3u << (3 * q);
          m32 |= 4u << (3 * q);
        } else if (mode[q] != SG_DONE) {
          work = true;
          m64 |= 7u << (3 * q);
        }
      }
      if (!work) break;
      float fv[K];
      double dv[K];
#pragma unroll
      for (int k = 0; k < K; ++k) { fv[k] = 0.0f; dv[k] = 0.0; }
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const SocGridVec& g = sv[q];
        const bool pos = g.pos != 0;
        if (mode[q] == SG_F32) {
          const float xf = g.xf;
#pragma unroll
          for (int k = 0; k < RC; ++k) {
            const float b = SG_BF(q, k), a = afc[q][k];  // a = 0 beyond the tail
            const float r = pos ? __frcp_rn(fmaf(2.0f, xf, b)) : __frcp_rn(fmaf(b, xf, 1.0f));
            const float ar2 = a * r * r;
            fv[3 * q] += ar2;
            fv[3 * q + 1] += pos ? ar2 * r : ar2 * b * r;
            fv[3 * q + 2] += pos ? ar2 * r * r : ar2 * b * b * r * r;
          }
          for (int64_t i = cbeg + t + RC * nt; i < cend; i += nt) {
            const float bf = f32_trunc(SG_BM(q, i)), vf = f32_trunc((double)vp[q][s + i], g.esh);
            const float a = vf * vf * bf;
            const float r = pos ? __frcp_rn(fmaf(2.0f, xf, bf)) : __frcp_rn(fmaf(bf, xf, 1.0f));
            const float ar2 = a * r * r;
            fv[3 * q] += ar2;
            fv[3 * q + 1] += pos ? ar2 * r : ar2 * bf * r;
            fv[3 * q + 2] += pos ? ar2 * r * r : ar2 * bf * bf * r * r;
          }
        } else if (mode[q] == SG_F64) {
          double f0 = 0.0, f1 = 0.0;
          float f2 = 0.0f;
#pragma unroll
          for (int k = 0; k < RC; ++k) {
            if (cbeg + t + k * nt >= cend) continue;
            soc_terms_f64(pos, vc[q][k] * g.sc, SG_BD(q, k), g.x, f0, f1, f2);
          }
          for (int64_t i = cbeg + t + RC * nt; i < cend; i += nt)
            soc_terms_f64(pos, (double)vp[q][s + i] * g.sc, SG_BM(q, i), g.x, f0, f1, f2);
          dv[3 * q] = f0;
          dv[3 * q + 1] = f1;
          fv[3 * q + 2] = f2;
        } else if (mode[q] == SG_ZERO_HEAD) {
          // |new tail / e|^2 with new v_i = v_i b_i / (b_i + e0^2)
          double wv = 0.0;
#pragma unroll
          for (int k = 0; k < RC; ++k) {
            if (cbeg + t + k * nt >= cend) continue;
            const double b = SG_BD(q, k), tt = vc[q][k] / (b + g.e02);
            wv += tt * tt * b;
          }
          for (int64_t i = cbeg + t + RC * nt; i < cend; i += nt) {
            const double b = SG_BM(q, i), tt = (double)vp[q][s + i] / (b + g.e02);
            wv += tt * tt * b;
          }
          dv[3 * q] = wv;
        }
      }
      const GridPart gp = grid_part(part, flip);
      if (m32) cta_rows_f32<K>(fv, m32, redf, gp);
      if (m64) cta_rows_f64<K>(dv, K, m64, red, gp);
      grid_sync(gs);
      grid_totals(gp, K, K, m32, tot, totf);
      flip ^= 1;
      // lane 0 of warp q takes vector q's step (separate schedulers)
      if (lane == 0 && w < NV) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          if (q != w) continue;
          SocGridVec& g = sv[q];
          if (g.mode >= SG_WRITE_ZERO) { g.mode = SG_DONE; continue; }
          if (g.mode == SG_ZERO_HEAD) {
            g.w = tot[3 * q];
            g.mode = SG_WRITE_ZH;
            continue;
          }
          const bool pos = g.pos != 0;
          if (g.mode == SG_F32) {
            // FP32 Halley step with bracket (FP32 state: the sums are FP32 too)
            const float f[3] = {totf[3 * q], totf[3 * q + 1], totf[3 * q + 2]};
            float F, dF, d2F;
            const float x = g.xf;
            soc_fderiv(pos, f, g.c0f, g.e02f, x, F, dF, d2F);
            bool handover = !(fabsf(F) < INFINITY && fabsf(dF) < INFINITY && fabsf(d2F) < INFINITY);
            if (!handover) {
              if (F > 0.0f) g.lof = x; else g.hif = x;
              const float step = F == 0.0f ? 0.0f : soc_halley(F, dF, d2F);
              float xn = x + step;
              if (!(xn > g.lof && xn < g.hif)) xn = 0.5f * (g.lof + g.hif);
              const float dist = fminf(x, g.topf - x);
              g.xf = xn;
              ++g.it;
              handover = fabsf(step) <= (float)kSgF32Tol * dist || g.it >= kSgF32Max ||
                         !(xn > g.lof && xn < g.hif);
            }
            if (handover) {  // the FP32 bracket is not trusted
              g.mode = SG_F64;
              g.it = 0;
              g.x = (double)g.xf;
              if (!(g.x > 0.0 && g.x < g.top)) g.x = 0.5 * g.top;
              g.lo = 0.0;
              g.hi = g.top;
            }
            continue;
          }
          if (g.mode != SG_F64) continue;
          // an FP32 f2 out of range (extreme scales) drops the curvature term
          const double f2 = (double)totf[3 * q + 2];
          const double f[3] = {tot[3 * q], tot[3 * q + 1], fabs(f2) < INFINITY ? f2 : 0.0};
          const double dist = fmin(g.x, g.top - g.x);
          const double step = soc_halley_step(pos, f, g.c0, g.e02, g.x, g.lo, g.hi);
          bool small = step == 0.0;
          if (!small) {
            double xn = g.x + step;
            if (!(xn > g.lo && xn < g.hi)) xn = 0.5 * (g.lo + g.hi);
            g.x = xn;
            small = fabs(step) <= kSgF64Tol * dist;
          }
          ++g.it;
          if (small || g.hi - g.lo <= 1e-15 * g.hi || g.it >= kSgF64Max) {
            g.mode = SG_WRITE;
            g.mu2 = pos ? 2.0 * g.x : 1.0 / g.x;
          }
        }
      }
      __syncthreads();
    }
  }
  ktimer_end(tm);
}
#undef SG_BD
#undef SG_BF
#undef SG_BM

}  // namespace pdcs
