// Batched persistent solver: many independent conic programs solved in one
// kernel launch, one CTA per instance at a time.
//
// The instances are laid out as one block-diagonal problem (set up, scaled
// and transposed by the ordinary set-up; Ruiz / Pock-Chambolle scaling,
// transposition and the RSOC rotation act block by block, so this equals
// setting every instance up on its own).  Each CTA of the persistent grid
// takes the next instance from a queue (largest first) and runs Algorithm 1
// with the restart checks of Algorithm 3 on it to the end: the same per-element
// functions as the grid-wide engine over the instance's row and column ranges,
// CTA-wide reductions in place of grid-wide ones, and the same thread-0
// control functions on the instance's own control block (kept in shared
// memory).  So every instance has its own step sizes, primal weight, restarts
// and termination.  SOC blocks are projected by the CTA (soc_proj_cta with the
// block in registers up to 4096 elements, streamed from memory beyond),
// exponential cones per thread.  The products use `tile`
// lanes per row, chosen per size bucket by an autotuner on the host.
#pragma once
#include "iterate.cuh"
#include "spmv.cuh"

namespace pdcs {

constexpr int kBatchThreads = 512;
constexpr int kBatchSocEpt = 8;  // SOC blocks of up to 512 * 8 = 4096 elements
constexpr int kBatchSh = kStatSums * kBatchThreads + kStatSums;

struct BInst {
  int64_t r0, m, c0, n;                      // row / column ranges in the batch problem
  int32_t soc_r0, soc_rn, soc_c0, soc_cn;    // ranges in the row / column SOC lists
  int32_t exp_r0, exp_rn, exp_c0, exp_cn;    // ranges in the row / column exp lists
  int32_t tile, pad;                         // lanes per row of the products
};

// T: the type of the matrix values (FP64, or FP32 in the FP32 mode); vectors
// are FP64.
template <typename T>
struct BatchArgs {
  Prob<double> p;  // batch-problem data, global indices
  const int64_t *rp, *rpT;
  const int32_t *ci, *ciT;
  const T *vv, *vvT;
  double *x, *y, *xh, *yh, *gx, *gty, *gxh, *gtyh, *x0, *y0, *gx0, *gty0;
  double *xb, *yb, *gxb, *gtyb, *xc, *yc, *gxc, *gtyc;
  double *xs, *ys;
  double *tm[2], *tn[2], *um[2], *un[2], *px[2], *py[2];
  const int64_t *soc_rs, *soc_cs;
  const int32_t *soc_rd, *soc_cd;
  const int64_t *exp_rs, *exp_cs;
  const uint8_t *exp_risd, *exp_cisd;
  const BInst* inst;
  const int32_t* order;   // queue order of the instances
  int32_t count;          // instances in the queue
  Ctl* ctls;              // per instance: final control block
  const Ctl* tmpl;        // options part of the control block
  unsigned int* queue;    // next queue position (zero at launch)
  unsigned long long* times;  // per instance: start and end (global ns)
  double time_limit_s;    // per instance
};

#define PDCS_BLOCK_LOOP(i, lo, hi) for (int64_t i = (lo) + threadIdx.x; i < (hi); i += blockDim.x)

// y[r0 + r] = sum_e v[e] x[ci[e]] for the rows r < nr, `tile` lanes per row
// (a power of two <= 32), FP64 products of the (FP64 or FP32) values; every
// group runs the same number of trips so the shuffles stay converged.
template <typename V>
PDCS_DEV void b_spmv(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                     const V* __restrict__ vv, const double* __restrict__ x, double* __restrict__ y,
                     int64_t r0, int64_t nr, int tile) {
  const int gid = threadIdx.x / tile, lane = threadIdx.x % tile, ng = blockDim.x / tile;
  const int64_t trips = (nr + ng - 1) / ng;
  for (int64_t q = 0; q < trips; ++q) {
    const int64_t r = gid + q * ng;
    Acc<double> acc;
    if (r < nr) {
      const int64_t s = rp[r0 + r], e = rp[r0 + r + 1];
      for (int64_t k = s + lane; k < e; k += tile)
        acc.add((double)__ldg(vv + k), __ldg(x + __ldg(ci + k)));
    }
    double v = acc.get();
    for (int o = tile / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, tile);
    if (lane == 0 && r < nr) y[r0 + r] = v;
  }
}

// One SOC block too large for registers (more than kBatchThreads *
// kBatchSocEpt elements), onto diag(e) K_soc: the root-finding of
// soc_proj_cta (inside / polar tests, the v0 = 0 case, normalisation by
// max |v|, the closed-form start and Halley steps with the same stopping
// rule), every pass streaming the block from memory (each thread takes
// elements tid, tid + NT, ... as soc_proj_cta does).  Kept out of line so the
// persistent kernel's register allocation does not grow.
template <typename B>
__device__ __noinline__ void b_proj_soc_stream(B* v, int64_t s, int dim, const double* d, int inv,
                                               double* sh) {
  const int tid = threadIdx.x, NT = blockDim.x;
  const double v0 = (double)v[s], e0 = cone_scale(d, s, inv);
  double* red = sh + 8;
  double s2[2] = {0.0, 0.0};  // sum (v/e)^2, sum (e v)^2 over the tail
  for (int i = tid; i < dim; i += NT) {
    if (i < 1) continue;
    const double vi = (double)v[s + i], e = cone_scale(d, s + i, inv);
    const double a = vi / e, b = vi * e;
    s2[0] += a * a;
    s2[1] += b * b;
  }
  block_sum<2>(s2, red);
  if (sqrt(s2[0]) <= v0 / e0) return;  // inside (the sums are the same in every thread)
  if (sqrt(s2[1]) <= -e0 * v0) {       // polar
    for (int i = tid; i < dim; i += NT) v[s + i] = (B)0.0;
    return;
  }
  const double e02 = e0 * e0;
  if (v0 == 0.0) {
    double acc[1] = {0.0};
    for (int i = tid; i < dim; i += NT) {
      if (i < 1) continue;
      const double e = cone_scale(d, s + i, inv), b = e * e;
      const double w = (double)v[s + i] * b / (b + e02);
      v[s + i] = (B)w;
      const double t = w / e;
      acc[0] += t * t;
    }
    block_sum<1>(acc, red);
    if (tid == 0) v[s] = (B)(e0 * sqrt(acc[0]));
    return;
  }
  double mx[1] = {fabs(v0)};
  for (int i = tid; i < dim; i += NT)
    if (i >= 1) mx[0] = fmax(mx[0], fabs((double)v[s + i]));
  block_max<1>(mx, red);
  const double sc = mx[0] > 0.0 ? 1.0 / mx[0] : 1.0;
  const double c0 = (v0 * sc) * (v0 * sc) * e02;
  const bool pos = v0 > 0.0;
  double lo = 0.0, hi = pos ? 0.5 * e02 : 1.0 / e02;
  const double top = hi;
  double x = soc_initial_guess(s2[0], s2[1], v0, e0);
  for (int it = 0; it < 200; ++it) {
    double f[3] = {0.0, 0.0, 0.0};
    for (int i = tid; i < dim; i += NT) {
      if (i < 1) continue;
      const double vv = (double)v[s + i] * sc, e = cone_scale(d, s + i, inv);
      const double b = e * e;
      soc_secular_terms(pos, vv * vv * b, b, x, f);
    }
    for (int k = 0; k < 3; ++k) red[k * NT + tid] = f[k];
    __syncthreads();
    if (tid < 32) {
      for (int k = 0; k < 3; ++k) {
        double a = 0.0;
        for (int t = tid; t < NT; t += 32) a += red[k * NT + t];
        f[k] = warp_sum(a);
      }
    }
    if (tid == 0) {  // the scalar step once per CTA, broadcast
      int stop = 0;
      const double dist = fmin(x, top - x);
      const double step = soc_halley_step(pos, f, c0, e02, x, lo, hi);
      if (step == 0.0) {
        stop = 1;
      } else {
        double xn = x + step;
        const bool inside = xn > lo && xn < hi;
        if (!inside) xn = 0.5 * (lo + hi);
        x = xn;
        if ((inside && fabs(step) <= kSocStepTol * dist) || hi - lo <= 1e-15 * hi) stop = 1;
      }
      sh[2] = x; sh[3] = lo; sh[4] = hi; sh[5] = (double)stop;
    }
    __syncthreads();
    x = sh[2]; lo = sh[3]; hi = sh[4];
    // thread 0 rewrites sh[2..5] only after the next pass's staging barrier,
    // which every thread reaches after these reads
    if (sh[5] != 0.0) break;
  }
  const double mu2 = pos ? 2.0 * x : 1.0 / x;  // 2 mu
  for (int i = tid; i < dim; i += NT) {
    if (i < 1) continue;
    const double e = cone_scale(d, s + i, inv), b = e * e;
    v[s + i] = (B)((double)v[s + i] * (b / (b + mu2)));
  }
  if (tid == 0) v[s] = (B)(pos ? v0 * e02 / (e02 - mu2) : v0 * e02 * x / (e02 * x - 1.0));
}

// SOC blocks [first, first + count) of a list, onto diag(e) K_soc (e from d, inv).
template <typename B>
PDCS_DEV void b_proj_soc(B* v, const int64_t* __restrict__ starts, const int32_t* __restrict__ dims,
                         int first, int count, const double* __restrict__ d, int inv, double* sh) {
  for (int j = first; j < first + count; ++j) {
    const int64_t s = starts[j];
    const int dim = dims[j];
    if (dim > kBatchThreads * kBatchSocEpt) {  // uniform
      b_proj_soc_stream(v, s, dim, d, inv, sh);
      __syncthreads();
      continue;
    }
    double vv[kBatchSocEpt], ee[kBatchSocEpt];
#pragma unroll
    for (int k = 0; k < kBatchSocEpt; ++k) {
      const int i = threadIdx.x + k * kBatchThreads;
      vv[k] = i < dim ? (double)v[s + i] : 0.0;
      ee[k] = i < dim ? cone_scale(d, s + i, inv) : 1.0;
    }
    soc_proj_cta<kBatchThreads, kBatchSocEpt>(vv, ee, dim, sh);
#pragma unroll
    for (int k = 0; k < kBatchSocEpt; ++k) {
      const int i = threadIdx.x + k * kBatchThreads;
      if (i < dim) v[s + i] = (B)vv[k];
    }
    __syncthreads();
  }
}

// Exponential-cone 3-blocks [first, first + count) of a list, one per thread.
template <typename B>
PDCS_DEV void b_proj_exp(B* v, const int64_t* __restrict__ starts, const uint8_t* __restrict__ isd,
                         int first, int count, const double* __restrict__ d, int inv, int dual) {
  for (int j = threadIdx.x; j < count; j += blockDim.x) {
    const int64_t s = starts[first + j];
    const double in[3] = {(double)v[s], (double)v[s + 1], (double)v[s + 2]};
    double e[3], ie[3];
    cone_scale_pair(d, nullptr, s, inv, e, ie);
    double out[3];
    proj_exp_family(in, e, ie, (isd[first + j] != 0) != (dual != 0), out);
    v[s] = (B)out[0];
    v[s + 1] = (B)out[1];
    v[s + 2] = (B)out[2];
  }
}

// The cone blocks of one instance's rows / columns (the product cone's zero /
// nonnegative / box parts are projected by the element functions).  The
// barrier between the two lists is taken only when both are present (the
// instance fields are the same for every thread of the CTA).
template <typename T, typename B>
PDCS_DEV void b_project_rows(const BatchArgs<T>& a, const BInst& I, B* v, const double* d, int inv,
                             int dual, double* sh) {
  b_proj_exp(v, a.exp_rs, a.exp_risd, I.exp_r0, I.exp_rn, d, inv, dual);
  if (I.exp_rn > 0 && I.soc_rn > 0) __syncthreads();
  b_proj_soc(v, a.soc_rs, a.soc_rd, I.soc_r0, I.soc_rn, d, inv, sh);
}

template <typename T, typename B>
PDCS_DEV void b_project_cols(const BatchArgs<T>& a, const BInst& I, B* v, const double* d, int inv,
                             int dual, double* sh) {
  b_proj_exp(v, a.exp_cs, a.exp_cisd, I.exp_c0, I.exp_cn, d, inv, dual);
  if (I.exp_cn > 0 && I.soc_cn > 0) __syncthreads();
  b_proj_soc(v, a.soc_cs, a.soc_cd, I.soc_c0, I.soc_cn, d, inv, sh);
}

// Statistics of one point into sc.st[slot] (k_res_prep, the projections and
// k_point_stats of the grid engine, restricted to the instance).
template <typename T, bool FULL>
PDCS_DEV void b_point_stats(const BatchArgs<T>& a, const BInst& I, Ctl& sc, int slot,
                            const PointRef<double>& pt, const double* x0, const double* y0, int buf, double* sh) {
  const Prob<double>& p = a.p;
  const TmpRef tr{a.tm[buf], a.tn[buf], FULL ? a.um[buf] : nullptr, FULL ? a.un[buf] : nullptr};
  PDCS_BLOCK_LOOP(i, I.r0, I.r0 + I.m) res_prep_row(p, pt, tr, i);
  PDCS_BLOCK_LOOP(j, I.c0, I.c0 + I.n) res_prep_col(p, pt, tr, j);
  __syncthreads();
  const bool ccones = I.exp_cn + I.soc_cn > 0;  // uniform: the instance's column cones
  b_project_rows(a, I, tr.tm, p.d1, 0, 0, sh);
  __syncthreads();
  if (ccones) {
    b_project_cols(a, I, tr.tn, p.d2, 0, 1, sh);
    __syncthreads();
  }
  if (FULL) {
    b_project_rows(a, I, tr.um, (const double*)nullptr, 0, 0, sh);
    __syncthreads();
    if (ccones) {
      b_project_cols(a, I, tr.un, (const double*)nullptr, 0, 1, sh);
      __syncthreads();
    }
  }
  double s[kStatSums], mx[kStatMax];
#pragma unroll
  for (int k = 0; k < kStatSums; ++k) s[k] = 0.0;
#pragma unroll
  for (int k = 0; k < kStatMax; ++k) mx[k] = 0.0;
  PDCS_BLOCK_LOOP(i, I.r0, I.r0 + I.m) stats_row<double, FULL>(p, pt, y0, tr, i, s, mx);
  PDCS_BLOCK_LOOP(j, I.c0, I.c0 + I.n) stats_col<double, FULL>(p, pt, x0, tr, j, s, mx);
  block_sum<kStatSums>(s, sh);
  block_max<kStatMax>(mx, sh);
  if (threadIdx.x == 0) ctl_stats_finalize(sc, slot, s, mx);
  __syncthreads();
}

// One attempt of Function 1 and, if accepted, maxErr, beta and the reflected
// Halpern step (the attempt body of the grid engine).
template <typename T>
PDCS_DEV void b_attempt(const BatchArgs<T>& a, const BInst& I, Ctl& sc, double* sh) {
  const Prob<double>& p = a.p;
  const int64_t r0 = I.r0, r1 = I.r0 + I.m, c0 = I.c0, c1 = I.c0 + I.n;
  const double tau = sc.eta / sc.omega, sigma = sc.eta * sc.omega;
  PDCS_BLOCK_LOOP(j, c0, c1) primal_elem(p, tau, a.x, a.gty, a.xh, j);
  __syncthreads();
  if (I.exp_cn + I.soc_cn > 0) {  // column cones: their projection, then a barrier
    b_project_cols(a, I, a.xh, p.d2, 1, 0, sh);
    __syncthreads();
  }
  b_spmv(a.rp, a.ci, a.vv, a.xh, a.gxh, r0, I.m, I.tile);
  __syncthreads();
  PDCS_BLOCK_LOOP(i, r0, r1) dual_elem(p, sigma, a.y, a.gxh, a.gx, a.yh, i);
  __syncthreads();
  b_project_rows(a, I, a.yh, p.d1, 1, 1, sh);
  __syncthreads();
  double s3[3] = {0.0, 0.0, 0.0};
  PDCS_BLOCK_LOOP(j, c0, c1) {
    const double d = (double)a.xh[j] - (double)a.x[j];
    s3[0] += d * d;
  }
  PDCS_BLOCK_LOOP(i, r0, r1) {
    const double d = (double)a.yh[i] - (double)a.y[i];
    s3[1] += d * d;
    s3[2] += d * ((double)a.gxh[i] - (double)a.gx[i]);
  }
  block_sum<3>(s3, sh);
  if (threadIdx.x == 0) ctl_step_finalize(sc, s3[0], s3[1], s3[2]);
  __syncthreads();
  if (!sc.g_accept) return;
  b_spmv(a.rpT, a.ciT, a.vvT, a.yh, a.gtyh, c0, I.n, I.tile);
  __syncthreads();
  const PointRef<double> ph{a.xh, a.yh, a.gxh, a.gtyh};
  b_point_stats<T, false>(a, I, sc, 0, ph, nullptr, nullptr, 0, sh);
  const double kk = (double)sc.k, beta = sc.beta, eta = sc.eta_acc;
  const HalpernCoefs hc = halpern_coefs(kk, beta);
  PDCS_BLOCK_LOOP(j, c0, c1) halpern_elem(hc, eta, a.x, a.gty, a.xh, a.gtyh, a.x0, a.gty0, a.xs, j);
  PDCS_BLOCK_LOOP(i, r0, r1) halpern_elem(hc, eta, a.y, a.gx, a.yh, a.gxh, a.y0, a.gx0, a.ys, i);
  __syncthreads();
  if (threadIdx.x == 0) ctl_halpern_finalize(sc, eta, beta, nullptr);
  __syncthreads();
}

// The restart / termination check (average, candidate statistics, Algorithm 3
// for both candidates, decision, candidate copy and the restart's products).
template <typename T>
PDCS_DEV void b_check(const BatchArgs<T>& a, const BInst& I, Ctl& sc, double* sh) {
  const Prob<double>& p = a.p;
  const int64_t r0 = I.r0, r1 = I.r0 + I.m, c0 = I.c0, c1 = I.c0 + I.n;
  const double w = sc.wsum;
  PDCS_BLOCK_LOOP(j, c0, c1) a.xb[j] = a.xs[j] / w;
  PDCS_BLOCK_LOOP(i, r0, r1) a.yb[i] = a.ys[i] / w;
  __syncthreads();
  b_spmv(a.rp, a.ci, a.vv, a.xb, a.gxb, r0, I.m, I.tile);
  b_spmv(a.rpT, a.ciT, a.vvT, a.yb, a.gtyb, c0, I.n, I.tile);
  __syncthreads();
  const PointRef<double> z{a.x, a.y, a.gx, a.gty}, zb{a.xb, a.yb, a.gxb, a.gtyb};
  b_point_stats<T, true>(a, I, sc, 1, z, a.x0, a.y0, 0, sh);
  b_point_stats<T, true>(a, I, sc, 2, zb, a.x0, a.y0, 1, sh);
  if (threadIdx.x == 0) ctl_bisect_init(sc);
  __syncthreads();
  while (sc.bs[0].active || sc.bs[1].active) {
    for (int c = 0; c < 2; ++c) {
      if (!sc.bs[c].active) continue;  // uniform
      const PointRef<double> pt = c == 0 ? z : zb;
      const double t = probe_t(sc.bs[c]);
      const double tt = t * sc.bs[c].tau, ts = t * sc.bs[c].sigma;
      PDCS_BLOCK_LOOP(j, c0, c1) probe_prep_col(p, pt, tt, a.px[c], j);
      PDCS_BLOCK_LOOP(i, r0, r1) probe_prep_row(p, pt, ts, a.py[c], i);
      __syncthreads();
      if (I.exp_cn + I.soc_cn > 0) {
        b_project_cols(a, I, a.px[c], p.d2, 1, 0, sh);
        __syncthreads();
      }
      b_project_rows(a, I, a.py[c], p.d1, 1, 1, sh);
      __syncthreads();
    }
    double s8[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < 2; ++c) {
      if (!sc.bs[c].active) continue;
      const PointRef<double> pt = c == 0 ? z : zb;
      double s4[4] = {0.0, 0.0, 0.0, 0.0};
      PDCS_BLOCK_LOOP(j, c0, c1) probe_sum_col(p, pt, a.px[c], j, s4);
      PDCS_BLOCK_LOOP(i, r0, r1) probe_sum_row(p, pt, a.py[c], i, s4);
      for (int k = 0; k < 4; ++k) s8[4 * c + k] = s4[k];
    }
    block_sum<8>(s8, sh);
    if (threadIdx.x == 0) {
      const double SS[2][4] = {{s8[0], s8[1], s8[2], s8[3]}, {s8[4], s8[5], s8[6], s8[7]}};
      ctl_probe_finalize(sc, SS);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) ctl_check_decide(sc, nullptr);
  __syncthreads();
  const PointRef<double> s = sc.cand ? zb : z;
  const bool rs = sc.g_restart != 0;
  PDCS_BLOCK_LOOP(j, c0, c1) {
    const double v = s.x[j];
    a.gtyc[j] = s.gty[j];
    a.xc[j] = v;
    if (rs) { a.x0[j] = v; a.x[j] = v; a.xs[j] = 0.0; }
  }
  PDCS_BLOCK_LOOP(i, r0, r1) {
    const double v = s.y[i];
    a.gxc[i] = s.gx[i];
    a.yc[i] = v;
    if (rs) { a.y0[i] = v; a.y[i] = v; a.ys[i] = 0.0; }
  }
  __syncthreads();
  if (rs) {
    b_spmv(a.rp, a.ci, a.vv, a.x0, a.gx0, r0, I.m, I.tile);
    b_spmv(a.rpT, a.ciT, a.vvT, a.y0, a.gty0, c0, I.n, I.tile);
    __syncthreads();
    PDCS_BLOCK_LOOP(j, c0, c1) a.gty[j] = a.gty0[j];
    PDCS_BLOCK_LOOP(i, r0, r1) a.gx[i] = a.gx0[i];
    __syncthreads();
  }
  if (threadIdx.x == 0) ctl_check_end(sc);
  __syncthreads();
}

// One instance from a cold start to termination; the returned point is left
// in (xc, yc, gxc, gtyc) and its statistics in sc.st[3].
template <typename T>
PDCS_DEV void b_solve(const BatchArgs<T>& a, const BInst& I, Ctl& sc, double* sh,
                      unsigned long long t_begin) {
  const Prob<double>& p = a.p;
  const int64_t r0 = I.r0, r1 = I.r0 + I.m, c0 = I.c0, c1 = I.c0 + I.n;
  // per-instance norms: ||hhat||_1, ||hhat||_2^2, ||chat||_1, ||chat||_2^2,
  // ||h||_inf, ||c||_inf (unscaled) and max |Ghat| (eta0 = 1 / max |Ghat|)
  double s4[4] = {0.0, 0.0, 0.0, 0.0}, mx3[3] = {0.0, 0.0, 0.0};
  PDCS_BLOCK_LOOP(i, r0, r1) {
    const double h = (double)p.h[i];
    s4[0] += fabs(h);
    s4[1] += h * h;
    mx3[0] = fmax(mx3[0], fabs(h / p.d1[i]));
  }
  PDCS_BLOCK_LOOP(j, c0, c1) {
    const double c = (double)p.c[j];
    s4[2] += fabs(c);
    s4[3] += c * c;
    mx3[1] = fmax(mx3[1], fabs(c / p.d2[j]));
  }
  if (I.m > 0) {
    PDCS_BLOCK_LOOP(e, a.rp[r0], a.rp[r1]) mx3[2] = fmax(mx3[2], fabs((double)a.vv[e]));
  }
  block_sum<4>(s4, sh);
  block_max<3>(mx3, sh);
  // largest row / column absolute sums of the instance's Ghat (fixed step)
  const bool fixed = !a.tmpl->adaptive_step;
  double rc[2] = {0.0, 0.0};
  if (fixed) {
    PDCS_BLOCK_LOOP(i, r0, r1) {
      double t = 0.0;
      for (int64_t e = a.rp[i]; e < a.rp[i + 1]; ++e) t += fabs((double)a.vv[e]);
      rc[0] = fmax(rc[0], t);
    }
    PDCS_BLOCK_LOOP(j, c0, c1) {
      double t = 0.0;
      for (int64_t e = a.rpT[j]; e < a.rpT[j + 1]; ++e) t += fabs((double)a.vvT[e]);
      rc[1] = fmax(rc[1], t);
    }
    block_max<2>(rc, sh);
  }
  if (threadIdx.x == 0) {
    sc = *a.tmpl;
    const double nh2 = sqrt(s4[1]), nc2 = sqrt(s4[3]);
    const double omega0 = (nc2 > 1e-10 && nh2 > 1e-10) ? nc2 / nh2 : 1.0;  // Sec. 2.5
    const double eta0 = mx3[2] > 0.0 ? 1.0 / mx3[2] : 1.0;                  // 1 / ||Ghat||_inf
    sc.eta = sc.eta_hat = sc.eta_acc = sc.eta0 = eta0;
    if (fixed) {
      sc.eta_fixed = (rc[0] > 0.0 && rc[1] > 0.0) ? 1.0 / sqrt(rc[1] * rc[0]) : 1.0;
      sc.eta = sc.eta_hat = sc.eta_acc = sc.eta_fixed;
    }
    sc.omega = sc.omega0 = omega0;
    sc.h1 = s4[0];
    sc.c1 = s4[2];
    sc.hinf = mx3[0];
    sc.cinf = mx3[1];
    sc.status = kRunning;
  }
  // cold start: x = y = 0, so every product is zero
  PDCS_BLOCK_LOOP(j, c0, c1) {
    a.x[j] = a.x0[j] = a.gty[j] = a.gty0[j] = 0.0;
    a.xs[j] = 0.0;
  }
  PDCS_BLOCK_LOOP(i, r0, r1) {
    a.y[i] = a.y0[i] = a.gx[i] = a.gx0[i] = 0.0;
    a.ys[i] = 0.0;
  }
  __syncthreads();
  const unsigned long long limit = (unsigned long long)(a.time_limit_s * 1e9);
  while (true) {
    if (threadIdx.x == 0) ctl_period_begin(sc);
    __syncthreads();
    while (sc.g_attempt) {
      b_attempt(a, I, sc, sh);
      if (threadIdx.x == 0) ctl_loop_ctl(sc);
      __syncthreads();
    }
    if (sc.g_check) b_check(a, I, sc, sh);
    if (threadIdx.x == 0 && sc.status == kRunning && global_ns() - t_begin > limit) sc.status = 6;
    __syncthreads();
    if (sc.status != kRunning) break;
  }
  // returned point: the last candidate, else the current iterate
  if (!sc.have_cand) {
    PDCS_BLOCK_LOOP(j, c0, c1) { a.xc[j] = a.x[j]; a.gtyc[j] = a.gty[j]; }
    PDCS_BLOCK_LOOP(i, r0, r1) { a.yc[i] = a.y[i]; a.gxc[i] = a.gx[i]; }
    __syncthreads();
  }
  const PointRef<double> pr{a.xc, a.yc, a.gxc, a.gtyc};
  b_point_stats<T, true>(a, I, sc, 3, pr, nullptr, nullptr, 0, sh);
}

template <typename T>
__global__ void __launch_bounds__(kBatchThreads) k_batch(BatchArgs<T> a) {
  __shared__ double sh[kBatchSh];
  __shared__ Ctl sc;
  __shared__ int s_next;
  for (;;) {
    if (threadIdx.x == 0) s_next = (int)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int q = s_next;
    __syncthreads();
    if (q >= a.count) break;
    const int idx = a.order[q];
    const BInst I = a.inst[idx];
    const unsigned long long t_begin = global_ns();
    b_solve(a, I, sc, sh, t_begin);
    if (threadIdx.x == 0) {
      a.ctls[idx] = sc;
      a.times[2 * idx] = t_begin;
      a.times[2 * idx + 1] = global_ns();
    }
    __syncthreads();
  }
}

}  // namespace pdcs
