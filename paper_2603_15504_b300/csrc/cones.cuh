// Projections onto diagonally rescaled cones (PDCS note, Sec. 2.6: after the
// rescaling G -> D1 G D2 the cones D1 K_d^* and D2^{-1} K_p are non-standard and
// their projections reduce to one-dimensional root finding).
//
// Exponential cone K_exp = cl{(x, y, z): y > 0, y e^{x/y} <= z}.  The boundary of
// E K_exp (E = diag(e), e > 0) is the surface {s E (r, 1, e^r) : s > 0} plus the
// flat face {(x, 0, z) : x <= 0, z >= 0}.  The nearest surface point to p lies
// on the ray a(r) = E (r, 1, e^r) that maximises phi(r) = <p, a>/||a||; its
// stationarity condition phi'(r) = 0 is, after multiplying out and cancelling
// the e^{3r} terms (with P = e o p, S = e o e),
//   g(r) = (P0 S1 - P1 S0 r) + P2 S0 e^r (r^2 - r + S1/S0)
//        + S2 e^{2r} (P0 (1 - r) - P1)                          (= 0),
// and phi' has the sign of g.  A coarse scan of phi (FP32) locates the two
// best local maxima on a grid; for each, the sign of g picks the neighbouring
// interval that holds the true local maximum; a safeguarded Newton iteration
// on g refines it (FP32, then FP64 polish).  The projection is the nearest of that surface point, the face
// projection (min(p0,0), 0, max(p2,0)) and the origin, after the membership
// tests for E K_exp and for the polar -E^{-1} K_exp^*.
//
// Second-order cone K_soc = {(t, w): ||w|| <= t}.  For E K_soc with e = (e0, ebar):
// inside if ||vbar/ebar|| <= v0/e0, zero if ||ebar o vbar|| <= -e0 v0, else
//   wbar_i = vbar_i b_i / (b_i + 2 mu),  w0 = v0 e0^2 / (e0^2 - 2 mu),  b_i = ebar_i^2,
// with mu the root of F(mu) = sum a_i/(b_i + 2mu)^2 - v0^2 e0^2/(e0^2 - 2mu)^2,
// a_i = vbar_i^2 b_i, on (0, e0^2/2) when v0 > 0; when v0 < 0 the variable
// nu = 1/(2 mu) in (0, 1/e0^2) is used with
//   H(nu) = sum a_i/(1 + b_i nu)^2 - v0^2 e0^2/(1 - e0^2 nu)^2;
// both are decreasing from a positive value to -inf, and are solved by
// safeguarded Halley steps from the closed-form root of the uniformly scaled
// case.  v0 = 0 gives mu = e0^2/2, w0 = e0 ||wbar/ebar||.
#pragma once
#include <math.h>

#include "common.cuh"

namespace pdcs {

#ifdef __CUDA_ARCH__
#define PDCS_FEXP(x) __expf(x)
#else
#define PDCS_FEXP(x) expf(x)
#endif
#define PDCS_HD __host__ __device__ __forceinline__

// 1/d by Newton-Raphson refinement (r <- r + r (1 - d r), twice) of an FP32
// seed: the seed (FP32 approximate reciprocal of d truncated to FP32) has a
// relative error below 2^-21, so the first step leaves below 2^-42 and the
// second rounding level.  On the device the seed and the range test run on
// the integer and FP32 pipes; only the four FMAs use the FP64 pipe, whose
// throughput is scarce.  Falls back to division outside |d| in
// [2^-100, 2^100].
PDCS_HD double rcp_nr(double d) {
#ifdef __CUDA_ARCH__
  const int e = (__double2hiint(d) >> 20) & 0x7ff;
  if (e < 1023 - 100 || e > 1023 + 100) return 1.0 / d;
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(f32_trunc(d)));
  double r = f64_of_f32(rf);
#else
  const double ad = fabs(d);
  if (!(ad > 0x1p-100 && ad < 0x1p100)) return 1.0 / d;
  double r = (double)(1.0f / (float)d);
#endif
  double e1 = fma(-d, r, 1.0);
  r = fma(r, e1, r);
  e1 = fma(-d, r, 1.0);
  return fma(r, e1, r);
}

// FP64 <-> FP32 for the FP32 screens and scans of the exponential cone: on the
// device through the integer pipes (f32_trunc truncates the mantissa and
// flushes subnormals, f64_of_f32 widens exactly), keeping the conversions out
// of the FP64 pipe these kernels are bound by; plain casts on the host.
PDCS_HD float exp_to_f32(double v) {
#ifdef __CUDA_ARCH__
  return f32_trunc(v);
#else
  return (float)v;
#endif
}
PDCS_HD double exp_to_f64(float v) {
#ifdef __CUDA_ARCH__
  return f64_of_f32(v);
#else
  return (double)v;
#endif
}

// ------------------------------------------------------------------ K_exp
PDCS_HD bool exp_member(double x, double y, double z) {
  if (y > 0.0) {
    if (z <= 0.0) return false;
    return x <= y * log(z / y);
  }
  return (y == 0.0) && (x <= 0.0) && (z >= 0.0);
}

PDCS_HD bool exp_dual_member(double u, double v, double w) {
  if (u < 0.0) {
    if (w <= 0.0) return false;
    return log(-u) + v / u <= 1.0 + log(w);
  }
  return (u == 0.0) && (v >= 0.0) && (w >= 0.0);
}

// Coarse grid of ray parameters: r_i = sinh(-14 + 0.25 i), i = 0..kExpGrid-1.
constexpr int kExpGrid = 113;
PDCS_HD float exp_grid_r(int i) { return sinhf(-14.0f + 0.25f * (float)i); }

// phi(r) for the coarse scan, in FP32, with the ray scaled by e^{-max(r,0)}.
// Of e^{-max(r,0)} and e^{r - max(r,0)} one is e^0 = 1, so one exponential
// is evaluated (the same values as evaluating both).
PDCS_HD float exp_phi_f(float r, float p0, float p1, float p2, float e0, float e1, float e2) {
  const float x = PDCS_FEXP(-fabsf(r));
  const float g = r > 0.0f ? x : 1.0f, h = r > 0.0f ? 1.0f : x;
  const float a0 = e0 * r * g, a1 = e1 * g, a2 = e2 * h;
  const float num = p0 * a0 + p1 * a1 + p2 * a2;
  const float den = sqrtf(a0 * a0 + a1 * a1 + a2 * a2);
  return num / den;
}

// g(r) and g'(r), both multiplied by e^{-2 max(r,0)} (the same factor, so the
// Newton step g/g' and the sign of g are unchanged).  One of e^{r - R} and
// e^{-R} is e^0 = 1, so one exponential is evaluated; s10 = S1 / S0.
template <typename F>
PDCS_HD void exp_g(F r, F P0, F P1, F P2, F S0, F S1, F S2, F s10, F& g, F& dg) {
  const F x = exp(-fabs(r));
  const F E1 = r > F(0) ? F(1) : x;  // e^{r} e^{-R}, R = max(r, 0)
  const F eR = r > F(0) ? x : F(1);  // e^{-R}
  const F E2 = E1 * E1;     // e^{2r} e^{-2R}
  const F q = r * r - r + s10;
  g = (P0 * S1 - P1 * S0 * r) * eR * eR + P2 * S0 * E1 * eR * q + S2 * E2 * (P0 * (F(1) - r) - P1);
  dg = -P1 * S0 * eR * eR + P2 * S0 * E1 * eR * (r * r + r - F(1) + s10) +
       S2 * E2 * (P0 * (F(1) - F(2) * r) - F(2) * P1);
}

// a / b for the Newton steps: FP32 division, or in FP64 a times the
// Newton-Raphson reciprocal (a few FMAs instead of a division sequence).
PDCS_HD float exp_quot(float a, float b) { return a / b; }
PDCS_HD double exp_quot(double a, double b) { return a * rcp_nr(b); }

// Safeguarded Newton on g inside [lo, hi] with g(lo) > 0 >= g(hi); s10 = S1 / S0.
template <typename F>
PDCS_HD F exp_newton(F r, F lo, F hi, F P0, F P1, F P2, F S0, F S1, F S2, F s10, int iters, F tol) {
  for (int it = 0; it < iters; ++it) {
    F g, dg;
    exp_g<F>(r, P0, P1, P2, S0, S1, S2, s10, g, dg);
    if (g > F(0)) lo = r; else hi = r;
    if (g == F(0)) break;
    const F step = -exp_quot(g, dg);
    F rn = r + step;
    // converged: the correction is below tolerance (it may not even move r)
    if (fabs(step) <= tol * (F(1) + fabs(r))) {
      if (rn >= lo && rn <= hi) r = rn;
      break;
    }
    if (!(rn > lo && rn < hi)) rn = F(0.5) * (lo + hi);
    r = rn;
  }
  return r;
}

// Nearest point of the ray through diag(e)(r, 1, e^r) to p; returns the squared
// distance (+inf when <p, a> <= 0, i.e. the ray is not visible from p).
PDCS_HD double exp_ray_point(double r, const double p[3], const double e[3], double c[3]) {
  const double x = exp(-fabs(r));
  const double g = r > 0.0 ? x : 1.0, h = r > 0.0 ? 1.0 : x;  // e^{-R}, e^{r - R}
  const double a0 = e[0] * r * g, a1 = e[1] * g, a2 = e[2] * h;
  const double pa = p[0] * a0 + p[1] * a1 + p[2] * a2;
  const double aa = a0 * a0 + a1 * a1 + a2 * a2;
  if (!(pa > 0.0) || !(aa > 0.0)) return INFINITY;
  const double s = pa * rcp_nr(aa);
  c[0] = s * a0; c[1] = s * a1; c[2] = s * a2;
  return (p[0] - c[0]) * (p[0] - c[0]) + (p[1] - c[1]) * (p[1] - c[1]) + (p[2] - c[2]) * (p[2] - c[2]);
}

// Membership tests screened in FP32: the FP32 value of the defining
// inequality decides unless it lies within a relative margin of the boundary,
// where the FP64 test decides (so the decisions are those of the FP64 tests,
// which cost logarithms in the scarce FP64 pipe).
PDCS_HD bool exp_member_fast(double x, double y, double z) {
  if (y > 0.0 && z > 0.0) {
    const float xf = exp_to_f32(x), yf = exp_to_f32(y), zf = exp_to_f32(z);
    const float l = yf * logf(zf / yf);
    const float t = l - xf;
    if (fabsf(t) > 1e-4f * (fabsf(xf) + fabsf(l)) + 1e-30f && isfinite(t)) return t >= 0.0f;
  }
  return exp_member(x, y, z);
}

PDCS_HD bool exp_dual_member_fast(double u, double v, double w) {
  if (u < 0.0 && w > 0.0) {
    const float uf = exp_to_f32(u), vf = exp_to_f32(v), wf = exp_to_f32(w);
    const float a = logf(-uf), b = vf / uf, c = logf(wf);
    const float t = 1.0f + c - a - b;
    if (fabsf(t) > 1e-4f * (fabsf(a) + fabsf(b) + 1.0f + fabsf(c)) && isfinite(t)) return t >= 0.0f;
  }
  return exp_dual_member(u, v, w);
}

// Projection of p onto diag(e) K_exp (ie = 1 / e, elementwise).  grid: the
// kExpGrid scan abscissae exp_grid_r(i) precomputed (e.g. in shared memory),
// or NULL to evaluate them here.
PDCS_HD void proj_exp_scaled(const double p[3], const double e[3], const double ie[3], double q[3],
                             const float* grid = nullptr) {
  if (exp_member_fast(p[0] * ie[0], p[1] * ie[1], p[2] * ie[2])) {
    q[0] = p[0]; q[1] = p[1]; q[2] = p[2];
    return;
  }
  if (exp_dual_member_fast(-e[0] * p[0], -e[1] * p[1], -e[2] * p[2])) {
    q[0] = q[1] = q[2] = 0.0;
    return;
  }
  // face candidate, and the origin
  double best[3] = {fmin(p[0], 0.0), 0.0, fmax(p[2], 0.0)};
  double bd = (p[0] - best[0]) * (p[0] - best[0]) + p[1] * p[1] + (p[2] - best[2]) * (p[2] - best[2]);
  const double d0 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
  if (d0 < bd) { best[0] = best[1] = best[2] = 0.0; bd = d0; }
  if (!(p[0] <= 0.0 && p[1] <= 0.0)) {
    // Coarse scan: the two largest local maxima of phi on the grid.  The
    // visible part of the surface (phi > 0) can be narrower than the grid
    // spacing, so refinement never requires a positive grid value.
    const float fp0 = exp_to_f32(p[0]), fp1 = exp_to_f32(p[1]), fp2 = exp_to_f32(p[2]);
    const float fe0 = exp_to_f32(e[0]), fe1 = exp_to_f32(e[1]), fe2 = exp_to_f32(e[2]);
    float b1 = -3.0e38f, b2 = -3.0e38f;
    int i1 = -1, i2 = -1;
    auto gr = [&](int i) { return grid ? grid[i] : exp_grid_r(i); };
    float prev2 = -3.0e38f, prev = exp_phi_f(gr(0), fp0, fp1, fp2, fe0, fe1, fe2);
    // the grid values are independent: evaluate them kScan at a time, then
    // walk them in order (the same values and comparisons as one at a time)
    constexpr int kScan = 4;
    for (int i0 = 0; i0 < kExpGrid; i0 += kScan) {
      float f[kScan];
#pragma unroll
      for (int j = 0; j < kScan; ++j)
        f[j] = i0 + j + 1 < kExpGrid ? exp_phi_f(gr(i0 + j + 1), fp0, fp1, fp2, fe0, fe1, fe2)
                                     : -3.0e38f;
#pragma unroll
      for (int j = 0; j < kScan; ++j) {
        const int i = i0 + j;
        if (i >= kExpGrid) break;
        const float cur = prev, nxt = f[j];
        if (cur >= prev2 && cur >= nxt) {
          if (cur > b1) { b2 = b1; i2 = i1; b1 = cur; i1 = i; }
          else if (cur > b2) { b2 = cur; i2 = i; }
        }
        prev2 = cur;
        prev = nxt;
      }
    }
    const double P0 = e[0] * p[0], P1 = e[1] * p[1], P2 = e[2] * p[2];
    const double S0 = e[0] * e[0], S1 = e[1] * e[1], S2 = e[2] * e[2];
    const float P0f = exp_to_f32(P0), P1f = exp_to_f32(P1), P2f = exp_to_f32(P2);
    const float S0f = exp_to_f32(S0), S1f = exp_to_f32(S1), S2f = exp_to_f32(S2);
    const double s10 = S1 * rcp_nr(S0);
    const float s10f = S1f / S0f;
    for (int pass = 0; pass < 2; ++pass) {
      const int bi = pass == 0 ? i1 : i2;
      if (bi < 0) continue;
      const float rbf = gr(bi);
      const float lof_n = bi > 0 ? gr(bi - 1) : rbf, hif_n = bi < kExpGrid - 1 ? gr(bi + 1) : rbf;
      const double rb = exp_to_f64(rbf);
      // neighbourhood of the grid maximum: phi rises then falls in it, so
      // g > 0 at its left end and g < 0 at its right end
      const double lo_n = exp_to_f64(lof_n), hi_n = exp_to_f64(hif_n);
      double c[3];
      if (!(hi_n > lo_n)) {
        const double dd = exp_ray_point(rb, p, e, c);
        if (dd < bd) { best[0] = c[0]; best[1] = c[1]; best[2] = c[2]; bd = dd; }
        continue;
      }
      // FP32: the side of the maximum, then Newton to FP32 accuracy
      float gf, dgf;
      exp_g<float>(rbf, P0f, P1f, P2f, S0f, S1f, S2f, s10f, gf, dgf);
      const float lof = gf > 0.0f ? rbf : lof_n, hif = gf > 0.0f ? hif_n : rbf;
      // a local maximum of phi needs g to change sign across that half of the
      // neighbourhood; grid "maxima" on flat stretches of phi (ties in the
      // FP32 scan) have no sign change and no root, and only the grid point
      // itself is kept as a candidate.  FP32 screens; where it sees no sign
      // change, FP64 values at both points decide.
      const float oend = gf > 0.0f ? hif_n : lof_n;
      bool root = oend != rbf;
      if (root) {
        float go, dgo;
        exp_g<float>(oend, P0f, P1f, P2f, S0f, S1f, S2f, s10f, go, dgo);
        root = gf > 0.0f ? !(go > 0.0f) : (go > 0.0f);
        if (!root) {
          double g0, dg0, g1, dg1;
          exp_g<double>(rb, P0, P1, P2, S0, S1, S2, s10, g0, dg0);
          exp_g<double>(exp_to_f64(oend), P0, P1, P2, S0, S1, S2, s10, g1, dg1);
          root = g0 > 0.0 ? !(g1 > 0.0) : (g1 > 0.0);
        }
      }
      if (!root) {
        const double dd = exp_ray_point(rb, p, e, c);
        if (dd < bd) { best[0] = c[0]; best[1] = c[1]; best[2] = c[2]; bd = dd; }
        continue;
      }
      double r = rb;
      if (hif > lof) {
        const float rf = exp_newton<float>(0.5f * (lof + hif), lof, hif, P0f, P1f, P2f, S0f, S1f,
                                           S2f, s10f, 40, 1e-6f);
        r = exp_to_f64(rf);
      }
      if (!(r > lo_n && r < hi_n)) r = 0.5 * (lo_n + hi_n);
      // FP64 polish in the whole neighbourhood: Newton converges
      // quadratically, so after a step below 1e-6 (1 + |r|) the root is
      // accurate far beyond what the candidate comparison needs
      r = exp_newton<double>(r, lo_n, hi_n, P0, P1, P2, S0, S1, S2, s10, 12, 1e-6);
      double dd = exp_ray_point(r, p, e, c);
      if (!(dd < INFINITY)) dd = exp_ray_point(rb, p, e, c);
      if (dd < bd) { best[0] = c[0]; best[1] = c[1]; best[2] = c[2]; bd = dd; }
    }
  }
  q[0] = best[0]; q[1] = best[1]; q[2] = best[2];
}

// Projection onto diag(e) K' where K' = K_exp (dual == false) or K_exp^* (dual ==
// true, via Moreau: P_{E K*}(v) = v + P_{E^{-1} K}(-v)); ie = 1 / e.
PDCS_HD void proj_exp_family(const double v[3], const double e[3], const double ie[3], bool dual,
                             double out[3], const float* grid = nullptr) {
  if (!dual) { proj_exp_scaled(v, e, ie, out, grid); return; }
  const double nv[3] = {-v[0], -v[1], -v[2]};
  double q[3];
  proj_exp_scaled(nv, ie, e, q, grid);
  out[0] = v[0] + q[0]; out[1] = v[1] + q[1]; out[2] = v[2] + q[2];
}

// ------------------------------------------------------------------ K_soc
// Per-element terms of the secular function and its first two derivatives:
// f += (a r^2, a r^3, a r^4) with r = 1/(b + 2x) (branch v0 > 0, x = mu) or
// (a r^2, a b r^3, a b^2 r^4) with r = 1/(1 + b x) (branch v0 < 0, x = nu).
PDCS_HD void soc_secular_terms(bool pos, double a, double b, double x, double (&f)[3]) {
  const double r = pos ? rcp_nr(b + 2.0 * x) : rcp_nr(1.0 + b * x);
  const double ar2 = a * r * r;
  if (pos) {
    f[0] += ar2;
    f[1] += ar2 * r;
    f[2] += ar2 * r * r;
  } else {
    f[0] += ar2;
    f[1] += ar2 * b * r;
    f[2] += ar2 * b * b * r * r;
  }
}

// F (v0 > 0: F(mu) = sum a/(b+2mu)^2 - c0/(e0^2-2mu)^2; v0 < 0: H(nu) =
// sum a/(1+b nu)^2 - c0/(1-e0^2 nu)^2) and its first two derivatives at x from
// the element sums f of soc_secular_terms; both functions decrease on their
// interval.  T = double, or float for the FP32 search phase.
template <typename T>
PDCS_HD void soc_fderiv(bool pos, const T (&f)[3], T c0, T e02, T x, T& F, T& dF, T& d2F) {
  if (pos) {
    const T r = T(1) / (e02 - T(2) * x);
    F = f[0] - c0 * r * r;
    dF = T(-4) * f[1] - T(4) * c0 * r * r * r;
    d2F = T(24) * f[2] - T(24) * c0 * r * r * r * r;
  } else {
    const T r = T(1) / (T(1) - e02 * x);
    F = f[0] - c0 * r * r;
    dF = T(-2) * f[1] - T(2) * c0 * e02 * r * r * r;
    d2F = T(6) * f[2] - T(6) * c0 * e02 * e02 * r * r * r * r;
  }
}

// Halley step -2 F F' / (2 F'^2 - F F''), Newton's where that is not finite.
template <typename T>
PDCS_HD T soc_halley(T F, T dF, T d2F) {
  T step = T(-2) * F * dF / (T(2) * dF * dF - F * d2F);
  if (!(fabs(step) < T(INFINITY))) step = -F / dF;
  return step;
}

// One safeguarded Halley step on F.  Updates the bracket [lo, hi] (F > 0 at
// lo); returns the step, 0 when converged (the caller then stops).
PDCS_HD double soc_halley_step(bool pos, const double (&f)[3], double c0, double e02, double& x,
                               double& lo, double& hi) {
  double F, dF, d2F;
  soc_fderiv(pos, f, c0, e02, x, F, dF, d2F);
  if (F > 0.0) lo = x; else hi = x;
  if (F == 0.0) return 0.0;
  const double step = soc_halley(F, dF, d2F);
  const double xn = x + step;
  if (fabs(step) <= 1e-15 * x) {  // converged; the step may not even move x
    if (xn >= lo && xn <= hi) x = xn;
    return 0.0;
  }
  return step;
}

// Starting point of the SOC root-finding from the closed-form root obtained
// when every ebar_i^2 equals b_eff = sqrt(sum a_i / sum a_i b_i^-2) (the value
// that matches the secular function at 0 and at infinity).  s0 = sum (v/e)^2,
// s1 = sum (e v)^2 over the tail, v0 / e0 the head; returns x in the variable
// of the branch (mu for v0 > 0, nu = 1/(2 mu) for v0 < 0), strictly inside
// its interval.
PDCS_HD double soc_initial_guess(double s0, double s1, double v0, double e0) {
  const double e02 = e0 * e0;
  const double sa = sqrt(s1);                 // sqrt(sum a_i) without the common scale
  const double beff = sqrt(s1 / s0);
  const double av = fabs(v0) * e0;
  double x, hi;
  if (v0 > 0.0) {
    x = 0.5 * (sa * e02 - av * beff) / (sa + av);  // mu
    hi = 0.5 * e02;
  } else {
    x = (sa - av) / (sa * e02 + av * beff);        // nu
    hi = 1.0 / e02;
  }
  if (!(x > 0.0 && x < hi)) x = 0.5 * hi;
  return x;
}

constexpr double kSocStepTol = 1e-6;

// CTA-wide projection of one block held in registers: each thread owns EPT
// elements (index = threadIdx.x + k * NT); element 0 is the head.  `sh` is
// scratch: 8 doubles of broadcast slots, then a block-reduction area of
// 3 * NT + 3 doubles.
template <int NT, int EPT>
__device__ __forceinline__ void soc_proj_cta(double (&v)[EPT], const double (&e)[EPT], int dim,
                                             double* sh) {
  const int tid = threadIdx.x;
  if (tid == 0) { sh[0] = v[0]; sh[1] = e[0]; }
  __syncthreads();
  const double v0 = sh[0], e0 = sh[1];
  __syncthreads();
  double* red = sh + 8;
  double s[2] = {0.0, 0.0};  // sum (v/e)^2, sum (e v)^2
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int i = tid + k * NT;
    if (i >= 1 && i < dim) {
      const double a = v[k] / e[k], b = v[k] * e[k];
      s[0] += a * a;
      s[1] += b * b;
    }
  }
  block_sum<2>(s, red);
  // Scalar set-up by thread 0, broadcast through sh: FP64 square roots and
  // divisions are long chains on this part, and every warp running them
  // would queue them on its scheduler's FP64 pipe (same values either way).
  if (tid == 0) {
    double mode = 0.0;
    if (sqrt(s[0]) <= v0 / e0) mode = 1.0;         // inside
    else if (sqrt(s[1]) <= -e0 * v0) mode = 2.0;   // polar
    sh[2] = mode;
  }
  __syncthreads();
  const double mode = sh[2];
  __syncthreads();
  if (mode == 1.0) return;  // inside
  if (mode == 2.0) {        // polar
#pragma unroll
    for (int k = 0; k < EPT; ++k) v[k] = 0.0;
    return;
  }
  const double e02 = e0 * e0;
  if (v0 == 0.0) {
    double acc[1] = {0.0};
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int i = tid + k * NT;
      if (i >= 1 && i < dim) {
        const double b = e[k] * e[k];
        v[k] = v[k] * b / (b + e02);
        const double t = v[k] / e[k];
        acc[0] += t * t;
      }
    }
    block_sum<1>(acc, red);
    if (tid == 0) v[0] = e0 * sqrt(acc[0]);
    return;
  }
  // normalise by max |v| for range safety (the projection is homogeneous)
  double mx[1] = {fabs(v0)};
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int i = tid + k * NT;
    if (i >= 1 && i < dim) mx[0] = fmax(mx[0], fabs(v[k]));
  }
  block_max<1>(mx, red);
  const bool pos = v0 > 0.0;
  if (tid == 0) {
    sh[2] = mx[0] > 0.0 ? 1.0 / mx[0] : 1.0;
    sh[3] = pos ? 0.5 * e02 : 1.0 / e02;
    sh[4] = soc_initial_guess(s[0], s[1], v0, e0);
  }
  __syncthreads();
  const double sc = sh[2];
  const double c0 = (v0 * sc) * (v0 * sc) * e02;
  double lo = 0.0, hi = sh[3];
  const double top = hi;
  double x = sh[4];
  __syncthreads();
  // Halley steps until one is below kSocStepTol of x's distance to the ends
  // of (0, top): cubic convergence leaves an error of order kSocStepTol^3 of
  // that distance after it, below what the FP64 sums resolve
  for (int it = 0; it < 200; ++it) {
    double f[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int i = tid + k * NT;
      if (i >= 1 && i < dim) {
        const double vv = v[k] * sc, b = e[k] * e[k], a = vv * vv * b;
        soc_secular_terms(pos, a, b, x, f);
      }
    }
    // block sums of the three terms and the scalar step: the staged values
    // of term k are added by warp k (warp 0 alone in a one-warp CTA; the
    // same order either way), thread 0 steps and publishes x, the bracket
    // and the stop flag (the next iteration's staging happens after every
    // thread has read them)
#pragma unroll
    for (int k = 0; k < 3; ++k) red[k * NT + tid] = f[k];
    __syncthreads();
    if (NT >= 96) {
      const int w = tid >> 5, lane = tid & 31;
      if (w < 3) {
        double a = 0.0;
        for (int t = lane; t < NT; t += 32) a += red[w * NT + t];
        a = warp_sum(a);
        if (lane == 0) red[3 * NT + w] = a;
      }
      __syncthreads();
      if (tid == 0) {
        f[0] = red[3 * NT];
        f[1] = red[3 * NT + 1];
        f[2] = red[3 * NT + 2];
      }
    } else if (tid < 32) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        double a = 0.0;
        for (int t = tid; t < NT; t += 32) a += red[k * NT + t];
        f[k] = warp_sum(a);
      }
    }
    if (tid == 0) {  // scalar step once per CTA, broadcast
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
      sh[6] = pos ? 2.0 * x : 1.0 / x;  // 2 mu at x
    }
    __syncthreads();
    x = sh[2]; lo = sh[3]; hi = sh[4];
    if (sh[5] != 0.0) break;
  }
  const double mu2 = sh[6];  // 2 mu
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int i = tid + k * NT;
    if (i >= 1 && i < dim) {
      const double b = e[k] * e[k];
      v[k] = v[k] * (b / (b + mu2));
    }
  }
  if (tid == 0) v[0] = pos ? v0 * e02 / (e02 - mu2) : v0 * e02 * x / (e02 * x - 1.0);
}

}  // namespace pdcs
