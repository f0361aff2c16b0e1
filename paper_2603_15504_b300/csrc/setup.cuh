// Set-up kernels (PDCS note, Algorithm 2 line 1 and Sec. 2.6): CSR validation,
// the rotated-SOC reformulation of Sec. 3 (row pairs (p, q) -> ((p+q)/sqrt2,
// (p-q)/sqrt2)), a deterministic CSR transpose, and the diagonal rescaling
// (Ruiz equilibration passes on row / column infinity norms, then one
// Pock-Chambolle pass with exponent alpha).
#pragma once
#include "common.cuh"

namespace pdcs {

#define PDCS_GRID_LOOP_S(i, N) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (N); i += (int64_t)gridDim.x * blockDim.x)

// err bits: 1 row_ptr, 2 column range, 4 column order, 8 non-finite value
__global__ void k_validate_csr(const int64_t* rp, const int32_t* ci, const double* v, int64_t m,
                               int64_t n, int64_t nnz, unsigned int* err) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < m; r += nwarps) {
    const int64_t s = rp[r], e = rp[r + 1];
    if (s < 0 || e < s || e > nnz) {
      if (lane == 0) atomicOr(err, 1u);
      continue;
    }
    for (int64_t k = s + lane; k < e; k += 32) {
      const int32_t c = ci[k];
      if (c < 0 || c >= n) atomicOr(err, 2u);
      if (k > s && ci[k - 1] >= c) atomicOr(err, 4u);
      if (!isfinite(v[k])) atomicOr(err, 8u);
    }
  }
}

__global__ void k_check_finite(const double* v, int64_t n, unsigned int bit, unsigned int* err) {
  PDCS_GRID_LOOP_S(i, n) {
    if (!isfinite(v[i])) atomicOr(err, bit);
  }
}

// Row lengths after merging each listed pair of rows (s, s+1) into the union of
// their patterns (both new rows share it).  One thread per pair (sequential
// merge of two sorted index lists).
__global__ void k_pair_union_len(const int64_t* rp, const int32_t* ci, const int64_t* pairs,
                                 int64_t npairs, int64_t* len) {
  PDCS_GRID_LOOP_S(b, npairs) {
    const int64_t s = pairs[b];
    int64_t i = rp[s], ie = rp[s + 1], j = rp[s + 1], je = rp[s + 2];
    int64_t cnt = 0;
    while (i < ie || j < je) {
      if (j >= je || (i < ie && ci[i] < ci[j])) ++i;
      else if (i >= ie || ci[j] < ci[i]) ++j;
      else { ++i; ++j; }
      ++cnt;
    }
    len[b] = cnt;
  }
}

// Copy every row to the new CSR (nrp from a host scan); rows in a listed pair
// are written as (r_s + r_{s+1})/sqrt2 and (r_s - r_{s+1})/sqrt2 on the union
// pattern.  pair_of[r] = pair index if r is the first row of a pair, -2 if it
// is the second, -1 otherwise.
__global__ void k_pair_merge(const int64_t* rp, const int32_t* ci, const double* v, int64_t m,
                             const int64_t* nrp, int32_t* nci, double* nv, const int64_t* pair_of) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const double r2 = 0.70710678118654752440;
  for (int64_t r = warp; r < m; r += nwarps) {
    const int64_t pf = pair_of[r];
    if (pf == -2) continue;
    if (pf == -1) {
      const int64_t s = rp[r], e = rp[r + 1], o = nrp[r];
      for (int64_t k = s + lane; k < e; k += 32) {
        nci[o + (k - s)] = ci[k];
        nv[o + (k - s)] = v[k];
      }
      continue;
    }
    if (lane != 0) continue;
    int64_t i = rp[r], ie = rp[r + 1], j = rp[r + 1], je = rp[r + 2];
    int64_t o1 = nrp[r], o2 = nrp[r + 1];
    while (i < ie || j < je) {
      int32_t c;
      double a = 0.0, b = 0.0;
      if (j >= je || (i < ie && ci[i] < ci[j])) { c = ci[i]; a = v[i]; ++i; }
      else if (i >= ie || ci[j] < ci[i]) { c = ci[j]; b = v[j]; ++j; }
      else { c = ci[i]; a = v[i]; b = v[j]; ++i; ++j; }
      nci[o1] = c; nv[o1] = r2 * a + r2 * b; ++o1;
      nci[o2] = c; nv[o2] = r2 * a - r2 * b; ++o2;
    }
  }
}

// (v_s, v_{s+1}) -> ((v_s + v_{s+1})/sqrt2, (v_s - v_{s+1})/sqrt2) at each listed
// offset; an involution.
__global__ void k_rotate_pairs(double* v, const int64_t* pairs, int64_t npairs) {
  const double r2 = 0.70710678118654752440;
  PDCS_GRID_LOOP_S(b, npairs) {
    const int64_t s = pairs[b];
    const double a = v[s], c = v[s + 1];
    v[s] = r2 * a + r2 * c;
    v[s + 1] = r2 * a - r2 * c;
  }
}

// -------------------------------------------------------------- transpose
__global__ void k_col_count(const int32_t* ci, int64_t nnz, unsigned long long* cnt) {
  PDCS_GRID_LOOP_S(k, nnz) atomicAdd(&cnt[ci[k]], 1ull);
}

// Scatter (row, value) into column segments with atomic cursors; the order
// inside a segment is fixed afterwards by k_segment_sort.
__global__ void k_transpose_scatter(const int64_t* rp, const int32_t* ci, const double* v,
                                    int64_t m, unsigned long long* cursor, int32_t* tci,
                                    double* tv) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < m; r += nwarps) {
    for (int64_t k = rp[r] + lane; k < rp[r + 1]; k += 32) {
      const unsigned long long pos = atomicAdd(&cursor[ci[k]], 1ull);
      tci[pos] = (int32_t)r;
      tv[pos] = v[k];
    }
  }
}

// Bitonic sort (ascending by key) of one segment of length len at (key, val),
// in shared or global memory, by one CTA.  The "flip" form of the network only
// compares pairs i < l with l < len, which is exactly the network on the
// segment padded with +inf up to the next power of two (padding never moves).
__device__ void bitonic_segment(int32_t* key, double* val, int64_t len) {
  int64_t N2 = 1;
  while (N2 < len) N2 <<= 1;
  for (int64_t k = 2; k <= N2; k <<= 1) {
    for (int64_t j = k >> 1; j > 0; j >>= 1) {
      for (int64_t i = threadIdx.x; i < N2; i += blockDim.x) {
        const int64_t l = (j == (k >> 1)) ? (i ^ (k - 1)) : (i ^ j);
        if (l > i && l < len && key[i] > key[l]) {
          const int32_t tk = key[i]; key[i] = key[l]; key[l] = tk;
          const double tv = val[i]; val[i] = val[l]; val[l] = tv;
        }
      }
      __syncthreads();
    }
  }
}

constexpr int kSortSmem = 2048;

__global__ void __launch_bounds__(256) k_segment_sort(const int64_t* trp, int32_t* tci, double* tv,
                                                      int64_t nseg) {
  __shared__ int32_t sk[kSortSmem];
  __shared__ double sv[kSortSmem];
  for (int64_t sgi = blockIdx.x; sgi < nseg; sgi += gridDim.x) {
    const int64_t s = trp[sgi], len = trp[sgi + 1] - s;
    if (len <= 1) continue;
    if (len <= kSortSmem) {
      for (int64_t i = threadIdx.x; i < len; i += blockDim.x) { sk[i] = tci[s + i]; sv[i] = tv[s + i]; }
      __syncthreads();
      bitonic_segment(sk, sv, len);
      for (int64_t i = threadIdx.x; i < len; i += blockDim.x) { tci[s + i] = sk[i]; tv[s + i] = sv[i]; }
      __syncthreads();
    } else {
      bitonic_segment(tci + s, tv + s, len);
    }
  }
}

// ---------------------------------------------------------------- scaling
// Per-row reduction of the scaled magnitudes (d1_i |g_ij|) d2_j: max (mode 0)
// or sum of the pw-th power (mode 1).  One warp per row.  For the transposed
// matrix (transposed = 1) drow holds D2 and dcol D1; the product is formed in
// the same order in both cases.
__global__ void k_row_norms(const int64_t* rp, const int32_t* ci, const double* v, int64_t m,
                            const double* drow, const double* dcol, int transposed, int mode,
                            double pw, double* out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < m; r += nwarps) {
    const double dr = drow[r];
    double acc = 0.0;
    for (int64_t k = rp[r] + lane; k < rp[r + 1]; k += 32) {
      const double a = transposed ? (dcol[ci[k]] * fabs(v[k])) * dr : (dr * fabs(v[k])) * dcol[ci[k]];
      if (mode == 0) acc = fmax(acc, a);
      else acc += (pw == 1.0 ? a : pow(a, pw));
    }
    acc = mode == 0 ? warp_max(acc) : warp_sum(acc);
    if (lane == 0) out[r] = acc;
  }
}

// d <- d * (1 / sqrt(norm)) where norm > 0.
__global__ void k_scale_update(double* d, const double* norm, int64_t n) {
  PDCS_GRID_LOOP_S(i, n) {
    const double s = norm[i];
    if (s > 0.0) d[i] = d[i] * (1.0 / sqrt(s));
  }
}

// Scaled values (d1_i g_ij) d2_j written in the solver's value type; also a
// running max of |value| (for eta0 = 1 / ||Ghat||_inf).
template <typename T>
__global__ void k_apply_scale(const int64_t* rp, const int32_t* ci, const double* v, int64_t m,
                              const double* drow, const double* dcol, int transposed, T* out,
                              unsigned long long* amax_bits) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double mx = 0.0;
  for (int64_t r = warp; r < m; r += nwarps) {
    const double dr = drow[r];
    for (int64_t k = rp[r] + lane; k < rp[r + 1]; k += 32) {
      const double a = transposed ? (dcol[ci[k]] * v[k]) * dr : (dr * v[k]) * dcol[ci[k]];
      out[k] = (T)a;
      mx = fmax(mx, fabs(a));
    }
  }
  mx = warp_max(mx);
  if (lane == 0 && amax_bits) atomicMax(amax_bits, (unsigned long long)__double_as_longlong(mx));
}

// out = d o in (mode 0), in / d (mode 1)
__global__ void k_scale_vec(const double* in, const double* d, int64_t n, int mode, double* out) {
  PDCS_GRID_LOOP_S(i, n) out[i] = mode == 0 ? d[i] * in[i] : in[i] / d[i];
}

// One-CTA set-up reduction: out = {sum |v|, sum v^2, max |v / div|}.
__global__ void k_vec_norms(const double* v, int64_t n, const double* div, double* out) {
  __shared__ double sh[2 * 1024 + 2];
  double s[2] = {0.0, 0.0};
  double mx[1] = {0.0};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = v[i];
    s[0] += fabs(a);
    s[1] += a * a;
    mx[0] = fmax(mx[0], fabs(div ? a / div[i] : a));
  }
  block_sum<2>(s, sh);
  block_max<1>(mx, sh);
  if (threadIdx.x == 0) { out[0] = s[0]; out[1] = s[1]; out[2] = mx[0]; }
}

}  // namespace pdcs
