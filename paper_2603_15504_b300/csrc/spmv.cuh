// CSR sparse matrix-vector product y = A x for the two products of every PDHG
// step, G xhat and G^T yhat (PDCS note, eq. PDHG).
//
// Rows are binned on the host into tasks, one CTA per task (runs of
// consecutive rows; the kind follows the longest row of the run):
//   kind 0  up to 256 rows of <= 4 nonzeros, one thread per row;
//   kind 1  one group of G lanes per row, lanes striding over the row so
//           loads are coalesced: G = 32 when a row has 513..4096 nonzeros,
//           else the smallest group whose loads still fill 32-byte sectors
//           (G = 4 for FP64, 8 for FP32), which keeps the FP64 shuffle-add tree
//           per row short (FP64 instructions are the scarce resource here);
//           a task holds at least one row per group, so no group idles, and
//           short rows ride along with longer neighbours;
//   kind 2  one chunk of <= kChunk nonzeros of a long row; the chunk sums are
//           written to a partial buffer and the last chunk CTA of the row (an
//           atomic ticket, no waiting) adds them in chunk order, so the result
//           is deterministic.
// Accumulation: in FP64 mode the values are FP64 and each nonzero is one
// DFMA.  In FP32 mode the values are FP32 and the gathered FP64 vector is read
// as a (hi, lo) pair of FP32 numbers (a "shadow" written by the kernel that
// produces the vector): each product v*hi is formed exactly as p + e (FMA
// error term), v*lo is added to e, and p is summed with an error-free
// two-sum into a float-float accumulator, so a row sum carries ~2^-48 relative
// error without using the FP64 pipe, which is the scarce unit of this GPU.
// Each lane issues the index, value and gather loads of kSpmvUnroll nonzeros
// before it adds them (in their order, so the sum is the plain strided one):
// the streams run near the read bandwidth only with that many loads in flight.
#pragma once
#include "common.cuh"

namespace pdcs {

constexpr int kSpmvThreads = 256;
constexpr int64_t kChunk = 8192;
constexpr int kSpmvUnroll = 8;

struct SpmvTask {
  int32_t kind;
  int32_t g;        // lanes per row (kind 1)
  int32_t counter;  // kind 2: ticket counter of this long row
  int32_t nchunks;  // kind 2: chunks of this long row
  int64_t a, b;     // kinds 0/1: rows [a, b); kind 2: row a, chunk index b
  int64_t c, d;     // kind 2: nonzero range [c, d)
  int64_t pbase;    // kind 2: first partial slot of this long row
  int64_t ra, rb;   // kind 2: the row's column run (nonzeros [ra, rb), see below)
  int32_t col0;     // kind 2: column of nonzero ra
  int32_t runs;     // kind 1: rows start with their column run (see runlen)
};

// Column runs.  A long row's longest stretch of nonzeros whose column indices
// are consecutive (ci[k + 1] = ci[k] + 1; the dense blocks a CSR matrix may
// hold, such as a factor model's loadings) is described by its first nonzero
// and first column; a chunk that lies wholly inside it reads no column index
// and its gathers are contiguous.

// Element type of the gathered vector for matrix values of type V.
template <typename V>
struct SpmvX {
  using type = double;
};
template <>
struct SpmvX<float> {
  using type = float2;  // (hi, lo) FP32 split of an FP64 value
};

template <typename V>
struct Acc;

template <>
struct Acc<double> {
  double s = 0.0;
  PDCS_DEV void add(double v, double x) { s = fma(v, x, s); }
  PDCS_DEV double get() const { return s; }
};

template <>
struct Acc<float> {
  float s = 0.0f, c = 0.0f;  // value s + c
  PDCS_DEV void add(float v, float2 x) {
    const float p = __fmul_rn(v, x.x);
    float e = __fmaf_rn(v, x.x, -p);  // v * hi = p + e exactly
    e = __fmaf_rn(v, x.y, e);
    const float t = __fadd_rn(s, p);  // two-sum: s + p = t + err exactly
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
  }
  PDCS_DEV double get() const { return f64_of_f32(s) + f64_of_f32(c); }
};

// FP32 (hi, lo) split of an FP64 value for the gathered-vector shadow.
PDCS_DEV float2 split_ff(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}

// Where a row's value goes: by default y[row]; a caller may pass a functor
// with the same interface that also applies an elementwise update to the
// row.  pre(row) issues the row's other loads before the product's, so their
// latency overlaps it; the call then finishes the row.
template <typename T>
struct StoreOut {
  static constexpr int kMinBlocks = 8;  // resident CTAs per SM (32 registers)
  T* y;
  struct Pre {};
  PDCS_DEV Pre pre(int64_t) const { return Pre{}; }
  PDCS_DEV void operator()(int64_t row, double v, const Pre&) const { y[row] = (T)v; }
};

// Group sum over G consecutive lanes (G a power of two <= 32).
template <int G>
PDCS_DEV double group_sum(double v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
  return v;
}

// A lane's share of nonzeros [k0, e), stride S: trips of kSpmvUnroll nonzeros
// issue their index, value and gather loads together, then the rest go one
// per step (the plain strided order of additions).  RUN: the nonzeros lie in
// a column run and the column of nonzero k is cb + k (no index is loaded).
template <typename V, int S, bool RUN>
PDCS_DEV void spmv_lane(Acc<V>& acc, int64_t k, int64_t e, const int32_t* __restrict__ ci,
                        const V* __restrict__ vv, const typename SpmvX<V>::type* __restrict__ x,
                        int64_t cb) {
  using X = typename SpmvX<V>::type;
  constexpr int U = kSpmvUnroll;
  for (; k + (int64_t)(U - 1) * S < e; k += (int64_t)U * S) {
    int32_t c[U];
    V v[U];
    X xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      c[u] = RUN ? (int32_t)(cb + k) + u * S : __ldg(ci + k + (int64_t)u * S);
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = __ldg(vv + k + (int64_t)u * S);
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = __ldg(x + c[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) acc.add(v[u], xv[u]);
  }
  for (; k < e; k += S)
    acc.add(__ldg(vv + k), __ldg(x + (RUN ? (int32_t)(cb + k) : __ldg(ci + k))));
}

template <typename V, int G, typename Out>
PDCS_DEV void spmv_group_rows(const SpmvTask& t, const int64_t* __restrict__ rp,
                              const int32_t* __restrict__ ci, const int32_t* __restrict__ runlen,
                              const V* __restrict__ vv,
                              const typename SpmvX<V>::type* __restrict__ x, const Out& out) {
  const int gid = threadIdx.x / G, lane = threadIdx.x % G, ng = kSpmvThreads / G;
  // every group runs the same number of trips so the shuffles stay converged
  const int64_t trips = (t.b - t.a + ng - 1) / ng;
  for (int64_t q = 0; q < trips; ++q) {
    const int64_t row = t.a + gid + q * ng;
    Acc<V> acc;
    typename Out::Pre pr{};
    if (lane == 0 && row < t.b) pr = out.pre(row);
    if (row < t.b) {
      const int64_t s = rp[row], e = rp[row + 1];
      // rows of run tasks start with their column run (runlen[row] nonzeros,
      // columns ci[s], ci[s] + 1, ...); the rest follow with their indices
      int64_t re = s, cb = 0;
      if (t.runs) {
        re = s + __ldg(runlen + row);
        if (re > s) cb = (int64_t)__ldg(ci + s) - s;
      }
      spmv_lane<V, G, true>(acc, s + lane, re, ci, vv, x, cb);
      spmv_lane<V, G, false>(acc, re + lane, e, ci, vv, x, 0);
    }
    const double r = group_sum<G>(acc.get());
    if (lane == 0 && row < t.b) out(row, r, pr);
  }
}

template <typename V, typename Out>
PDCS_DEV void spmv_task(const SpmvTask& t, const int64_t* __restrict__ rp,
                        const int32_t* __restrict__ ci, const int32_t* __restrict__ runlen,
                        const V* __restrict__ vv, const typename SpmvX<V>::type* __restrict__ x,
                        const Out& out, double* __restrict__ partial,
                        unsigned int* __restrict__ counters);

// y = A x over the task list, each row's value handed to `out` (StoreOut:
// y[row]).  When `gate` is non-NULL and *gate == 0 the kernel does nothing
// (used to skip products inside a captured graph).  partial / counters are the
// scratch of kind-2 tasks (counters are left at zero).  tm, when non-NULL,
// accumulates the launch's duration.
// (Out::kMinBlocks resident CTAs per SM: the product is bound by memory
// latency, and the highest occupancy the epilogue's registers allow keeps the
// most loads in flight)
template <typename V, typename Out>
__global__ void __launch_bounds__(kSpmvThreads, Out::kMinBlocks)
k_spmv(const SpmvTask* __restrict__ tasks, const int64_t* __restrict__ rp,
       const int32_t* __restrict__ ci, const int32_t* __restrict__ runlen,
       const V* __restrict__ vv, const typename SpmvX<V>::type* __restrict__ x, Out out, double* __restrict__ partial,
       unsigned int* __restrict__ counters, const int* __restrict__ gate, KTimer* tm) {
  pdl_wait();
  pdl_trigger();
  if (gate != nullptr && *gate == 0) return;
  ktimer_begin(tm);
  spmv_task<V, Out>(tasks[blockIdx.x], rp, ci, runlen, vv, x, out, partial, counters);
  ktimer_end(tm);
}

template <typename V, typename Out>
PDCS_DEV void spmv_task(const SpmvTask& t, const int64_t* __restrict__ rp,
                        const int32_t* __restrict__ ci, const int32_t* __restrict__ runlen,
                        const V* __restrict__ vv, const typename SpmvX<V>::type* __restrict__ x,
                        const Out& out, double* __restrict__ partial,
                        unsigned int* __restrict__ counters) {
  if (t.kind == 0) {
    const int64_t row = t.a + threadIdx.x;
    if (row < t.b) {
      const typename Out::Pre pr = out.pre(row);
      const int64_t s = rp[row], e = rp[row + 1];
      Acc<V> acc;
      for (int64_t k = s; k < e; ++k) acc.add(__ldg(vv + k), __ldg(x + __ldg(ci + k)));
      out(row, acc.get(), pr);
    }
    return;
  }
  if (t.kind == 1) {
    if (t.g == 4) spmv_group_rows<V, 4>(t, rp, ci, runlen, vv, x, out);
    else if (t.g == 8) spmv_group_rows<V, 8>(t, rp, ci, runlen, vv, x, out);
    else spmv_group_rows<V, 32>(t, rp, ci, runlen, vv, x, out);
    return;
  }
  // kind 2: chunk of a long row
  __shared__ double sh[kSpmvThreads + 1];
  Acc<V> acc;
  if (t.ra <= t.c && t.d <= t.rb)  // the whole chunk inside the row's column run
    spmv_lane<V, kSpmvThreads, true>(acc, t.c + threadIdx.x, t.d, ci, vv, x,
                                     (int64_t)t.col0 - t.ra);
  else
    spmv_lane<V, kSpmvThreads, false>(acc, t.c + threadIdx.x, t.d, ci, vv, x, 0);
  double r[1] = {acc.get()};
  block_sum<1>(r, sh);
  if (t.nchunks == 1) {
    if (threadIdx.x == 0) out(t.a, r[0], out.pre(t.a));
    return;
  }
  if (threadIdx.x == 0) partial[t.pbase + t.b] = r[0];
  __shared__ unsigned int s_ticket;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(counters + t.counter, 1u);
  __syncthreads();
  if (s_ticket == (unsigned)(t.nchunks - 1)) {
    __threadfence();
    if (threadIdx.x < 32) {
      // lanes take chunks lane, lane + 32, ... (loads issued together), add
      // them in order, then a fixed butterfly: deterministic
      double s = 0.0;
      for (int j = threadIdx.x; j < t.nchunks; j += 32) s += __ldcg(partial + t.pbase + j);
      s = warp_sum(s);
      if (threadIdx.x == 0) {
        out(t.a, s, out.pre(t.a));
        counters[t.counter] = 0u;
      }
    }
  }
}

}  // namespace pdcs
