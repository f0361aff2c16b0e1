// Shared device helpers for the PDCS kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define PDCS_DEV __device__ __forceinline__

namespace pdcs {

// Programmatic dependent launch.  A kernel launched with the programmatic
// stream-serialization attribute may be scheduled before its predecessor in
// the stream has finished: pdl_wait() blocks until the predecessor grid has
// completed and its memory operations are visible (a no-op for an ordinary
// launch), so every kernel calls it before reading anything a predecessor
// wrote; pdl_trigger() allows the successor's CTAs to be scheduled once every
// CTA of this grid has called it (or exited), which hides the launch gap
// behind this grid's last wave.
PDCS_DEV void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
PDCS_DEV void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

PDCS_DEV double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP64 <-> FP32 conversions on the integer pipes, from the IEEE-754 binary64
// and binary32 layouts (the FP64 pipe, which would execute cvt, is scarce).
// f32_trunc: v * 2^-shift with the mantissa truncated to 24 bits; zero,
// subnormal and underflowing values give a signed zero, overflowing ones (and
// inf / NaN inputs) a signed infinity.
PDCS_DEV float f32_trunc(double v, int shift = 0) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const int ef = e - 1023 + 127 - shift;
  unsigned r;
  if (e == 0 || ef <= 0) r = sign;
  else if (ef >= 255) r = sign | 0x7f800000u;
  else r = sign | ((unsigned)ef << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  return __uint_as_float(r);
}

// Exact widening of a normal FP32 value (zero and subnormals give zero,
// inf / NaN an infinity).
PDCS_DEV double f64_of_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu;
  if (e == 0u) return __hiloint2double((int)sign, 0);
  if (e == 255u) return __hiloint2double((int)(sign | 0x7ff00000u), 0);
  const unsigned hi = sign | ((e - 127u + 1023u) << 20) | ((u >> 3) & 0xfffffu);
  return __hiloint2double((int)hi, (int)(u << 29));
}

PDCS_DEV double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block reductions.  FP64 instructions are scarce on this GPU (one FP64 pipe
// slot serves a handful of lanes per cycle, and a single warp's dependent FP64
// chain is slow), so the trees avoid redundant FP64 work and spread what is
// left over the SM's four schedulers: every thread stages its K values in
// shared memory, then warp w adds values w, w + nwarps, ... (lane l takes
// threads l, l+32, ... in order, then a fixed butterfly), and the totals are
// broadcast back.  Deterministic, and the same sums whichever warp adds them.
// `sh` must hold K * blockDim.x + K doubles.
template <int K>
PDCS_DEV void block_sum(double (&v)[K], double* sh) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, nw = nt >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) sh[k * nt + tid] = v[k];
  __syncthreads();
  for (int k = tid >> 5; k < K; k += nw) {
    double s = 0.0;
    for (int t = lane; t < nt; t += 32) s += sh[k * nt + t];
    s = warp_sum(s);
    if (lane == 0) sh[K * nt + k] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = sh[K * nt + k];
  __syncthreads();
}

// Maxima of non-negative values (NaN propagates): for non-negative IEEE
// doubles the order of the values equals the order of their bit patterns, so
// the comparisons run on the integer pipes.
PDCS_DEV long long warp_max_bits(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, (long long)__shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

PDCS_DEV double warp_max_nonneg(double v) {
  return __longlong_as_double(warp_max_bits(__double_as_longlong(v)));
}

template <int K>
PDCS_DEV void block_max(double (&v)[K], double* sh) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, nw = nt >> 5;
  long long* shl = reinterpret_cast<long long*>(sh);
#pragma unroll
  for (int k = 0; k < K; ++k) shl[k * nt + tid] = __double_as_longlong(v[k]);
  __syncthreads();
  for (int k = tid >> 5; k < K; k += nw) {
    long long s = 0;
    for (int t = lane; t < nt; t += 32) s = max(s, shl[k * nt + t]);
    s = warp_max_bits(s);
    if (lane == 0) shl[K * nt + k] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = __longlong_as_double(shl[K * nt + k]);
  __syncthreads();
}

// Reduction of per-CTA partials by one whole CTA, in a fixed order (thread t
// adds parts t, t + blockDim, ... sequentially, then a fixed tree): partial
// b's value k sits at part[b * stride + off + k].  KS sums then KM maxima.
template <int KS, int KM>
PDCS_DEV void cta_reduce_parts(const double* part, unsigned nparts, int stride, double (&S)[KS],
                               double (&M)[KM], double* sh) {
#pragma unroll
  for (int k = 0; k < KS; ++k) S[k] = 0.0;
#pragma unroll
  for (int k = 0; k < KM; ++k) M[k] = 0.0;
  for (unsigned b = threadIdx.x; b < nparts; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < KS; ++k) S[k] += __ldcg(part + (size_t)b * stride + k);
#pragma unroll
    for (int k = 0; k < KM; ++k)
      M[k] = __longlong_as_double(max(__double_as_longlong(M[k]),
                                      __double_as_longlong(__ldcg(part + (size_t)b * stride + KS + k))));
  }
  block_sum<KS>(S, sh);
  block_max<KM>(M, sh);
}

template <int KS>
PDCS_DEV void cta_reduce_sums(const double* part, unsigned nparts, int stride, double (&S)[KS],
                              double* sh) {
#pragma unroll
  for (int k = 0; k < KS; ++k) S[k] = 0.0;
  for (unsigned b = threadIdx.x; b < nparts; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < KS; ++k) S[k] += __ldcg(part + (size_t)b * stride + k);
  }
  block_sum<KS>(S, sh);
}

// "Last CTA done" protocol: each CTA publishes its partials, then the CTA that
// observes the final ticket performs the grid-level epilogue.  No CTA waits on
// another, so this cannot hang.  Returns true in exactly one CTA.
PDCS_DEV bool last_block_done(unsigned int* counter) {
  __shared__ unsigned int s_ticket;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(counter, 1u);
  __syncthreads();
  const bool last = (s_ticket == gridDim.x * gridDim.y - 1);
  if (last) __threadfence();
  return last;
}

// Live kernel timer: span from the first CTA's start to the last CTA's end of
// each launch, read from %globaltimer (ns) and accumulated on the device.  A
// NULL timer disables the bookkeeping.  ktimer_end must be reached by every
// thread of the CTA.
struct KTimer {
  unsigned long long start;  // ~0 between launches
  unsigned long long total_ns;
  unsigned int ticket;
  unsigned int launches;
};

PDCS_DEV unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

PDCS_DEV void ktimer_begin(KTimer* tm) {
  if (tm != nullptr && threadIdx.x == 0) atomicMin(&tm->start, global_ns());
}

PDCS_DEV void ktimer_end(KTimer* tm) {
  if (tm == nullptr) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int tk = atomicAdd(&tm->ticket, 1u);
    if (tk == gridDim.x * gridDim.y - 1) {
      __threadfence();
      const unsigned long long t1 = global_ns();
      const unsigned long long t0 = atomicAdd(&tm->start, 0ull);
      tm->total_ns += t1 > t0 ? t1 - t0 : 0ull;
      tm->launches += 1u;
      tm->start = ~0ull;
      tm->ticket = 0u;
    }
  }
}

// Timer slots of one solver (pdcs_get_kernel_times lists them in this order).
enum : int { TM_SPMV_G = 0, TM_SPMV_GT, TM_SPMV_CHECK, TM_SOC_GRID, TM_SOC_CTA, TM_EXP, TM_PRIMAL,
             TM_DUAL, TM_STEP, TM_RES_PREP, TM_STATS_ATTEMPT, TM_STATS_CHECK, TM_HALPERN,
             TM_PROBE_PREP, TM_PROBE_REDUCE, TM_CHECK_MISC, TM_NUM };

PDCS_DEV KTimer* tslot(KTimer* base, int id) { return base == nullptr ? nullptr : base + id; }

}  // namespace pdcs
