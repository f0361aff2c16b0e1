// Allocation-free sparse product y = G x (include/pdcs.h: pdcs_spmv_noalloc).
//
// The paper has no counterpart: this is a service entry point for callers that
// must not allocate device memory at the time of the call, for example code
// running while a caching allocator (such as PyTorch's) owns the device's whole
// memory budget, where a cudaMalloc would fail or force the allocator to
// release its cache.  It is a variant of the solver's k_spmv: rows of up to
// kNaChunk nonzeros are summed by one warp each; longer rows are split into
// kNaChunk-nonzero chunks whose partial sums are combined, in chunk order, by
// the warp that finishes a row's last chunk (the same ticket scheme as k_spmv).
// Where k_spmv keeps its task plan, chunk partials and tickets in memory the
// solver handle allocated, this variant keeps them in one file-scope device
// array of fixed size (g_na_scratch, below) and builds the chunk list on the
// device, so a call allocates nothing.
//
// Scratch facts (documented in the header as well):
//  * the tickets must be zero when a call starts.  Static device memory is
//    zero when the library is loaded, and every call that completes leaves the
//    tickets zero again; a call cut short by a device error leaves them
//    undefined, and later results are then wrong;
//  * all calls on one device share the scratch, so calls that overlap in time
//    (two streams, or two host threads, without ordering between them) race
//    and give wrong results: serialise them;
//  * the first call on a device looks up the scratch's device address
//    (cudaGetSymbolAddress, with that device current) and caches it;
//  * a call never synchronises: the size check runs on the device, and a
//    matrix beyond the scratch makes the product kernel return without
//    writing y and adds one to a sticky count of rejected calls, which
//    pdcs_spmv_noalloc_status reads (synchronising then) and clears.  So
//    the call can be captured into a graph, except the first one on a
//    device, which looks up the scratch's address.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "../../include/pdcs.h"
#include "common.cuh"

namespace pdcs {
extern thread_local std::string g_last_error;  // defined with the rest of the ABI
}

namespace {

using pdcs::warp_sum;

constexpr int64_t kNaChunk = 4096;       // nonzeros per chunk; longer rows are split
constexpr int kNaMaxLongRows = 4096;     // rows longer than kNaChunk, per call
constexpr int kNaMaxChunks = 65536;      // chunks of those rows, per call
constexpr int kNaMaxDevices = 64;
constexpr int kNaScanThreads = 1024;

struct NaStatus {
  long long long_rows;  // rows longer than kNaChunk
  long long chunks;     // their chunks
  int overflow;         // 1: more than the scratch holds (nothing computed)
  unsigned int rejected;  // calls rejected since the last status query (sticky)
};

// Everything a call needs beyond the caller's arrays (about 0.8 MB).
struct NaScratch {
  double partial[kNaMaxChunks];          // chunk partial sums
  int chunk_slot[kNaMaxChunks];          // long-row slot of each chunk
  int first[kNaMaxLongRows + 1];         // first chunk of each slot (prefix sums)
  long long row[kNaMaxLongRows];         // row index of each slot
  unsigned int ticket[kNaMaxLongRows];   // chunks finished per slot; zero between calls
  NaStatus status;
};

static __device__ __align__(256) NaScratch g_na_scratch;

// Device address of g_na_scratch per device (looked up once per device).
NaScratch* g_na_addr[kNaMaxDevices] = {};
std::mutex g_na_mutex;

// One CTA: list the rows longer than kNaChunk in row order, with their chunk
// ranges.  Warp w owns a contiguous range of rows and reads it 32 rows at a
// time (lane l takes row r0 + l, so the row-pointer loads coalesce); ballots
// count and, in a second sweep, place the long rows of each 32-row group in
// order.  A block-wide exclusive scan of the warps' counts gives every warp
// its output offsets.
__global__ void __launch_bounds__(kNaScanThreads) k_na_scan(const int64_t* __restrict__ rp,
                                                            int64_t m, NaScratch* s) {
  constexpr int kWarps = kNaScanThreads / 32;
  __shared__ long long sh_rows[kWarps], sh_chunks[kWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t per = ((m + kWarps - 1) / kWarps + 31) / 32 * 32;  // whole 32-row groups
  const int64_t r0 = min(m, (int64_t)w * per), r1 = min(m, r0 + per);
  long long nr = 0, nc = 0;
  for (int64_t base = r0; base < r1; base += 32) {
    const int64_t r = base + lane;
    const int64_t len = r < r1 ? rp[r + 1] - rp[r] : 0;
    const bool lng = len > kNaChunk;
    long long ch = lng ? (len + kNaChunk - 1) / kNaChunk : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ch += __shfl_xor_sync(0xffffffffu, ch, o);
    nr += __popc(__ballot_sync(0xffffffffu, lng));
    nc += ch;
  }
  if (lane == 0) { sh_rows[w] = nr; sh_chunks[w] = nc; }
  __syncthreads();
  long long slot = 0, chunk = 0, tot_rows = 0, tot_chunks = 0;
  for (int k = 0; k < kWarps; ++k) {  // exclusive scan (integers: order is irrelevant)
    if (k < w) { slot += sh_rows[k]; chunk += sh_chunks[k]; }
    tot_rows += sh_rows[k];
    tot_chunks += sh_chunks[k];
  }
  const bool overflow = tot_rows > kNaMaxLongRows || tot_chunks > kNaMaxChunks;
  if (threadIdx.x == 0) {
    s->status.long_rows = tot_rows;
    s->status.chunks = tot_chunks;
    s->status.overflow = overflow ? 1 : 0;
    if (overflow) s->status.rejected += 1u;  // one thread, ordered by the stream
    if (!overflow) s->first[tot_rows] = (int)tot_chunks;
  }
  if (overflow || nr == 0) return;
  for (int64_t base = r0; base < r1; base += 32) {
    const int64_t r = base + lane;
    const int64_t len = r < r1 ? rp[r + 1] - rp[r] : 0;
    const bool lng = len > kNaChunk;
    const unsigned bal = __ballot_sync(0xffffffffu, lng);
    if (bal == 0u) continue;
    const long long k = lng ? (len + kNaChunk - 1) / kNaChunk : 0;
    // chunks of the long rows of this group before lane l (inclusive scan - own)
    long long pre = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long v = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= o) pre += v;
    }
    if (lng) {
      const long long my_slot = slot + __popc(bal & ((1u << lane) - 1u));
      const long long my_chunk = chunk + pre - k;
      s->row[my_slot] = r;
      s->first[my_slot] = (int)my_chunk;
      for (long long c = 0; c < k; ++c) s->chunk_slot[my_chunk + c] = (int)my_slot;
    }
    slot += __popc(bal);
    chunk += __shfl_sync(0xffffffffu, pre, 31);
  }
}

// y = G x: warps take the short rows (one row each), then the chunks of the
// long rows; the warp finishing a long row's last chunk adds its partials in
// chunk order (lane-strided, then a fixed butterfly) and resets the ticket.
__global__ void __launch_bounds__(256) k_na_spmv(const int64_t* __restrict__ rp,
                                                 const int32_t* __restrict__ ci,
                                                 const double* __restrict__ val,
                                                 const double* __restrict__ x, double* __restrict__ y,
                                                 int64_t m, NaScratch* s) {
  const int lane = threadIdx.x & 31;
  if (s->status.overflow) return;  // rejected by the scan: y stays as it was
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = wid; r < m; r += nw) {
    const int64_t a = rp[r], b = rp[r + 1];
    if (b - a > kNaChunk) continue;  // done chunk by chunk below
    double acc = 0.0;
    for (int64_t e = a + lane; e < b; e += 32) acc = fma(val[e], x[ci[e]], acc);
    acc = warp_sum(acc);
    if (lane == 0) y[r] = acc;
  }
  const int64_t nch = s->status.chunks;
  for (int64_t c = wid; c < nch; c += nw) {
    const int slot = s->chunk_slot[c];
    const int64_t r = s->row[slot];
    const int f0 = s->first[slot], f1 = s->first[slot + 1];
    const int64_t a = rp[r] + (c - f0) * kNaChunk, b = min(rp[r + 1], a + kNaChunk);
    double acc = 0.0;
    for (int64_t e = a + lane; e < b; e += 32) acc = fma(val[e], x[ci[e]], acc);
    acc = warp_sum(acc);
    unsigned int done = 0;
    if (lane == 0) {
      s->partial[c] = acc;
      __threadfence();
      done = atomicAdd(&s->ticket[slot], 1u) + 1u;
    }
    done = __shfl_sync(0xffffffffu, done, 0);
    if (done == (unsigned int)(f1 - f0)) {
      __threadfence();
      double tot = 0.0;
      for (int j = f0 + lane; j < f1; j += 32) tot += __ldcg(s->partial + j);
      tot = warp_sum(tot);
      if (lane == 0) {
        y[r] = tot;
        s->ticket[slot] = 0u;
      }
    }
  }
}

int na_fail(int code, const char* msg) {
  pdcs::g_last_error = msg;
  return code;
}

// Device memory (or managed) on the current device?
bool na_device_ptr(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

// Device address of the scratch on the current device; the first lookup on a
// device may load the module, so it is refused inside a stream capture.
int na_scratch(bool capturing, NaScratch** out, int* dev_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices)
    return na_fail(PDCS_ERR_CUDA, "pdcs_spmv_noalloc: no usable current device");
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_addr[dev]) {
    if (capturing)
      return na_fail(PDCS_ERR_INVALID,
                     "pdcs_spmv_noalloc: the first call on a device cannot be captured (it "
                     "looks up the scratch's address); make one call before capturing");
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess) return na_fail(PDCS_ERR_CUDA, cudaGetErrorString(e));
    g_na_addr[dev] = static_cast<NaScratch*>(p);
  }
  *out = g_na_addr[dev];
  *dev_out = dev;
  return PDCS_OK;
}

int na_capturing(cudaStream_t st, bool* capturing) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    return na_fail(PDCS_ERR_CUDA, "pdcs_spmv_noalloc: cannot query the stream's capture state");
  }
  *capturing = cap != cudaStreamCaptureStatusNone;
  return PDCS_OK;
}

}  // namespace

extern "C" int pdcs_spmv_noalloc(int64_t m, int64_t n, const int64_t* row_ptr,
                                 const int32_t* col_idx, const double* val, const double* x,
                                 double* y, void* cuda_stream) {
  if (m < 0 || n < 0) return na_fail(PDCS_ERR_INVALID, "pdcs_spmv_noalloc: m and n must be >= 0");
  if (m == 0) return PDCS_OK;
  if (!row_ptr || !y || (n > 0 && (!col_idx || !val || !x)))
    return na_fail(PDCS_ERR_INVALID, "pdcs_spmv_noalloc: NULL array");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  bool capturing = false;
  int rc = na_capturing(st, &capturing);
  if (rc != PDCS_OK) return rc;
  NaScratch* s = nullptr;
  int dev = 0;
  rc = na_scratch(capturing, &s, &dev);
  if (rc != PDCS_OK) return rc;
  if (!na_device_ptr(row_ptr, dev) || !na_device_ptr(y, dev) ||
      (n > 0 && (!na_device_ptr(col_idx, dev) || !na_device_ptr(val, dev) ||
                 !na_device_ptr(x, dev))))
    return na_fail(PDCS_ERR_INVALID,
                   "pdcs_spmv_noalloc: every array must be device memory of the current device");
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    sms = 148;
  // the chunk count is known only on the device: 16 CTAs per SM stride over
  // the short rows and then the chunks
  const int64_t blocks = (int64_t)sms * 16;
  k_na_scan<<<1, kNaScanThreads, 0, st>>>(row_ptr, m, s);
  k_na_spmv<<<(unsigned)blocks, 256, 0, st>>>(row_ptr, col_idx, val, x, y, m, s);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(PDCS_ERR_CUDA, cudaGetErrorString(e));
  return PDCS_OK;
}

extern "C" int pdcs_spmv_noalloc_status(void* cuda_stream, int64_t* rejected) {
  if (!rejected) return na_fail(PDCS_ERR_INVALID, "pdcs_spmv_noalloc_status: NULL output");
  *rejected = 0;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  bool capturing = false;
  int rc = na_capturing(st, &capturing);
  if (rc != PDCS_OK) return rc;
  if (capturing)
    return na_fail(PDCS_ERR_INVALID,
                   "pdcs_spmv_noalloc_status: synchronises its stream, which is being captured");
  NaScratch* s = nullptr;
  int dev = 0;
  rc = na_scratch(false, &s, &dev);
  if (rc != PDCS_OK) return rc;
  unsigned int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, &s->status.rejected, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(&s->status.rejected, 0, sizeof(h), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return na_fail(PDCS_ERR_CUDA, cudaGetErrorString(e));
  *rejected = (int64_t)h;
  return PDCS_OK;
}
