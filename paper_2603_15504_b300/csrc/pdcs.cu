// Host side of the PDCS C ABI (include/pdcs.h): problem set-up on the device,
// the captured-graph solve loop, checkpoint / resume, and result unscaling.
//
// Solve loop (PDCS note, Algorithm 1 inside Algorithm 2): one CUDA graph per
// check period, relaunched by the host until the device status leaves
// "running":
//   period_begin
//   WHILE attempts needed:        Function 1 attempt + (if accepted) Halpern step
//   [gated on a completed period] check: average candidate, KKT statistics,
//   WHILE bisection unfinished:   Algorithm 3 probes for both candidates
//   decide / copy / refresh products / end of period
// The WHILE nodes are CUDA conditional graph nodes whose condition is written
// by the last kernel of each body, so the loop runs without host round trips;
// every loop has a hard per-launch cap.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/pdcs.h"
#include "common.cuh"
#include "cones.cuh"
#include "iterate.cuh"
#include "setup.cuh"
#include "spmv.cuh"
#include "batch.cuh"

namespace pdcs {

thread_local std::string g_last_error;

struct Fail {
  int code;
  std::string msg;
};

static void cuda_check(cudaError_t e, const char* what, int line) {
  if (e != cudaSuccess) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s failed (line %d): %s", what, line, cudaGetErrorString(e));
    throw Fail{e == cudaErrorMemoryAllocation ? PDCS_ERR_NOMEM : PDCS_ERR_CUDA, buf};
  }
}
#define CK(call) cuda_check((call), #call, __LINE__)

static void invalid(const std::string& msg) { throw Fail{PDCS_ERR_INVALID, msg}; }

// Owner of every device allocation of a handle.
struct Arena {
  std::vector<void*> ptrs;
  template <typename T>
  T* alloc(int64_t count) {
    void* p = nullptr;
    const size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(T);
    CK(cudaMalloc(&p, bytes));
    ptrs.push_back(p);
    return (T*)p;
  }
  void release(void* p) {
    for (auto& q : ptrs)
      if (q == p) { cudaFree(q); q = nullptr; }
  }
  ~Arena() {
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }
};

template <typename T>
static void copy_in(T* dst, const T* src, int64_t count, cudaStream_t st) {
  if (count <= 0) return;
  CK(cudaMemcpyAsync(dst, src, (size_t)count * sizeof(T), cudaMemcpyDefault, st));
}

template <typename T>
static std::vector<T> to_host(const T* dptr, int64_t count, cudaStream_t st) {
  std::vector<T> h((size_t)std::max<int64_t>(count, 0));
  if (count > 0) CK(cudaMemcpyAsync(h.data(), dptr, (size_t)count * sizeof(T), cudaMemcpyDefault, st));
  CK(cudaStreamSynchronize(st));
  return h;
}

static int ew_grid(int64_t n) {
  const int64_t b = (n + kEwThreads - 1) / kEwThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 148 * 4));
}
static int warp_grid(int64_t rows) {
  const int64_t b = (rows * 32 + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 148 * 16));
}

// ----------------------------------------------------------- SpMV plans
struct SpmvPlan {
  SpmvTask* tasks = nullptr;
  int ntasks = 0;
  double* partial = nullptr;
  unsigned int* counters = nullptr;
  int32_t* runlen = nullptr;  // per row: length of the leading column run (see runs_first)
  int64_t run_nnz = 0;        // nonzeros whose column index the products do not read
  int64_t run_rows = 0;       // rows whose run length (and first column) they read
};

// Rows of up to 4096 nonzeros are stored with their column run first: a row
// whose longest stretch of consecutive columns has at least kMinRun nonzeros is
// rotated (run, then the nonzeros before it, then those after it); the
// products then take the run's columns from its first index.  One warp per
// row; roff / rlen: offset of the run within the row and its length (0: the
// row is copied as it is).
__global__ void k_run_first(const int64_t* __restrict__ rp, const int32_t* __restrict__ roff,
                            const int32_t* __restrict__ rlen, int64_t rows,
                            const int32_t* __restrict__ ci, const double* __restrict__ v64,
                            const float* __restrict__ v32, int32_t* __restrict__ ci2,
                            double* __restrict__ w64, float* __restrict__ w32) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < rows; r += nwarps) {
    const int64_t s = rp[r], len = rp[r + 1] - s, L = rlen[r], off = roff[r];
    for (int64_t j = lane; j < len; j += 32) {
      int64_t src = j;
      if (L > 0) src = j < L ? off + j : (j - L < off ? j - L : j);
      ci2[s + j] = ci[s + src];
      w64[s + j] = v64[s + src];
      if (v32 != nullptr) w32[s + j] = v32[s + src];
    }
  }
}

// Shortest stretch of consecutive column indices worth a run descriptor.
constexpr int64_t kMinRun = 16;

// Longest stretch [a, b) of nonzeros in [s, e) with consecutive columns.
static void longest_run(const std::vector<int32_t>& ci, int64_t s, int64_t e, int64_t& a,
                        int64_t& b) {
  a = b = s;
  int64_t k = s;
  while (k < e) {
    int64_t j = k + 1;
    while (j < e && ci[j] == ci[j - 1] + 1) ++j;
    if (j - k > b - a) { a = k; b = j; }
    k = j;
  }
}

// Bin rows into SpMV tasks (see spmv.cuh): long rows (> 4096 nonzeros) split
// into kChunk-nonzero chunks; every other run of consecutive rows becomes a
// task whose kind follows its longest row: one thread per row when no row has
// more than 4 nonzeros, else one lane group per row (small_g lanes up to 512
// nonzeros, a warp beyond).  Rows of different lengths share tasks, so
// interleaved short and medium rows (the three rows of an exponential cone)
// do not fragment the plan into one-row tasks.
//
// Column runs (spmv.cuh): each long row's longest stretch of at least kMinRun
// nonzeros with consecutive columns is recorded in its chunks (ci: the column
// indices on the host); chunks wholly inside it read no index.
static SpmvPlan build_plan(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                           const std::vector<int32_t>& runlen, int32_t* runlen_dev, Arena& ar,
                           cudaStream_t st, int small_g) {
  const int64_t m = (int64_t)rp.size() - 1;
  std::vector<SpmvTask> tasks;
  int64_t run_nnz = 0, run_rows = 0;
  int64_t npart = 0;
  int ncnt = 0;
  int64_t r = 0;
  while (r < m) {
    if (rp[r + 1] - rp[r] > 4096) {
      const int64_t s = rp[r], e = rp[r + 1];
      int64_t ra, rb;
      longest_run(ci, s, e, ra, rb);
      if (rb - ra < kMinRun) ra = rb = 0;
      const int64_t nch = (e - s + kChunk - 1) / kChunk;
      for (int64_t k = 0; k < nch; ++k) {
        SpmvTask t{};
        t.kind = 2;
        t.counter = ncnt;
        t.nchunks = (int32_t)nch;
        t.a = r;
        t.b = k;
        t.c = s + k * kChunk;
        t.d = std::min(e, s + (k + 1) * kChunk);
        t.pbase = npart;
        t.ra = ra;
        t.rb = rb;
        t.col0 = rb > ra ? ci[ra] : 0;
        if (rb > ra && ra <= t.c && t.d <= rb) run_nnz += t.d - t.c;
        tasks.push_back(t);
      }
      npart += nch;
      ncnt += 1;
      ++r;
      continue;
    }
    // extend while the task stays within the limits of the kind it would
    // have: 256 rows (one thread each); 4 rows per lane group and 8,192
    // nonzeros (small groups); 32 rows and 16,384 nonzeros (warps) -- the
    // nonzero caps apply only beyond one row per group
    int64_t e = r, nnz = 0, maxlen = 0;
    while (e < m) {
      const int64_t len = rp[e + 1] - rp[e];
      if (len > 4096) break;
      const int64_t ml = std::max(maxlen, len), cnt = e - r + 1;
      int64_t lim_rows, lim_nnz, groups;
      if (ml <= 4) { lim_rows = 256; lim_nnz = INT64_MAX; groups = 1; }
      else if (ml <= 512) { groups = kSpmvThreads / small_g; lim_rows = 4 * groups; lim_nnz = 8192; }
      else { groups = kSpmvThreads / 32; lim_rows = 32; lim_nnz = 16384; }
      if (cnt > lim_rows) break;
      if (cnt > groups && nnz + len > lim_nnz) break;
      nnz += len;
      maxlen = ml;
      ++e;
    }
    SpmvTask t{};
    t.kind = maxlen <= 4 ? 0 : 1;
    t.g = maxlen <= 512 ? small_g : 32;
    t.a = r;
    t.b = e;
    if (t.kind == 1 && runlen_dev != nullptr) {
      int64_t rn = 0;
      for (int64_t q = r; q < e; ++q) rn += runlen[(size_t)q];
      if (rn > 0) {
        t.runs = 1;
        run_nnz += rn;
        run_rows += e - r;
      }
    }
    tasks.push_back(t);
    r = e;
  }
  SpmvPlan p;
  p.ntasks = (int)tasks.size();
  if (p.ntasks > 0) {
    p.tasks = ar.alloc<SpmvTask>(p.ntasks);
    CK(cudaMemcpyAsync(p.tasks, tasks.data(), tasks.size() * sizeof(SpmvTask), cudaMemcpyHostToDevice, st));
  }
  p.run_nnz = run_nnz;
  p.run_rows = run_rows;
  p.runlen = runlen_dev;
  p.partial = ar.alloc<double>(std::max<int64_t>(npart, 1));
  p.counters = ar.alloc<unsigned int>(std::max(ncnt, 1));
  CK(cudaMemsetAsync(p.counters, 0, sizeof(unsigned int) * std::max(ncnt, 1), st));
  CK(cudaStreamSynchronize(st));
  return p;
}

// Launch with, when pdl is set, the programmatic stream-serialization
// attribute (programmatic dependent launch: the kernel may be scheduled while
// its predecessor's last wave runs and waits in pdl_wait()).
template <typename... KArgs, typename... Args>
static void launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, bool pdl,
                     Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? at : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  CK(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
}

// V: matrix value type; x: the gathered vector (FP64, or its FP32 (hi, lo)
// shadow for FP32 values).
template <typename V, typename Out>
static void launch_spmv_out(const SpmvPlan& p, const int64_t* rp, const int32_t* ci, const V* vv,
                            const typename SpmvX<V>::type* x, const Out& out, const int* gate,
                            cudaStream_t st, KTimer* tm = nullptr, bool pdl = false) {
  if (p.ntasks == 0) return;
  launch_k(k_spmv<V, Out>, dim3(p.ntasks), dim3(kSpmvThreads), st, pdl,
           (const SpmvTask*)p.tasks, rp, ci, (const int32_t*)p.runlen, vv, x, out, p.partial,
           p.counters, gate, tm);
}

template <typename V>
static void launch_spmv(const SpmvPlan& p, const int64_t* rp, const int32_t* ci, const V* vv,
                        const typename SpmvX<V>::type* x, double* y, const int* gate,
                        cudaStream_t st, KTimer* tm = nullptr) {
  launch_spmv_out<V>(p, rp, ci, vv, x, StoreOut<double>{y}, gate, st, tm);
}

// FP32 (hi, lo) shadow of an FP64 vector (the gathered operand of FP32-value
// products).
__global__ void k_split(const double* __restrict__ v, float2* __restrict__ out, int64_t n,
                        const int* __restrict__ gate) {
  pdl_wait();
  pdl_trigger();
  if (gate != nullptr && *gate == 0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = split_ff(v[i]);
}

// ------------------------------------------------------------- cone tables
struct ConeTable {
  // SOC tiers by block dimension: <= 128 (32 threads), <= 4096 (256), <= 8192 (512),
  // larger blocks grid-wide (k_cone_soc_grid)
  int64_t* soc_s[3] = {nullptr, nullptr, nullptr};
  int32_t* soc_d[3] = {nullptr, nullptr, nullptr};
  int64_t nsoc[3] = {0, 0, 0};
  int64_t* big_s = nullptr;
  int64_t* big_d = nullptr;
  int64_t* big_o = nullptr;   // offset of each big block in big_b / big_bi
  double* big_b = nullptr;    // d_i^2 over the big blocks (in block order)
  double* big_bi = nullptr;   // 1 / d_i^2
  int nbig = 0;
  int64_t* exp_s = nullptr;
  uint8_t* exp_isd = nullptr;
  int64_t nexp = 0;
  double* dinv = nullptr;     // 1 / d over the whole side (exp blocks read it)
  // grid-wide kernel resources (shared by both tables)
  double* gpart = nullptr;
  GridSync gsync = {nullptr, nullptr};
  int big_grid = 0;
  KTimer* timers = nullptr;  // profiling slots (NULL: off)
  bool any() const { return nexp > 0 || nsoc[0] > 0 || nsoc[1] > 0 || nsoc[2] > 0 || nbig > 0; }
};

// r[i] = 1 / d[i] for i < n.
__global__ void k_reciprocal(const double* __restrict__ d, int64_t n, double* __restrict__ r) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    r[i] = 1.0 / d[i];
}

// b[i] = d[i]^2, bi[i] = 1 / d[i]^2 for i < n.
__global__ void k_square_scales(const double* __restrict__ d, int64_t n, double* __restrict__ b,
                                double* __restrict__ bi) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double di = d[i], r = 1.0 / di;
    b[i] = di * di;
    bi[i] = r * r;
  }
}

static const int kSocTierMax[3] = {128, 4096, 8192};

// Projection of one or two vectors onto a product of cones: the blocks are
// projected onto diag(e) K_b (dual = 0) or diag(e) K_b^* (dual = 1) with
// e = d, 1/d (inv) or 1 (d == NULL).  flip1 (two vectors, d != NULL): the
// second vector takes the other mode and the inverse scales (1 - dual,
// 1 - inv).  Zero / nonnegative blocks are handled by the producing kernels.
template <typename B>
static void project(const ConeTable& t, B* v0, B* v1, int nvec, const double* d, int inv, int dual,
                    const int* g0, const int* g1, cudaStream_t st, bool flip1 = false,
                    bool pdl = false) {
  KTimer* tm = t.timers;
  const int fl = flip1 ? 1 : 0;
  if (t.nexp > 0) {
    dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((t.nexp + 127) / 128, 148 * 8)), nvec);
    launch_k(k_cone_exp<B>, grid, dim3(128), st, pdl, v0, v1, (const int64_t*)t.exp_s,
             (const uint8_t*)t.exp_isd, t.nexp, d, (const double*)(d ? t.dinv : nullptr), inv, dual,
             fl, g0, g1, tm ? tm + TM_EXP : (KTimer*)nullptr);
  }
  KTimer* tsc = tm ? tm + TM_SOC_CTA : nullptr;
  if (t.nsoc[0] > 0)
    launch_k(k_cone_soc<B, 32, 4>, dim3((unsigned)t.nsoc[0], nvec), dim3(32), st, pdl, v0, v1,
             (const int64_t*)t.soc_s[0], (const int32_t*)t.soc_d[0], d, inv, fl, g0, g1, tsc);
  if (t.nsoc[1] > 0)
    launch_k(k_cone_soc<B, 256, 16>, dim3((unsigned)t.nsoc[1], nvec), dim3(256), st, pdl, v0, v1,
             (const int64_t*)t.soc_s[1], (const int32_t*)t.soc_d[1], d, inv, fl, g0, g1, tsc);
  if (t.nsoc[2] > 0)
    launch_k(k_cone_soc<B, 512, 16>, dim3((unsigned)t.nsoc[2], nvec), dim3(512), st, pdl, v0, v1,
             (const int64_t*)t.soc_s[2], (const int32_t*)t.soc_d[2], d, inv, fl, g0, g1, tsc);
  if (t.nbig > 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)t.big_grid);
    cfg.blockDim = dim3(512);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // squared scales of the target diag(e) K: e = d (b = d^2), 1/d (b = 1/d^2)
    // or 1 (no arrays)
    const double* bq = d == nullptr ? nullptr : (inv ? t.big_bi : t.big_b);
    const double* bqi = d == nullptr ? nullptr : (inv ? t.big_b : t.big_bi);
    KTimer* tg = tm ? tm + TM_SOC_GRID : (KTimer*)nullptr;
    const int64_t* bs = t.big_s;
    const int64_t* bd = t.big_d;
    const int64_t* bo = t.big_o;
    if (nvec == 2 && flip1 && d != nullptr)
      CK(cudaLaunchKernelEx(&cfg, k_cone_soc_grid<B, 2, true>, v0, v1, bs, bd, bo, t.nbig, bq, bqi,
                            g0, g1, t.gpart, t.gsync, tg));
    else if (nvec == 2)
      CK(cudaLaunchKernelEx(&cfg, k_cone_soc_grid<B, 2, false>, v0, v1, bs, bd, bo, t.nbig, bq,
                            bqi, g0, g1, t.gpart, t.gsync, tg));
    else
      CK(cudaLaunchKernelEx(&cfg, k_cone_soc_grid<B, 1, false>, v0, v1, bs, bd, bo, t.nbig, bq,
                            bqi, g0, g1, t.gpart, t.gsync, tg));
  }
}

}  // namespace pdcs

using namespace pdcs;

// ------------------------------------------------------------------ handle
struct SolverBase {
  virtual ~SolverBase() {}
  virtual void solve(const double* x0, const double* y0, double* x, double* y, double* s,
                     pdcs_result* res) = 0;
  virtual void resume(int64_t max_iter, double* x, double* y, double* s, pdcs_result* res) = 0;
  virtual void evaluate(const double* x, const double* y, pdcs_result* res) = 0;
  virtual void get_state(pdcs_state* st, double* x, double* y, double* x0, double* y0,
                         double* xs, double* ys) = 0;
  virtual void set_state(const pdcs_state* st, const double* x, const double* y,
                         const double* x0, const double* y0, const double* xs,
                         const double* ys) = 0;
  virtual void get_iterate(int which, double* x, double* y) = 0;
  virtual void get_profile(pdcs_profile* pr) = 0;
  virtual int get_kernel_times(double* sec, int64_t* launches, int cap) = 0;
  virtual int64_t get_trace(double* out, int64_t cap) = 0;
  int64_t m = 0, n = 0, nnz = 0;
};

struct BatchBase {
  virtual ~BatchBase() {}
  virtual void solve(double* x, double* y, double* s, pdcs_result* res, double* finish_s) = 0;
};

struct pdcs_handle {
  int device = 0;
  SolverBase* solver = nullptr;  // single problem
  BatchBase* batch = nullptr;    // batch of problems (pdcs_setup_batch)
};

namespace pdcs {

// MV: type of the stored matrix values used by the iteration (double: FP64
// mode; float: FP32 mode, with FP64 vectors and float-float products, and
// the FP64 values kept for the checks' products).  Vectors are FP64 (T).
template <typename MV>
struct Solver : SolverBase {
  using T = double;
  static constexpr bool kF32 = std::is_same<MV, float>::value;
  Arena ar;
  cudaStream_t st = nullptr;       // this handle's stream (captured graphs run here)
  cudaStream_t user_st = nullptr;  // caller's stream: work is ordered after it
  cudaStream_t st2 = nullptr;      // capture of conditional-node bodies
  pdcs_options opt;
  int64_t nb = 0;
  // matrix (scaled) and its transpose
  int64_t *rp = nullptr, *rpT = nullptr;
  int32_t *ci = nullptr, *ciT = nullptr;
  MV *vv = nullptr, *vvT = nullptr;        // values of the iteration's products
  double *vv64 = nullptr, *vvT64 = nullptr;  // FP64 values (== vv in FP64 mode)
  float2 *sx = nullptr, *sy = nullptr;     // FP32 mode: shadows of the gathered vectors
  double *gxt = nullptr, *gtyt = nullptr;  // FP32 mode: FP64 products of z at checks
  SpmvPlan planG, planGT;
  // problem data
  T *h = nullptr, *c = nullptr;
  double *lo = nullptr, *hi = nullptr, *d1 = nullptr, *d2 = nullptr;
  uint8_t *rk = nullptr, *ck = nullptr;
  ConeTable rows, cols;
  int64_t *row_rot = nullptr, *col_rot = nullptr;
  int64_t nrow_rot = 0, ncol_rot = 0;
  double eta0 = 1.0, omega0 = 1.0, h1 = 0, c1 = 0, hinf = 0, cinf = 0;
  double eta_fixed = 1.0;  // step of the non-adaptive mode: 1 / sqrt(||Ghat||_1 ||Ghat||_inf)
  bool infeas_on = false;
  // state
  T *x, *y, *xh, *yh, *x0, *y0, *gx, *gty, *gxh, *gtyh, *gx0, *gty0;
  T *xb, *yb, *gxb, *gtyb, *xc, *yc, *gxc, *gtyc;
  double *xs, *ys;
  double *tm[2], *tn[2], *um[2], *un[2], *px[2], *py[2];
  double* part = nullptr;
  double* trace = nullptr;
  double *obuf_n = nullptr, *obuf_m = nullptr, *obuf_s = nullptr;
  Ctl* ctl = nullptr;
  Ctl* hctl = nullptr;
  KTimer* timers = nullptr;             // TM_NUM slots (profile option)
  unsigned long long* gsync_count = nullptr;  // grid barrier of k_cone_soc_grid
  int* gsync_err = nullptr;             // set if a bounded barrier wait gave up
  double* gpart = nullptr;
  int big_grid = 0;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int64_t trace_rows = 0;
  int use_cond = 1;  // 0 in eager mode (kernels launched from the host, no graphs)
  bool pdl_ = false;  // programmatic dependent launches in the captured loop bodies
  // the dual step runs as the epilogue of G xhat when the rows are long
  // (16 nonzeros or more on average): there it costs the product nothing,
  // while on short rows the epilogue's registers cost the product occupancy
  bool dual_in_product = false;
  int64_t cone_rows = 0;  // rows whose cone is SOC or exponential
  int64_t nk_a = 0, nk_b = 0, nk_top = 0;  // kernel nodes: attempt body, probe body, top level
  int64_t eager_a = 0, eager_b = 0;        // attempt / probe bodies run by the eager loop
  int64_t graph_launches = 0;
  long long bodies_a0 = 0, bodies_b0 = 0;  // loop-body counters at the start of the call

  Prob<T> prob() const {
    Prob<T> p;
    p.m = m; p.n = n; p.nb = nb; p.h = h; p.c = c; p.lo = lo; p.hi = hi; p.d1 = d1; p.d2 = d2;
    p.rk = rk; p.ck = ck; p.tm = timers;
    return p;
  }

  ~Solver() override {
    if (st) cudaStreamSynchronize(st);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (hctl) cudaFreeHost(hctl);
    if (st2) cudaStreamDestroy(st2);
    if (st) cudaStreamDestroy(st);
  }

  // Make this handle's stream wait for work already queued on the caller's stream.
  void order_after_user() {
    if (!user_st) return;
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CK(cudaEventRecord(ev, user_st));
    CK(cudaStreamWaitEvent(st, ev, 0));
    CK(cudaEventDestroy(ev));
  }

  // -------------------------------------------------------------- set-up
  // Column layout of a block-diagonal batch: each segment is one instance's
  // columns [off, end): nb boxed columns, then its column cones.
  struct ColSeg {
    int64_t off, nb, end;
    std::vector<pdcs_cone> cones;
  };

  // segs == NULL: the columns are nb_in boxed columns then the cones cc, and
  // lb / ub hold nb_in entries.  Otherwise the segments give the layout and
  // lb / ub hold n0 entries (read only at boxed columns).
  void setup(int64_t m0, int64_t n0, const int64_t* rp_in, const int32_t* ci_in, const double* v_in,
             const double* h_in, const double* c_in, int64_t nb_in, const double* lb,
             const double* ub, const std::vector<pdcs_cone>& rc, const std::vector<pdcs_cone>& cc,
             const pdcs_options& o, cudaStream_t stream, const std::vector<ColSeg>* segs = nullptr) {
    user_st = stream;
    opt = o;
    m = m0;
    n = n0;
    nb = nb_in;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking));
    order_after_user();
    // ---- row pointer to host for validation and plans
    std::vector<int64_t> hrp((size_t)m + 1);
    CK(cudaMemcpy(hrp.data(), rp_in, sizeof(int64_t) * (m + 1), cudaMemcpyDefault));
    if (hrp[0] != 0) invalid("row_ptr[0] must be 0");
    for (int64_t r = 0; r < m; ++r)
      if (hrp[r + 1] < hrp[r]) invalid("row_ptr must be nondecreasing");
    nnz = hrp[m];
    if (nnz > INT64_C(2000000000)) invalid("nnz too large");
    if (nnz > 0 && (!ci_in || !v_in)) invalid("col_idx and val are required");
    int64_t* drp = ar.alloc<int64_t>(m + 1);
    int32_t* dci = ar.alloc<int32_t>(nnz);
    double* dv = ar.alloc<double>(nnz);
    copy_in(drp, rp_in, m + 1, st);
    copy_in(dci, ci_in, nnz, st);
    copy_in(dv, v_in, nnz, st);
    double* dh = ar.alloc<double>(m);
    double* dc = ar.alloc<double>(n);
    copy_in(dh, h_in, m, st);
    copy_in(dc, c_in, n, st);
    unsigned int* derr = ar.alloc<unsigned int>(1);
    CK(cudaMemsetAsync(derr, 0, sizeof(unsigned int), st));
    if (m > 0) k_validate_csr<<<warp_grid(m), 256, 0, st>>>(drp, dci, dv, m, n, nnz, derr);
    k_check_finite<<<ew_grid(m), 256, 0, st>>>(dh, m, 16u, derr);
    k_check_finite<<<ew_grid(n), 256, 0, st>>>(dc, n, 32u, derr);
    CK(cudaGetLastError());
    unsigned int herr = 0;
    CK(cudaMemcpyAsync(&herr, derr, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr & 1u) invalid("row_ptr entries out of range");
    if (herr & 2u) invalid("column index out of range");
    if (herr & 4u) invalid("column indices must be strictly increasing within each row");
    if (herr & 8u) invalid("non-finite matrix value");
    if (herr & 16u) invalid("non-finite entry in h");
    if (herr & 32u) invalid("non-finite entry in c");
    const int64_t nbl = segs ? n : nb;  // length of the bound arrays
    std::vector<std::pair<int64_t, int64_t>> boxes;  // boxed column ranges
    if (segs) {
      for (const auto& sg : *segs) boxes.push_back({sg.off, sg.off + sg.nb});
    } else {
      boxes.push_back({0, nb});
    }
    std::vector<double> hlo((size_t)nbl), hhi((size_t)nbl);
    if (nbl > 0) {
      if (!lb || !ub) invalid("lb and ub are required when nb > 0");
      CK(cudaMemcpy(hlo.data(), lb, sizeof(double) * nbl, cudaMemcpyDefault));
      CK(cudaMemcpy(hhi.data(), ub, sizeof(double) * nbl, cudaMemcpyDefault));
      for (const auto& bx : boxes)
        for (int64_t j = bx.first; j < bx.second; ++j) {
          if (std::isnan(hlo[j]) || std::isnan(hhi[j]) || hlo[j] > hhi[j]) invalid("bounds must satisfy lb <= ub");
          if (hlo[j] == INFINITY || hhi[j] == -INFINITY) invalid("infinite bound on the wrong side");
        }
    }
    // ---- cone layout and RSOC pairs
    std::vector<int64_t> rpairs, cpairs;
    std::vector<uint8_t> hrk((size_t)m), hck((size_t)n);
    std::vector<std::vector<std::pair<int64_t, int32_t>>> rsoc(3), csoc(3);
    std::vector<std::pair<int64_t, int64_t>> rbig, cbig;
    std::vector<int64_t> rexp, cexp;
    std::vector<uint8_t> rexpd, cexpd;
    layout(rc, 0, m, true, hrk, rpairs, rsoc, rbig, rexp, rexpd);
    if (segs) {
      for (const auto& sg : *segs) {
        for (int64_t j = sg.off; j < sg.off + sg.nb; ++j) hck[j] = CK_BOX;
        layout(sg.cones, sg.off + sg.nb, sg.end, false, hck, cpairs, csoc, cbig, cexp, cexpd);
      }
    } else {
      for (int64_t j = 0; j < nb; ++j) hck[j] = CK_BOX;
      layout(cc, nb, n, false, hck, cpairs, csoc, cbig, cexp, cexpd);
    }
    // ---- RSOC reformulation on rows
    if (!rpairs.empty()) {
      merge_row_pairs(hrp, drp, dci, dv, rpairs, m);
      row_rot = ar.alloc<int64_t>((int64_t)rpairs.size());
      nrow_rot = (int64_t)rpairs.size();
      copy_in(row_rot, rpairs.data(), nrow_rot, st);
      k_rotate_pairs<<<ew_grid(nrow_rot), 256, 0, st>>>(dh, row_rot, nrow_rot);
    }
    // ---- transpose
    std::vector<int64_t> hrpT;
    int64_t* drpT = nullptr;
    int32_t* dciT = nullptr;
    double* dvT = nullptr;
    transpose(hrp, drp, dci, dv, m, n, hrpT, drpT, dciT, dvT);
    // ---- RSOC reformulation on columns: row pairs of the transpose
    if (!cpairs.empty()) {
      merge_row_pairs(hrpT, drpT, dciT, dvT, cpairs, n);
      col_rot = ar.alloc<int64_t>((int64_t)cpairs.size());
      ncol_rot = (int64_t)cpairs.size();
      copy_in(col_rot, cpairs.data(), ncol_rot, st);
      k_rotate_pairs<<<ew_grid(ncol_rot), 256, 0, st>>>(dc, col_rot, ncol_rot);
      ar.release(drp); ar.release(dci); ar.release(dv);
      transpose(hrpT, drpT, dciT, dvT, n, m, hrp, drp, dci, dv);
    }
    nnz = hrp[m];
    dual_in_product = nnz >= 16 * m;
    // ---- scaling (Ruiz + Pock-Chambolle), Sec. 2.6
    d1 = ar.alloc<double>(m);
    d2 = ar.alloc<double>(n);
    k_fill<double><<<ew_grid(m), 256, 0, st>>>(d1, m, 1.0);
    k_fill<double><<<ew_grid(n), 256, 0, st>>>(d2, n, 1.0);
    if (opt.use_preconditioner && m > 0) {
      double* rn = ar.alloc<double>(m);
      double* cn = ar.alloc<double>(n);
      for (int it = 0; it < opt.ruiz_iters; ++it) {
        k_row_norms<<<warp_grid(m), 256, 0, st>>>(drp, dci, dv, m, d1, d2, 0, 0, 1.0, rn);
        k_row_norms<<<warp_grid(n), 256, 0, st>>>(drpT, dciT, dvT, n, d2, d1, 1, 0, 1.0, cn);
        k_scale_update<<<ew_grid(m), 256, 0, st>>>(d1, rn, m);
        k_scale_update<<<ew_grid(n), 256, 0, st>>>(d2, cn, n);
      }
      if (opt.pc_alpha >= 0) {
        k_row_norms<<<warp_grid(m), 256, 0, st>>>(drp, dci, dv, m, d1, d2, 0, 1, opt.pc_alpha, rn);
        k_row_norms<<<warp_grid(n), 256, 0, st>>>(drpT, dciT, dvT, n, d2, d1, 1, 1, 2.0 - opt.pc_alpha, cn);
        k_scale_update<<<ew_grid(m), 256, 0, st>>>(d1, rn, m);
        k_scale_update<<<ew_grid(n), 256, 0, st>>>(d2, cn, n);
      }
      CK(cudaStreamSynchronize(st));
      ar.release(rn);
      ar.release(cn);
    }
    unsigned long long* amax = ar.alloc<unsigned long long>(1);
    CK(cudaMemsetAsync(amax, 0, sizeof(unsigned long long), st));
    rp = drp; ci = dci; rpT = drpT; ciT = dciT;
    vv64 = ar.alloc<double>(nnz);
    vvT64 = ar.alloc<double>(nnz);
    if (m > 0) {
      k_apply_scale<double><<<warp_grid(m), 256, 0, st>>>(drp, dci, dv, m, d1, d2, 0, vv64, amax);
      k_apply_scale<double><<<warp_grid(n), 256, 0, st>>>(drpT, dciT, dvT, n, d2, d1, 1, vvT64, nullptr);
    }
    if constexpr (kF32) {
      // the same scaled values rounded to FP32 (G and G^T stay transposes)
      vv = ar.alloc<float>(nnz);
      vvT = ar.alloc<float>(nnz);
      if (m > 0) {
        k_apply_scale<float><<<warp_grid(m), 256, 0, st>>>(drp, dci, dv, m, d1, d2, 0, vv, nullptr);
        k_apply_scale<float><<<warp_grid(n), 256, 0, st>>>(drpT, dciT, dvT, n, d2, d1, 1, vvT, nullptr);
      }
    } else {
      vv = vv64;
      vvT = vvT64;
    }
    double* sh_ = ar.alloc<double>(m);
    double* sc_ = ar.alloc<double>(n);
    k_scale_vec<<<ew_grid(m), 256, 0, st>>>(dh, d1, m, 0, sh_);
    k_scale_vec<<<ew_grid(n), 256, 0, st>>>(dc, d2, n, 0, sc_);
    h = ar.alloc<T>(m);
    c = ar.alloc<T>(n);
    k_convert<double, T><<<ew_grid(m), 256, 0, st>>>(sh_, h, m);
    k_convert<double, T><<<ew_grid(n), 256, 0, st>>>(sc_, c, n);
    lo = ar.alloc<double>(nbl);
    hi = ar.alloc<double>(nbl);
    if (nbl > 0) {
      double* tmp = ar.alloc<double>(nbl);
      copy_in(tmp, hlo.data(), nbl, st);
      k_scale_vec<<<ew_grid(nbl), 256, 0, st>>>(tmp, d2, nbl, 1, lo);
      CK(cudaStreamSynchronize(st));
      copy_in(tmp, hhi.data(), nbl, st);
      k_scale_vec<<<ew_grid(nbl), 256, 0, st>>>(tmp, d2, nbl, 1, hi);
      CK(cudaStreamSynchronize(st));
      ar.release(tmp);
    }
    double* nrm = ar.alloc<double>(16);
    k_vec_norms<<<1, 1024, 0, st>>>(sh_, m, d1, nrm);
    k_vec_norms<<<1, 1024, 0, st>>>(sc_, n, d2, nrm + 4);
    {
      // largest row / column absolute sums of Ghat (the non-adaptive step)
      double* rs = ar.alloc<double>(std::max<int64_t>(m, 1));
      double* cs = ar.alloc<double>(n);
      if (m > 0) k_row_norms<<<warp_grid(m), 256, 0, st>>>(drp, dci, dv, m, d1, d2, 0, 1, 1.0, rs);
      k_row_norms<<<warp_grid(n), 256, 0, st>>>(drpT, dciT, dvT, n, d2, d1, 1, 1, 1.0, cs);
      k_vec_norms<<<1, 1024, 0, st>>>(rs, m, nullptr, nrm + 8);
      k_vec_norms<<<1, 1024, 0, st>>>(cs, n, nullptr, nrm + 12);
      CK(cudaStreamSynchronize(st));
      ar.release(rs);
      ar.release(cs);
    }
    CK(cudaGetLastError());
    double hn[16];
    unsigned long long hamax = 0;
    CK(cudaMemcpyAsync(hn, nrm, sizeof(hn), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&hamax, amax, sizeof(hamax), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    h1 = hn[0]; hinf = hn[2]; c1 = hn[4]; cinf = hn[6];
    const double nh2 = std::sqrt(hn[1]), nc2 = std::sqrt(hn[5]);
    omega0 = (nc2 > 1e-10 && nh2 > 1e-10) ? nc2 / nh2 : 1.0;  // Sec. 2.5
    double gmax;
    std::memcpy(&gmax, &hamax, sizeof(double));
    eta0 = gmax > 0 ? 1.0 / gmax : 1.0;  // Algorithm 1: 1 / ||G||_inf
    eta_fixed = (hn[10] > 0 && hn[14] > 0) ? 1.0 / std::sqrt(hn[14] * hn[10]) : 1.0;
    infeas_on = opt.eps_primal_infeasible_low_acc > 0 || opt.eps_dual_infeasible_low_acc > 0 ||
                opt.eps_primal_infeasible_high_acc > 0 || opt.eps_dual_infeasible_high_acc > 0;
    ar.release(dv); ar.release(dvT); ar.release(dh); ar.release(dc);
    ar.release(sh_); ar.release(sc_); ar.release(nrm); ar.release(amax); ar.release(derr);
    // ---- kinds, cone tables, plans
    rk = ar.alloc<uint8_t>(m);
    ck = ar.alloc<uint8_t>(n);
    copy_in(rk, hrk.data(), m, st);
    cone_rows = 0;
    for (int64_t i = 0; i < m; ++i) cone_rows += hrk[i] >= RK_SOC;
    copy_in(ck, hck.data(), n, st);
    fill_table(rows, rsoc, rbig, rexp, rexpd, d1, m);
    fill_table(cols, csoc, cbig, cexp, cexpd, d2, n);
    // four lanes per row of up to 512 nonzeros in both precisions (FP32
    // values: Gt yhat on the portfolio, rows of ~200 nonzeros, 63 us with
    // four lanes against 114 us with eight, A/B on one B300)
    const int small_g = 4;
    {
      // column indices on the host for the run detection of the plans; rows
      // of up to 4096 nonzeros are then stored run first (k_run_first)
      std::vector<int32_t> hci((size_t)nnz), hrl;
      if (nnz > 0) CK(cudaMemcpy(hci.data(), ci, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
      int32_t* rl = runs_first(hrp, hci, ci, vv64, kF32 ? (float*)vv : nullptr, hrl);
      planG = build_plan(hrp, hci, hrl, rl, ar, st, small_g);
      if (nnz > 0) CK(cudaMemcpy(hci.data(), ciT, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
      rl = runs_first(hrpT, hci, ciT, vvT64, kF32 ? (float*)vvT : nullptr, hrl);
      planGT = build_plan(hrpT, hci, hrl, rl, ar, st, small_g);
    }
    alloc_state();
    if (opt.eager) {
      use_cond = 0;
      count_eager();
    } else {
      pdl_ = opt.overlap_launches != 0;
      capture();
    }
  }

  // Store every row of up to 4096 nonzeros whose longest column run has at
  // least kMinRun nonzeros with that run first (k_run_first), in the column
  // indices and in both value arrays (v32 may be NULL); the long rows keep
  // their order (their chunks use the run in place).  hci: the column indices
  // before the rotation.  Returns the device array of run lengths (NULL when
  // no row qualifies) and fills hrl with it.
  int32_t* runs_first(const std::vector<int64_t>& hrp, const std::vector<int32_t>& hci,
                      int32_t* dci, double* v64, float* v32, std::vector<int32_t>& hrl) {
    const int64_t rows = (int64_t)hrp.size() - 1;
    hrl.assign((size_t)std::max<int64_t>(rows, 0), 0);
    std::vector<int32_t> hoff((size_t)std::max<int64_t>(rows, 0), 0);
    bool any = false;
    for (int64_t r = 0; r < rows; ++r) {
      const int64_t len = hrp[r + 1] - hrp[r];
      if (len > 4096 || len < kMinRun) continue;
      int64_t a, b;
      longest_run(hci, hrp[r], hrp[r + 1], a, b);
      if (b - a < kMinRun) continue;
      hrl[(size_t)r] = (int32_t)(b - a);
      hoff[(size_t)r] = (int32_t)(a - hrp[r]);
      any = true;
    }
    if (!any) return nullptr;
    int32_t* drl = ar.alloc<int32_t>(rows);
    int32_t* doff = ar.alloc<int32_t>(rows);
    copy_in(drl, hrl.data(), rows, st);
    copy_in(doff, hoff.data(), rows, st);
    const int64_t nz = hrp[rows];
    int32_t* c2 = ar.alloc<int32_t>(nz);
    double* w64 = ar.alloc<double>(nz);
    float* w32 = v32 ? ar.alloc<float>(nz) : nullptr;
    int64_t* drp_ = ar.alloc<int64_t>(rows + 1);
    copy_in(drp_, hrp.data(), rows + 1, st);
    k_run_first<<<warp_grid(rows), 256, 0, st>>>(drp_, doff, drl, rows, dci, v64, v32, c2, w64, w32);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(dci, c2, sizeof(int32_t) * nz, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(v64, w64, sizeof(double) * nz, cudaMemcpyDeviceToDevice, st));
    if (v32) CK(cudaMemcpyAsync(v32, w32, sizeof(float) * nz, cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    ar.release(c2);
    ar.release(w64);
    if (w32) ar.release(w32);
    ar.release(drp_);
    ar.release(doff);
    return drl;
  }

  // Per-element kinds and cone tables from an ordered cone list starting at off.
  void layout(const std::vector<pdcs_cone>& cl, int64_t off, int64_t end, bool is_row,
              std::vector<uint8_t>& kind, std::vector<int64_t>& pairs,
              std::vector<std::vector<std::pair<int64_t, int32_t>>>& soc,
              std::vector<std::pair<int64_t, int64_t>>& big, std::vector<int64_t>& ex,
              std::vector<uint8_t>& exd) {
    for (const auto& cn : cl) {
      const int64_t d = cn.dim;
      if (off + d > end) invalid("cone dimensions exceed the vector length");
      switch (cn.type) {
        case PDCS_CONE_ZERO:
          for (int64_t i = 0; i < d; ++i) kind[off + i] = is_row ? (uint8_t)RK_FREE : (uint8_t)CK_ZERO;
          break;
        case PDCS_CONE_NONNEG:
          for (int64_t i = 0; i < d; ++i) kind[off + i] = is_row ? (uint8_t)RK_NONNEG : (uint8_t)CK_NONNEG;
          break;
        case PDCS_CONE_RSOC:
        case PDCS_CONE_SOC: {
          if (cn.type == PDCS_CONE_RSOC) pairs.push_back(off);
          for (int64_t i = 0; i < d; ++i) kind[off + i] = is_row ? (uint8_t)RK_SOC : (uint8_t)CK_SOC;
          if (d > kSocTierMax[2]) {
            big.push_back({off, d});
          } else {
            const int tier = d <= kSocTierMax[0] ? 0 : (d <= kSocTierMax[1] ? 1 : 2);
            soc[tier].push_back({off, (int32_t)d});
          }
          break;
        }
        case PDCS_CONE_EXP:
        case PDCS_CONE_DUAL_EXP: {
          const bool de = cn.type == PDCS_CONE_DUAL_EXP;
          for (int64_t i = 0; i < 3; ++i)
            kind[off + i] = is_row ? (uint8_t)(de ? RK_DEXP : RK_EXP) : (uint8_t)(de ? CK_DEXP : CK_EXP);
          ex.push_back(off);
          exd.push_back(de ? 1 : 0);
          break;
        }
        default:
          invalid("unknown cone type");
      }
      off += d;
    }
  }

  void fill_table(ConeTable& t, const std::vector<std::vector<std::pair<int64_t, int32_t>>>& soc,
                  const std::vector<std::pair<int64_t, int64_t>>& big,
                  const std::vector<int64_t>& ex, const std::vector<uint8_t>& exd,
                  const double* dscale, int64_t dlen) {
    t.nbig = (int)big.size();
    if (t.nbig > 0) {
      std::vector<int64_t> bs, bd, bo;
      int64_t tot = 0;
      for (auto& pr : big) {
        bs.push_back(pr.first);
        bd.push_back(pr.second);
        bo.push_back(tot);
        tot += pr.second;
      }
      t.big_s = ar.alloc<int64_t>(t.nbig);
      t.big_d = ar.alloc<int64_t>(t.nbig);
      t.big_o = ar.alloc<int64_t>(t.nbig);
      copy_in(t.big_s, bs.data(), (int64_t)t.nbig, st);
      copy_in(t.big_d, bd.data(), (int64_t)t.nbig, st);
      copy_in(t.big_o, bo.data(), (int64_t)t.nbig, st);
      t.big_b = ar.alloc<double>(tot);
      t.big_bi = ar.alloc<double>(tot);
      for (int b = 0; b < t.nbig; ++b)
        k_square_scales<<<ew_grid(bd[b]), 256, 0, st>>>(dscale + bs[b], bd[b], t.big_b + bo[b],
                                                       t.big_bi + bo[b]);
      CK(cudaGetLastError());
      CK(cudaStreamSynchronize(st));
      if (!gsync_count) {
        int dev = 0, sms = 0, occ = 2, o = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        // one grid size for every variant (cooperative launches need all CTAs resident)
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_cone_soc_grid<T, 1, false>, 512, 0));
        occ = std::min(occ, o);
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_cone_soc_grid<T, 2, false>, 512, 0));
        occ = std::min(occ, o);
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_cone_soc_grid<double, 1, false>, 512, 0));
        occ = std::min(occ, o);
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_cone_soc_grid<double, 2, true>, 512, 0));
        occ = std::min(occ, o);
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_cone_soc_grid<double, 2, false>, 512, 0));
        occ = std::max(1, std::min(occ, o));
        big_grid = std::min(sms * occ, kMaxGridParts);
        gsync_count = ar.alloc<unsigned long long>(1);
        gsync_err = ar.alloc<int>(1);
        gpart = ar.alloc<double>(2 * kSgHalf * (int64_t)big_grid);
        CK(cudaMemsetAsync(gsync_count, 0, sizeof(unsigned long long), st));
        CK(cudaMemsetAsync(gsync_err, 0, sizeof(int), st));
      }
    }
    t.gpart = gpart;
    t.gsync = GridSync{gsync_count, gsync_err};
    t.big_grid = big_grid;
    for (int k = 0; k < 3; ++k) {
      t.nsoc[k] = (int64_t)soc[k].size();
      if (t.nsoc[k] == 0) continue;
      std::vector<int64_t> s;
      std::vector<int32_t> d;
      for (auto& pr : soc[k]) { s.push_back(pr.first); d.push_back(pr.second); }
      t.soc_s[k] = ar.alloc<int64_t>(t.nsoc[k]);
      t.soc_d[k] = ar.alloc<int32_t>(t.nsoc[k]);
      copy_in(t.soc_s[k], s.data(), t.nsoc[k], st);
      copy_in(t.soc_d[k], d.data(), t.nsoc[k], st);
      CK(cudaStreamSynchronize(st));
    }
    t.nexp = (int64_t)ex.size();
    if (t.nexp > 0 && dlen > 0) {
      // the exponential-cone kernels take e = d or 1/d per element: the
      // reciprocals once here instead of three FP64 divisions per projection
      t.dinv = ar.alloc<double>(dlen);
      k_reciprocal<<<ew_grid(dlen), 256, 0, st>>>(dscale, dlen, t.dinv);
      CK(cudaGetLastError());
    }
    if (t.nexp > 0) {
      t.exp_s = ar.alloc<int64_t>(t.nexp);
      t.exp_isd = ar.alloc<uint8_t>(t.nexp);
      copy_in(t.exp_s, ex.data(), t.nexp, st);
      copy_in(t.exp_isd, exd.data(), t.nexp, st);
    }
    CK(cudaStreamSynchronize(st));
  }

  // Merge each listed row pair of a CSR (host row pointer hrp, device arrays)
  // into ((r_s + r_{s+1})/sqrt2, (r_s - r_{s+1})/sqrt2); replaces the arrays.
  void merge_row_pairs(std::vector<int64_t>& hrp, int64_t*& drp, int32_t*& dci, double*& dv,
                       const std::vector<int64_t>& pairs, int64_t rws) {
    const int64_t np = (int64_t)pairs.size();
    int64_t* dp = ar.alloc<int64_t>(np);
    int64_t* dlen = ar.alloc<int64_t>(np);
    copy_in(dp, pairs.data(), np, st);
    k_pair_union_len<<<ew_grid(np), 256, 0, st>>>(drp, dci, dp, np, dlen);
    CK(cudaGetLastError());
    std::vector<int64_t> len = to_host(dlen, np, st);
    std::vector<int64_t> rl((size_t)rws);
    for (int64_t r = 0; r < rws; ++r) rl[r] = hrp[r + 1] - hrp[r];
    std::vector<int64_t> pair_of((size_t)rws, -1);
    for (int64_t b = 0; b < np; ++b) {
      rl[pairs[b]] = len[b];
      rl[pairs[b] + 1] = len[b];
      pair_of[pairs[b]] = b;
      pair_of[pairs[b] + 1] = -2;
    }
    std::vector<int64_t> nrp((size_t)rws + 1, 0);
    for (int64_t r = 0; r < rws; ++r) nrp[r + 1] = nrp[r] + rl[r];
    const int64_t nnz2 = nrp[rws];
    int64_t* dnrp = ar.alloc<int64_t>(rws + 1);
    int32_t* dnci = ar.alloc<int32_t>(nnz2);
    double* dnv = ar.alloc<double>(nnz2);
    int64_t* dpo = ar.alloc<int64_t>(rws);
    copy_in(dnrp, nrp.data(), rws + 1, st);
    copy_in(dpo, pair_of.data(), rws, st);
    k_pair_merge<<<warp_grid(rws), 256, 0, st>>>(drp, dci, dv, rws, dnrp, dnci, dnv, dpo);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    ar.release(drp); ar.release(dci); ar.release(dv); ar.release(dp); ar.release(dlen); ar.release(dpo);
    drp = dnrp; dci = dnci; dv = dnv;
    hrp.swap(nrp);
  }

  // CSR (rws x cls) -> CSR of the transpose, entries sorted by row index.
  void transpose(const std::vector<int64_t>& hrp_, const int64_t* drp, const int32_t* dci,
                 const double* dv, int64_t rws, int64_t cls, std::vector<int64_t>& hrpT,
                 int64_t*& drpT, int32_t*& dciT, double*& dvT) {
    const int64_t nz = hrp_[rws];
    unsigned long long* cnt = ar.alloc<unsigned long long>(cls);
    CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * std::max<int64_t>(cls, 1), st));
    if (nz > 0) k_col_count<<<ew_grid(nz), 256, 0, st>>>(dci, nz, cnt);
    CK(cudaGetLastError());
    std::vector<unsigned long long> hc = to_host(cnt, cls, st);
    hrpT.assign((size_t)cls + 1, 0);
    for (int64_t j = 0; j < cls; ++j) hrpT[j + 1] = hrpT[j] + (int64_t)hc[j];
    drpT = ar.alloc<int64_t>(cls + 1);
    dciT = ar.alloc<int32_t>(nz);
    dvT = ar.alloc<double>(nz);
    copy_in(drpT, hrpT.data(), cls + 1, st);
    copy_in((int64_t*)cnt, hrpT.data(), cls, st);  // cursors start at the segment offsets
    if (rws > 0) k_transpose_scatter<<<warp_grid(rws), 256, 0, st>>>(drp, dci, dv, rws, cnt, dciT, dvT);
    if (cls > 0) k_segment_sort<<<(unsigned)std::min<int64_t>(cls, 148 * 32), 256, 0, st>>>(drpT, dciT, dvT, cls);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    ar.release(cnt);
  }

  void alloc_state() {
    T** vn[] = {&x, &xh, &x0, &gty, &gtyh, &gty0, &xb, &gtyb, &xc, &gtyc};
    for (auto p : vn) *p = ar.alloc<T>(n);
    T** vm[] = {&y, &yh, &y0, &gx, &gxh, &gx0, &yb, &gxb, &yc, &gxc};
    for (auto p : vm) *p = ar.alloc<T>(m);
    xs = ar.alloc<double>(n);
    ys = ar.alloc<double>(m);
    for (int k = 0; k < 2; ++k) {
      tm[k] = ar.alloc<double>(m); um[k] = ar.alloc<double>(m); py[k] = ar.alloc<double>(m);
      tn[k] = ar.alloc<double>(n); un[k] = ar.alloc<double>(n); px[k] = ar.alloc<double>(n);
    }
    if constexpr (kF32) {
      sx = ar.alloc<float2>(n);
      sy = ar.alloc<float2>(std::max<int64_t>(m, 1));
      gxt = ar.alloc<double>(std::max<int64_t>(m, 1));
      gtyt = ar.alloc<double>(n);
    } else {
      gxt = gx;
      gtyt = gty;
    }
    const int g = ew_grid(std::max(m, n));
    part = ar.alloc<double>((int64_t)g * kStatK * 2 + 64);
    ctl = ar.alloc<Ctl>(1);
    CK(cudaMallocHost(&hctl, sizeof(Ctl)));
    std::memset(hctl, 0, sizeof(Ctl));
    obuf_n = ar.alloc<double>(n);
    obuf_m = ar.alloc<double>(m);
    obuf_s = ar.alloc<double>(m);
    if (opt.trace_capacity > 0) trace = ar.alloc<double>((int64_t)opt.trace_capacity * PDCS_TRACE_FIELDS);
    if (opt.profile) {
      timers = ar.alloc<KTimer>(TM_NUM);
      reset_timers();
    }
    rows.timers = timers;
    cols.timers = timers;
  }

  void reset_timers() {
    if (!timers) return;
    KTimer z[TM_NUM];
    for (auto& t : z) { t.start = ~0ull; t.total_ns = 0; t.ticket = 0; t.launches = 0; }
    CK(cudaMemcpyAsync(timers, z, sizeof(z), cudaMemcpyHostToDevice, st));
  }

  int get_kernel_times(double* sec, int64_t* launches, int cap) override {
    if (!timers) return 0;
    KTimer z[TM_NUM];
    CK(cudaMemcpyAsync(z, timers, sizeof(z), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int k = std::min(cap, (int)TM_NUM);
    for (int i = 0; i < k; ++i) {
      if (sec) sec[i] = 1e-9 * (double)z[i].total_ns;
      if (launches) launches[i] = z[i].launches;
    }
    return k;
  }

  void get_profile(pdcs_profile* pr) override {
    std::memset(pr, 0, sizeof(*pr));
    // values + column indices once, row pointers once, the gathered vector
    // (FP64 or its 8-byte FP32 pair) and the result once
    // (column indices only outside the chunks that lie in column runs)
    const double vb = (double)sizeof(MV);
    // (a row stored run first costs its run length and its first index)
    auto idx_bytes = [&](const SpmvPlan& pl) {
      return 4.0 * (double)(nnz - pl.run_nnz) + 8.0 * (double)pl.run_rows;
    };
    pr->g_bytes = (double)nnz * vb + idx_bytes(planG) + 8.0 * (double)(m + 1) + 8.0 * (double)(n + m);
    // the dual step in the product's epilogue: y, G x, h and the row kind
    // read, yhat written per row, G xhat - h on the cone rows
    if (dual_in_product) pr->g_bytes += (double)m * (4.0 * 8.0 + 1.0) + 8.0 * (double)cone_rows;
    pr->gt_bytes = (double)nnz * vb + idx_bytes(planGT) + 8.0 * (double)(n + 1) + 8.0 * (double)(n + m);
    pr->nnz_flops = 2.0 * (double)nnz;
    pr->graph_launches = graph_launches;
    if (use_cond)
      pr->kernel_launches = graph_launches * nk_top + (hctl->bodies_a - bodies_a0) * nk_a +
                            (hctl->bodies_b - bodies_b0) * nk_b;
    else
      pr->kernel_launches = graph_launches * nk_top + eager_a * nk_a + eager_b * nk_b;
    if (!timers) return;
    KTimer z[TM_NUM];
    CK(cudaMemcpyAsync(z, timers, sizeof(z), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    pr->g_launches = z[0].launches;
    pr->g_seconds = 1e-9 * (double)z[0].total_ns;
    pr->gt_launches = z[1].launches;
    pr->gt_seconds = 1e-9 * (double)z[1].total_ns;
  }

  // ------------------------------------------------------- graph capture
  cudaGraph_t add_while(cudaStream_t s, cudaGraphConditionalHandle hnd) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = hnd;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
    CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return p.conditional.phGraph_out[0];
  }

  cudaGraphConditionalHandle new_handle(cudaStream_t s) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    cudaGraphConditionalHandle hnd;
    CK(cudaGraphConditionalHandleCreate(&hnd, g, 0, cudaGraphCondAssignDefault));
    return hnd;
  }

  PointRef<T> pz() const { return PointRef<T>{x, y, gx, gty}; }
  PointRef<T> pzb() const { return PointRef<T>{xb, yb, gxb, gtyb}; }
  // z with the products the checks use (FP64 values; in FP64 mode the carried ones)
  PointRef<T> pzc() const { return PointRef<T>{x, y, gxt, gtyt}; }

  // Product with the iteration's values: the FP64 vector x, or (FP32 values)
  // its FP32 shadow xs.  tr selects G^T.
  template <typename Out>
  void spmv_it_out(bool tr, const double* xv, const float2* xs, const Out& out, const int* gate,
                   cudaStream_t s, KTimer* tmr = nullptr, bool pdl = false) {
    const SpmvPlan& pl = tr ? planGT : planG;
    if constexpr (kF32)
      launch_spmv_out<float>(pl, tr ? rpT : rp, tr ? ciT : ci, tr ? vvT : vv, xs, out, gate, s,
                             tmr, pdl);
    else
      launch_spmv_out<double>(pl, tr ? rpT : rp, tr ? ciT : ci, tr ? vvT : vv, xv, out, gate, s,
                              tmr, pdl);
  }
  void spmv_it(bool tr, const double* xv, const float2* xs, double* yv, const int* gate,
               cudaStream_t s, KTimer* tmr = nullptr, bool pdl = false) {
    spmv_it_out(tr, xv, xs, StoreOut<double>{yv}, gate, s, tmr, pdl);
  }
  // Product with the FP64 values (statistics of the checks).
  void spmv64(bool tr, const double* xv, double* yv, const int* gate, cudaStream_t s,
              KTimer* tmr = nullptr) {
    launch_spmv<double>(tr ? planGT : planG, tr ? rpT : rp, tr ? ciT : ci, tr ? vvT64 : vv64, xv,
                        yv, gate, s, tmr);
  }

  void rec_attempt(cudaStream_t s, cudaGraphConditionalHandle hA) {
    const Prob<T> p = prob();
    const int gn = ew_grid(n), gm = ew_grid(m), gmx = ew_grid(std::max(m, n));
    const bool q = pdl_;  // programmatic dependent launches inside the loop body
    launch_k(k_primal<T>, dim3(gn), dim3(kEwThreads), s, q, p, (const Ctl*)ctl, (const T*)x,
             (const T*)gty, xh, kF32 && !cols.any() ? sx : (float2*)nullptr);
    project<T>(cols, xh, xh, 1, d2, 1, 0, &ctl->g_attempt, nullptr, s, false, q);
    if (kF32 && cols.any())
      launch_k(k_split, dim3(gn), dim3(256), s, q, (const double*)xh, sx, n,
               (const int*)&ctl->g_attempt);
    // the dual iterate (onto diag(1/d1) K*) and the primal residual's
    // argument G xhat - h (onto diag(d1) K) are projected in one launch; the
    // residual is then also formed for rejected attempts, where it is unused
    double* res = tm[0];
    KTimer* tg = timers ? timers + TM_SPMV_G : nullptr;
    if (dual_in_product) {
      // long rows: the dual step rides on the product's epilogue
      spmv_it_out(false, xh, sx, DualOut<T>{p, ctl, y, gx, gxh, yh, res}, &ctl->g_attempt, s, tg, q);
    } else {
      spmv_it(false, xh, sx, gxh, &ctl->g_attempt, s, tg, q);
      launch_k(k_dual<T>, dim3(gm), dim3(kEwThreads), s, q, p, (const Ctl*)ctl, (const T*)y,
               (const T*)gxh, (const T*)gx, yh, res);
    }
    project<T>(rows, yh, reinterpret_cast<T*>(tm[0]), 2, d1, 1, 1, &ctl->g_attempt,
               &ctl->g_attempt, s, true, q);
    launch_k(k_step<T>, dim3(gmx), dim3(kEwThreads), s, q, p, ctl, (const T*)x, (const T*)xh,
             (const T*)y, (const T*)yh, (const T*)gxh, (const T*)gx, part, sy);
    spmv_it(true, yh, sy, gtyh, &ctl->g_accept, s, timers ? timers + TM_SPMV_GT : nullptr, q);
    const PointRef<T> ph{xh, yh, gxh, gtyh};
    const TmpRef t0{tm[0], tn[0], nullptr, nullptr};
    if (cols.any()) {
      const TmpRef tc{nullptr, tn[0], nullptr, nullptr};
      launch_k(k_res_prep<T>, dim3(gmx, 1), dim3(kEwThreads), s, q, p,
               (const int*)&ctl->g_accept, ph, ph, tc, tc);
    }
    project<double>(cols, tn[0], tn[0], 1, d2, 0, 1, &ctl->g_accept, nullptr, s, false, q);
    launch_k(k_point_stats<T, false>, dim3(gmx), dim3(kEwThreads), s, q, p, ctl,
             (const int*)&ctl->g_accept, 0, ph, (const T*)nullptr, (const T*)nullptr, t0, part);
    launch_k(k_halpern<T>, dim3(gmx), dim3(kEwThreads), s, q, p, ctl, x, y, gx, gty,
             (const T*)xh, (const T*)yh, (const T*)gxh, (const T*)gtyh, (const T*)x0,
             (const T*)y0, (const T*)gx0, (const T*)gty0, xs, ys, trace, hA, use_cond);
  }

  void rec_check_stats(cudaStream_t s) {
    const Prob<T> p = prob();
    const int gmx = ew_grid(std::max(m, n));
    int* g = &ctl->g_check;
    KTimer* tmisc = timers ? timers + TM_CHECK_MISC : nullptr;
    KTimer* tchk = timers ? timers + TM_SPMV_CHECK : nullptr;
    k_average<T><<<gmx, kEwThreads, 0, s>>>(n, m, ctl, xs, ys, xb, yb, tmisc);
    spmv64(false, xb, gxb, g, s, tchk);
    spmv64(true, yb, gtyb, g, s, tchk);
    if constexpr (kF32) {
      // FP64 products of z: the checks' statistics refer to the FP64 matrix
      spmv64(false, x, gxt, g, s, tchk);
      spmv64(true, y, gtyt, g, s, tchk);
    }
    const TmpRef ta{tm[0], tn[0], um[0], un[0]}, tb{tm[1], tn[1], um[1], un[1]};
    k_res_prep<T><<<dim3(gmx, 2), kEwThreads, 0, s>>>(p, g, pzc(), pzb(), ta, tb);
    project<double>(rows, tm[0], tm[1], 2, d1, 0, 0, g, g, s);
    project<double>(cols, tn[0], tn[1], 2, d2, 0, 1, g, g, s);
    project<double>(rows, um[0], um[1], 2, nullptr, 0, 0, g, g, s);
    project<double>(cols, un[0], un[1], 2, nullptr, 0, 1, g, g, s);
    k_point_stats<T, true><<<gmx, kEwThreads, 0, s>>>(p, ctl, g, 1, pzc(), x0, y0, ta, part);
    k_point_stats<T, true><<<gmx, kEwThreads, 0, s>>>(p, ctl, g, 2, pzb(), x0, y0, tb, part + (int64_t)gmx * kStatK);
  }

  void rec_probe(cudaStream_t s, cudaGraphConditionalHandle hB) {
    const Prob<T> p = prob();
    const int gmx = ew_grid(std::max(m, n));
    const bool q = pdl_;
    launch_k(k_probe_prep<T>, dim3(gmx, 2), dim3(kEwThreads), s, q, p, (const Ctl*)ctl, pzc(),
             pzb(), px[0], py[0], px[1], py[1]);
    project<double>(cols, px[0], px[1], 2, d2, 1, 0, &ctl->bs[0].active, &ctl->bs[1].active, s,
                    false, q);
    project<double>(rows, py[0], py[1], 2, d1, 1, 1, &ctl->bs[0].active, &ctl->bs[1].active, s,
                    false, q);
    launch_k(k_probe_reduce<T>, dim3(gmx, 2), dim3(kEwThreads), s, q, p, ctl, pzc(), pzb(),
             (const double*)px[0], (const double*)py[0], (const double*)px[1],
             (const double*)py[1], part, hB, use_cond);
  }

  void rec_check_end(cudaStream_t s) {
    const int gmx = ew_grid(std::max(m, n));
    if (infeas_on) {
      // infeasibility ratios of both candidates' change since the last candidate
      const Prob<T> p = prob();
      const PointRef<T> pc{xc, yc, gxc, gtyc};
      const TmpRef ta{tm[0], tn[0], um[0], un[0]}, tb{tm[1], tn[1], um[1], un[1]};
      const int* g0 = &ctl->infeas_gate[0];
      const int* g1 = &ctl->infeas_gate[1];
      k_infeas_prep<T><<<dim3(gmx, 2), kEwThreads, 0, s>>>(p, ctl, pzc(), pzb(), pc, ta, tb);
      project<double>(rows, tm[0], tm[1], 2, nullptr, 0, 0, g0, g1, s);
      project<double>(rows, um[0], um[1], 2, nullptr, 0, 1, g0, g1, s);
      project<double>(cols, tn[0], tn[1], 2, nullptr, 0, 1, g0, g1, s);
      project<double>(cols, un[0], un[1], 2, nullptr, 0, 0, g0, g1, s);
      k_infeas_reduce<T><<<dim3(gmx, 2), kEwThreads, 0, s>>>(p, ctl, pzc(), pzb(), pc, ta, tb, part);
    }
    k_check_decide<<<1, 1, 0, s>>>(ctl, trace);
    KTimer* tmisc = timers ? timers + TM_CHECK_MISC : nullptr;
    KTimer* tchk = timers ? timers + TM_SPMV_CHECK : nullptr;
    k_cand_copy<T><<<gmx, kEwThreads, 0, s>>>(n, m, ctl, pzc(), pzb(), xc, yc, gxc, gtyc, x0, y0, x, y,
                                              xs, ys, sx, sy, tmisc);
    spmv_it(false, x0, sx, gx0, &ctl->g_restart, s, tchk);
    spmv_it(true, y0, sy, gty0, &ctl->g_restart, s, tchk);
    k_copy_products<T><<<gmx, kEwThreads, 0, s>>>(n, m, &ctl->g_restart, gx0, gty0, gx, gty, tmisc);
    k_check_end<<<1, 1, 0, s>>>(ctl);
  }

  // Kernel nodes of a graph (conditional nodes and their bodies not included).
  static int64_t kernel_nodes(cudaGraph_t g) {
    size_t num = 0;
    CK(cudaGraphGetNodes(g, nullptr, &num));
    std::vector<cudaGraphNode_t> nodes(num);
    if (num) CK(cudaGraphGetNodes(g, nodes.data(), &num));
    int64_t k = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      CK(cudaGraphNodeGetType(nd, &t));
      if (t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
  }

  // Kernel counts of the eager mode's launch sequences (captured, never run).
  void count_eager() {
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(st2, cudaStreamCaptureModeRelaxed));
    rec_attempt(st2, 0);
    CK(cudaStreamEndCapture(st2, &g));
    nk_a = kernel_nodes(g);
    CK(cudaGraphDestroy(g));
    CK(cudaStreamBeginCapture(st2, cudaStreamCaptureModeRelaxed));
    rec_probe(st2, 0);
    CK(cudaStreamEndCapture(st2, &g));
    nk_b = kernel_nodes(g);
    CK(cudaGraphDestroy(g));
    CK(cudaStreamBeginCapture(st2, cudaStreamCaptureModeRelaxed));
    k_period_begin<<<1, 1, 0, st2>>>(ctl, 0, 0);
    rec_check_stats(st2);
    k_bisect_init<<<1, 1, 0, st2>>>(ctl, 0, 0);
    rec_check_end(st2);
    CK(cudaStreamEndCapture(st2, &g));
    nk_top = kernel_nodes(g);
    CK(cudaGraphDestroy(g));
  }

  void capture() {
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
    cudaGraphConditionalHandle hA = new_handle(st);
    cudaGraphConditionalHandle hB = new_handle(st);
    k_period_begin<<<1, 1, 0, st>>>(ctl, hA, 1);
    cudaGraph_t bodyA = add_while(st, hA);
    CK(cudaStreamBeginCaptureToGraph(st2, bodyA, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    rec_attempt(st2, hA);
    CK(cudaStreamEndCapture(st2, &bodyA));
    rec_check_stats(st);
    k_bisect_init<<<1, 1, 0, st>>>(ctl, hB, 1);
    cudaGraph_t bodyB = add_while(st, hB);
    CK(cudaStreamBeginCaptureToGraph(st2, bodyB, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    rec_probe(st2, hB);
    CK(cudaStreamEndCapture(st2, &bodyB));
    rec_check_end(st);
    CK(cudaStreamEndCapture(st, &graph));
    nk_a = kernel_nodes(bodyA);
    nk_b = kernel_nodes(bodyB);
    nk_top = kernel_nodes(graph);
    CK(cudaGraphInstantiate(&exec, graph, 0));
  }

  // ---------------------------------------------------------------- solve
  void init_ctl() {
    Ctl& c0 = *hctl;
    std::memset(&c0, 0, sizeof(Ctl));
    c0.eta = eta0; c0.eta_hat = eta0; c0.eta_acc = eta0; c0.omega = omega0; c0.omega0 = omega0;
    c0.eta0 = eta0;
    c0.status = kRunning;
    c0.h1 = h1; c0.c1 = c1; c0.hinf = hinf; c0.cinf = cinf;
    c0.rel_tol = opt.rel_tol; c0.abs_tol = opt.abs_tol; c0.bisect_tol = opt.bisect_rel_tol;
    c0.check_freq = std::max<int64_t>(1, opt.check_freq);
    c0.max_iter = opt.max_iter;
    c0.method = opt.method;
    c0.adaptive_restart = opt.use_adaptive_restart;
    c0.require_abs = opt.require_abs;
    c0.trace_cap = trace ? opt.trace_capacity : 0;
    c0.guard_cap = (int)std::min<int64_t>(4 * c0.check_freq + 16, 1 << 20);
    c0.probe_cap = 256;
    c0.adaptive_step = opt.use_adaptive_step_size_weight ? 1 : 0;
    c0.gap_restart = opt.use_duality_gap_restart ? 1 : 0;
    c0.kkt_restart = opt.use_kkt_restart ? 1 : 0;
    c0.kkt_freq = std::max<int64_t>(1, opt.kkt_restart_freq);
    c0.eta_fixed = eta_fixed;
    if (!c0.adaptive_step) c0.eta = c0.eta_hat = c0.eta_acc = eta_fixed;
    c0.eps_pl = opt.eps_primal_infeasible_low_acc;
    c0.eps_dl = opt.eps_dual_infeasible_low_acc;
    c0.eps_ph = opt.eps_primal_infeasible_high_acc;
    c0.eps_dh = opt.eps_dual_infeasible_high_acc;
    c0.infeas_on = infeas_on ? 1 : 0;
  }

  void upload_ctl() { CK(cudaMemcpyAsync(ctl, hctl, sizeof(Ctl), cudaMemcpyHostToDevice, st)); }

  void start_point(const double* x0u, const double* y0u) {
    const int gn = ew_grid(n), gm = ew_grid(m);
    if (x0u) {
      copy_in(obuf_n, x0u, n, st);
      if (ncol_rot) k_rotate_pairs<<<ew_grid(ncol_rot), 256, 0, st>>>(obuf_n, col_rot, ncol_rot);
      k_warm<T><<<gn, 256, 0, st>>>(x, obuf_n, d2, n);
    } else {
      k_fill<T><<<gn, 256, 0, st>>>(x, n, 0.0);
    }
    if (y0u) {
      copy_in(obuf_m, y0u, m, st);
      if (nrow_rot) k_rotate_pairs<<<ew_grid(nrow_rot), 256, 0, st>>>(obuf_m, row_rot, nrow_rot);
      k_warm<T><<<gm, 256, 0, st>>>(y, obuf_m, d1, m);
    } else {
      k_fill<T><<<gm, 256, 0, st>>>(y, m, 0.0);
    }
    k_convert<T, T><<<gn, 256, 0, st>>>(x, x0, n);
    k_convert<T, T><<<gm, 256, 0, st>>>(y, y0, m);
    k_fill<double><<<gn, 256, 0, st>>>(xs, n, 0.0);
    k_fill<double><<<gm, 256, 0, st>>>(ys, m, 0.0);
    refresh_products();
  }

  // G x, G^T y, G x0, G^T y0 from the current vectors.
  void refresh_products() {
    const int gn = ew_grid(n), gm = ew_grid(m);
    const double* vs[4] = {x, y, x0, y0};
    double* ps[4] = {gx, gty, gx0, gty0};
    for (int k = 0; k < 4; ++k) {
      const bool tr = (k & 1) != 0;
      if (kF32) k_split<<<tr ? gm : gn, 256, 0, st>>>(vs[k], tr ? sy : sx, tr ? m : n, nullptr);
      spmv_it(tr, vs[k], tr ? sy : sx, ps[k], nullptr, st);
    }
    CK(cudaGetLastError());
  }

  void solve(const double* x0u, const double* y0u, double* xo, double* yo, double* so,
             pdcs_result* res) override {
    const auto t0 = std::chrono::steady_clock::now();
    order_after_user();
    init_ctl();
    upload_ctl();
    start_point(x0u, y0u);
    if (trace) CK(cudaMemsetAsync(trace, 0, sizeof(double) * (size_t)opt.trace_capacity * PDCS_TRACE_FIELDS, st));
    run(xo, yo, so, res, t0);
  }

  // KKT errors of a given point: load it as the iterate, refresh the products
  // and take the final statistics (Sec. 3.2.3) without any iteration.
  void evaluate(const double* x0u, const double* y0u, pdcs_result* res) override {
    const auto t0 = std::chrono::steady_clock::now();
    order_after_user();
    init_ctl();
    upload_ctl();
    start_point(x0u, y0u);
    finish(0, nullptr, nullptr, nullptr, res, t0);
    if (res) {
      const PointStats& s3 = hctl->st[3];
      bool ok = std::max(s3.inf_rel_p, std::max(s3.inf_rel_d, s3.inf_rel_gap)) <= opt.rel_tol;
      if (opt.require_abs)
        ok = ok && std::max(s3.inf_abs_p, std::max(s3.inf_abs_d, s3.gap)) <= opt.abs_tol;
      res->exit_code = ok ? 0 : -1;
      res->iters = res->attempts = res->restarts = 0;
    }
  }

  void resume(int64_t max_iter, double* xo, double* yo, double* so, pdcs_result* res) override {
    const auto t0 = std::chrono::steady_clock::now();
    order_after_user();
    CK(cudaMemcpyAsync(hctl, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    hctl->max_iter = max_iter > 0 ? max_iter : opt.max_iter;
    hctl->status = hctl->iter >= hctl->max_iter ? 1 : kRunning;
    hctl->period_done = 0;
    hctl->have_cand = 0;
    hctl->g_attempt = hctl->g_accept = hctl->g_check = hctl->g_restart = 0;
    upload_ctl();
    if (hctl->status != kRunning) {
      finish(hctl->status, xo, yo, so, res, t0);
      return;
    }
    run(xo, yo, so, res, t0);
  }

  // One check period launched kernel by kernel from the host (the same kernels
  // and gates as the captured graph; the host reads the loop conditions).  Slow;
  // meant for per-kernel profilers, which cannot see inside conditional graphs.
  int read_flag(const int* dflag) {
    int v = 0;
    CK(cudaMemcpyAsync(&v, dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return v;
  }

  void run_period_eager() {
    k_period_begin<<<1, 1, 0, st>>>(ctl, 0, 0);
    for (int guard = 0; guard < 1 << 20 && read_flag(&ctl->g_attempt); ++guard) {
      rec_attempt(st, 0);
      ++eager_a;
    }
    rec_check_stats(st);
    k_bisect_init<<<1, 1, 0, st>>>(ctl, 0, 0);
    for (int guard = 0; guard < 1024 && (read_flag(&ctl->bs[0].active) || read_flag(&ctl->bs[1].active));
         ++guard) {
      rec_probe(st, 0);
      ++eager_b;
    }
    rec_check_end(st);
    CK(cudaGetLastError());
  }

  void run(double* xo, double* yo, double* so, pdcs_result* res,
           std::chrono::steady_clock::time_point t0) {
    int status = kRunning;
    reset_timers();
    graph_launches = 0;
    eager_a = eager_b = 0;
    bodies_a0 = hctl->bodies_a;
    bodies_b0 = hctl->bodies_b;
    long long printed = hctl->iter;
    const long long pf = std::max<int64_t>(1, opt.print_freq);
    while (true) {
      if (use_cond) CK(cudaGraphLaunch(exec, st));
      else run_period_eager();
      ++graph_launches;
      CK(cudaMemcpyAsync(hctl, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      status = hctl->status;
      if (opt.verbose && (hctl->iter / pf != printed / pf || status != kRunning)) {
        printed = hctl->iter;
        fprintf(stderr, "[pdcs] iter %lld kbar %lld restarts %lld eta %.3e omega %.3e maxErr %.3e\n",
                hctl->iter, hctl->kbar, hctl->restarts, hctl->eta_acc, hctl->omega, hctl->st[0].max_err);
      }
      if (status != kRunning) break;
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > opt.time_limit) {
        status = 6;
        break;
      }
    }
    finish(status, xo, yo, so, res, t0);
  }

  void finish(int status, double* xo, double* yo, double* so, pdcs_result* res,
              std::chrono::steady_clock::time_point t0) {
    const Prob<T> p = prob();
    const int gmx = ew_grid(std::max(m, n));
    const bool cand = hctl->have_cand != 0;
    if (kF32 && !cand) {
      // no candidate yet: FP64 products of z for the reported errors
      spmv64(false, x, gxt, nullptr, st);
      spmv64(true, y, gtyt, nullptr, st);
    }
    const PointRef<T> pr = cand ? PointRef<T>{xc, yc, gxc, gtyc} : pzc();
    // final statistics of the returned point (slot 3); g_check serves as an
    // always-on gate here (no graph runs until the next call re-initialises it)
    int* one = &ctl->g_check;
    const int hone = 1;
    CK(cudaMemcpyAsync(one, &hone, sizeof(int), cudaMemcpyHostToDevice, st));
    const TmpRef ta{tm[0], tn[0], um[0], un[0]};
    k_res_prep<T><<<dim3(gmx, 1), kEwThreads, 0, st>>>(p, one, pr, pr, ta, ta);
    project<double>(rows, tm[0], tm[0], 1, d1, 0, 0, one, nullptr, st);
    project<double>(cols, tn[0], tn[0], 1, d2, 0, 1, one, nullptr, st);
    project<double>(rows, um[0], um[0], 1, nullptr, 0, 0, one, nullptr, st);
    project<double>(cols, un[0], un[0], 1, nullptr, 0, 1, one, nullptr, st);
    k_point_stats<T, true><<<gmx, kEwThreads, 0, st>>>(p, ctl, one, 3, pr, nullptr, nullptr, ta, part);
    k_unscale<T><<<gmx, 256, 0, st>>>(p, pr.x, pr.y, pr.gx, obuf_n, obuf_m, obuf_s);
    if (ncol_rot) k_rotate_pairs<<<ew_grid(ncol_rot), 256, 0, st>>>(obuf_n, col_rot, ncol_rot);
    if (nrow_rot) {
      k_rotate_pairs<<<ew_grid(nrow_rot), 256, 0, st>>>(obuf_m, row_rot, nrow_rot);
      k_rotate_pairs<<<ew_grid(nrow_rot), 256, 0, st>>>(obuf_s, row_rot, nrow_rot);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(hctl, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    if (xo) CK(cudaMemcpyAsync(xo, obuf_n, sizeof(double) * n, cudaMemcpyDefault, st));
    if (yo && m) CK(cudaMemcpyAsync(yo, obuf_m, sizeof(double) * m, cudaMemcpyDefault, st));
    if (so && m) CK(cudaMemcpyAsync(so, obuf_s, sizeof(double) * m, cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    trace_rows = std::min<int64_t>(hctl->iter, opt.trace_capacity);
    if (gsync_err) {
      int herr = 0;
      CK(cudaMemcpy(&herr, gsync_err, sizeof(int), cudaMemcpyDeviceToHost));
      if (herr) {
        CK(cudaMemset(gsync_err, 0, sizeof(int)));
        throw Fail{PDCS_ERR_TIMEOUT, "a grid barrier wait of the SOC projection gave up"};
      }
    }
    if (res) {
      const PointStats& s3 = hctl->st[3];
      res->exit_code = status;
      res->pobj = s3.pobj;
      res->dobj = s3.dobj;
      res->err_rel_p = s3.inf_rel_p;
      res->err_rel_d = s3.inf_rel_d;
      res->err_rel_gap = s3.inf_rel_gap;
      res->err_abs_p = s3.inf_abs_p;
      res->err_abs_d = s3.inf_abs_d;
      res->err_abs_gap = s3.gap;
      res->iters = hctl->iter;
      res->attempts = hctl->kbar;
      res->restarts = hctl->restarts;
      res->solve_time_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
  }

  // ------------------------------------------------------ state access
  void to_user(const T* src, double* buf, double* dst, int64_t cnt) {
    if (!dst || cnt == 0) return;
    k_convert<T, double><<<ew_grid(cnt), 256, 0, st>>>(src, buf, cnt);
    CK(cudaMemcpyAsync(dst, buf, sizeof(double) * cnt, cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
  }

  void get_state(pdcs_state* s, double* xo, double* yo, double* x0o, double* y0o, double* xso,
                 double* yso) override {
    CK(cudaMemcpyAsync(hctl, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (s) {
      const Ctl& c0 = *hctl;
      s->iter = c0.iter; s->kbar = c0.kbar; s->k = c0.k; s->period = c0.period;
      s->restarts = c0.restarts; s->eta_hat = c0.eta; s->eta_last = c0.eta_acc;
      s->omega = c0.omega; s->wsum = c0.wsum; s->has_ref = c0.has_ref; s->has_prev = c0.has_prev;
      s->ref_rho = c0.ref_rho; s->ref_abs_p = c0.ref_ep; s->ref_abs_d = c0.ref_ed;
      s->ref_abs_gap = c0.ref_eg; s->prev_rho = c0.prev_rho; s->prev_abs_p = c0.prev_ep;
      s->prev_abs_d = c0.prev_ed; s->prev_abs_gap = c0.prev_eg;
    }
    to_user(x, obuf_n, xo, n);
    to_user(y, obuf_m, yo, m);
    to_user(x0, obuf_n, x0o, n);
    to_user(y0, obuf_m, y0o, m);
    if (xso) CK(cudaMemcpyAsync(xso, xs, sizeof(double) * n, cudaMemcpyDefault, st));
    if (yso && m) CK(cudaMemcpyAsync(yso, ys, sizeof(double) * m, cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
  }

  void set_state(const pdcs_state* s, const double* xi, const double* yi, const double* x0i,
                 const double* y0i, const double* xsi, const double* ysi) override {
    order_after_user();
    init_ctl();
    Ctl& c0 = *hctl;
    c0.iter = s->iter; c0.kbar = s->kbar; c0.k = s->k; c0.period = s->period;
    c0.restarts = s->restarts; c0.eta = s->eta_hat; c0.eta_hat = s->eta_hat;
    c0.eta_acc = s->eta_last; c0.omega = s->omega; c0.wsum = s->wsum;
    c0.has_ref = s->has_ref; c0.has_prev = s->has_prev;
    c0.ref_rho = s->ref_rho; c0.ref_ep = s->ref_abs_p; c0.ref_ed = s->ref_abs_d;
    c0.ref_eg = s->ref_abs_gap; c0.prev_rho = s->prev_rho; c0.prev_ep = s->prev_abs_p;
    c0.prev_ed = s->prev_abs_d; c0.prev_eg = s->prev_abs_gap;
    upload_ctl();
    const int gn = ew_grid(n), gm = ew_grid(m);
    T* dn[2] = {x, x0};
    const double* sn[2] = {xi, x0i};
    T* dm[2] = {y, y0};
    const double* sm[2] = {yi, y0i};
    for (int k = 0; k < 2; ++k) {
      copy_in(obuf_n, sn[k], n, st);
      k_convert<double, T><<<gn, 256, 0, st>>>(obuf_n, dn[k], n);
      copy_in(obuf_m, sm[k], m, st);
      k_convert<double, T><<<gm, 256, 0, st>>>(obuf_m, dm[k], m);
      CK(cudaStreamSynchronize(st));
    }
    copy_in(xs, xsi, n, st);
    copy_in(ys, ysi, m, st);
    refresh_products();
    CK(cudaStreamSynchronize(st));
  }

  void get_iterate(int which, double* xo, double* yo) override {
    if (which == 3) {
      if (xo) CK(cudaMemcpyAsync(xo, d2, sizeof(double) * n, cudaMemcpyDefault, st));
      if (yo && m) CK(cudaMemcpyAsync(yo, d1, sizeof(double) * m, cudaMemcpyDefault, st));
      CK(cudaStreamSynchronize(st));
      return;
    }
    const T* a = which == 0 ? x : (which == 1 ? x0 : xh);
    const T* b = which == 0 ? y : (which == 1 ? y0 : yh);
    to_user(a, obuf_n, xo, n);
    to_user(b, obuf_m, yo, m);
  }

  int64_t get_trace(double* out, int64_t cap) override {
    const int64_t rows_ = std::min(cap, trace_rows);
    if (rows_ > 0 && trace)
      CK(cudaMemcpy(out, trace, sizeof(double) * rows_ * PDCS_TRACE_FIELDS, cudaMemcpyDeviceToHost));
    return std::max<int64_t>(rows_, 0);
  }
};


// ------------------------------------------------------------------ batch
// Many independent problems as one block-diagonal problem: set up by the
// ordinary set-up (column layout in segments), solved by k_batch (one CTA per
// instance at a time).
template <typename T>
struct BatchSolver : BatchBase {
  Solver<T> sv;
  int64_t count = 0;
  std::vector<BInst> hinst;
  std::vector<int32_t> horder;
  BInst* dinst = nullptr;
  int32_t* dorder = nullptr;
  Ctl* dctls = nullptr;
  Ctl* dtmpl = nullptr;
  unsigned int* dqueue = nullptr;
  unsigned long long* dtimes = nullptr;
  int64_t *soc_rs = nullptr, *soc_cs = nullptr, *exp_rs = nullptr, *exp_cs = nullptr;
  int32_t *soc_rd = nullptr, *soc_cd = nullptr;
  uint8_t *exp_risd = nullptr, *exp_cisd = nullptr;
  int grid = 0;
  double time_limit = 0.0;

  template <typename U>
  U* upload(const std::vector<U>& v) {
    U* d = sv.ar.template alloc<U>((int64_t)v.size());
    if (!v.empty()) copy_in(d, v.data(), (int64_t)v.size(), sv.st);
    return d;
  }

  void setup(const pdcs_instance* in, int64_t cnt, const pdcs_options& o, cudaStream_t stream) {
    count = cnt;
    int64_t M = 0, N = 0, NNZ = 0;
    std::vector<int64_t> nnz_i((size_t)cnt);
    for (int64_t i = 0; i < cnt; ++i) {
      int64_t last = 0;
      CK(cudaMemcpy(&last, in[i].row_ptr + in[i].m, sizeof(int64_t), cudaMemcpyDefault));
      nnz_i[i] = last;
      M += in[i].m;
      N += in[i].n;
      NNZ += last;
    }
    std::vector<int64_t> rp((size_t)M + 1);
    std::vector<int32_t> ci((size_t)NNZ);
    std::vector<double> val((size_t)NNZ), h((size_t)M), c((size_t)N);
    std::vector<double> lb((size_t)N, -INFINITY), ub((size_t)N, INFINITY);
    std::vector<pdcs_cone> rcones;
    std::vector<typename Solver<T>::ColSeg> segs;
    std::vector<int64_t> srs, scs, ers, ecs;
    std::vector<int32_t> srd, scd;
    std::vector<uint8_t> erd, ecd;
    hinst.resize((size_t)cnt);
    int64_t r0 = 0, c0 = 0, e0 = 0;
    rp[0] = 0;
    for (int64_t i = 0; i < cnt; ++i) {
      const pdcs_instance& I = in[i];
      if (N + 0 > INT32_MAX) invalid("batch has more than 2^31 columns");
      std::vector<int64_t> lrp((size_t)I.m + 1);
      CK(cudaMemcpy(lrp.data(), I.row_ptr, sizeof(int64_t) * (I.m + 1), cudaMemcpyDefault));
      const int64_t nz = nnz_i[i];
      if (nz > 0) {
        std::vector<int32_t> lci((size_t)nz);
        CK(cudaMemcpy(lci.data(), I.col_idx, sizeof(int32_t) * nz, cudaMemcpyDefault));
        CK(cudaMemcpy(val.data() + e0, I.val, sizeof(double) * nz, cudaMemcpyDefault));
        for (int64_t e = 0; e < nz; ++e) {
          if (lci[e] < 0 || lci[e] >= I.n) invalid("column index out of range in a batch instance");
          ci[e0 + e] = (int32_t)(lci[e] + c0);
        }
      }
      for (int64_t r = 0; r < I.m; ++r) rp[r0 + r + 1] = e0 + lrp[r + 1];
      if (I.m > 0) CK(cudaMemcpy(h.data() + r0, I.h, sizeof(double) * I.m, cudaMemcpyDefault));
      CK(cudaMemcpy(c.data() + c0, I.c, sizeof(double) * I.n, cudaMemcpyDefault));
      if (I.nb > 0) {
        CK(cudaMemcpy(lb.data() + c0, I.lb, sizeof(double) * I.nb, cudaMemcpyDefault));
        CK(cudaMemcpy(ub.data() + c0, I.ub, sizeof(double) * I.nb, cudaMemcpyDefault));
      }
      BInst& b = hinst[(size_t)i];
      b = BInst{};
      b.r0 = r0; b.m = I.m; b.c0 = c0; b.n = I.n; b.tile = 32;
      b.soc_r0 = (int32_t)srs.size(); b.exp_r0 = (int32_t)ers.size();
      int64_t off = r0;
      for (int64_t k = 0; k < I.n_row_cones; ++k) {
        const pdcs_cone& cn = I.row_cones[k];
        rcones.push_back(cn);
        if (cn.type == PDCS_CONE_SOC || cn.type == PDCS_CONE_RSOC) {
          srs.push_back(off); srd.push_back((int32_t)cn.dim);
        } else if (cn.type == PDCS_CONE_EXP || cn.type == PDCS_CONE_DUAL_EXP) {
          ers.push_back(off); erd.push_back(cn.type == PDCS_CONE_DUAL_EXP ? 1 : 0);
        }
        off += cn.dim;
      }
      b.soc_rn = (int32_t)srs.size() - b.soc_r0; b.exp_rn = (int32_t)ers.size() - b.exp_r0;
      typename Solver<T>::ColSeg sg;
      sg.off = c0; sg.nb = I.nb; sg.end = c0 + I.n;
      sg.cones.assign(I.col_cones, I.col_cones + I.n_col_cones);
      segs.push_back(sg);
      b.soc_c0 = (int32_t)scs.size(); b.exp_c0 = (int32_t)ecs.size();
      off = c0 + I.nb;
      for (int64_t k = 0; k < I.n_col_cones; ++k) {
        const pdcs_cone& cn = I.col_cones[k];
        if (cn.type == PDCS_CONE_SOC || cn.type == PDCS_CONE_RSOC) {
          scs.push_back(off); scd.push_back((int32_t)cn.dim);
        } else if (cn.type == PDCS_CONE_EXP || cn.type == PDCS_CONE_DUAL_EXP) {
          ecs.push_back(off); ecd.push_back(cn.type == PDCS_CONE_DUAL_EXP ? 1 : 0);
        }
        off += cn.dim;
      }
      b.soc_cn = (int32_t)scs.size() - b.soc_c0; b.exp_cn = (int32_t)ecs.size() - b.exp_c0;
      r0 += I.m;
      c0 += I.n;
      e0 += nz;
    }
    pdcs_options so = o;
    so.eager = 1;    // the batch runs its own kernel: no single-problem graphs
    so.profile = 0;
    so.trace_capacity = 0;
    time_limit = o.time_limit;
    const std::vector<pdcs_cone> none;
    sv.setup(M, N, rp.data(), ci.data(), val.data(), h.data(), c.data(), 0, lb.data(), ub.data(),
             rcones, none, so, stream, &segs);
    soc_rs = upload(srs); soc_rd = upload(srd); soc_cs = upload(scs); soc_cd = upload(scd);
    exp_rs = upload(ers); exp_risd = upload(erd); exp_cs = upload(ecs); exp_cisd = upload(ecd);
    // queue order: most nonzeros first
    horder.resize((size_t)cnt);
    for (int64_t i = 0; i < cnt; ++i) horder[i] = (int32_t)i;
    std::stable_sort(horder.begin(), horder.end(),
                     [&](int32_t a, int32_t b) { return nnz_i[a] > nnz_i[b]; });
    dorder = sv.ar.template alloc<int32_t>(cnt);
    dinst = sv.ar.template alloc<BInst>(cnt);
    dctls = sv.ar.template alloc<Ctl>(cnt);
    dtmpl = sv.ar.template alloc<Ctl>(1);
    dqueue = sv.ar.template alloc<unsigned int>(1);
    dtimes = sv.ar.template alloc<unsigned long long>(2 * cnt);
    sv.init_ctl();
    sv.hctl->infeas_on = 0;  // the batched engine does not run the infeasibility tests
    CK(cudaMemcpyAsync(dtmpl, sv.hctl, sizeof(Ctl), cudaMemcpyHostToDevice, sv.st));
    int dev = 0, sms = 0, occ = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<T>, kBatchThreads, 0));
    grid = std::max(1, sms * std::max(1, occ));
    autotune(nnz_i);
  }

  BatchArgs<T> args(int32_t n_queue) {
    BatchArgs<T> a;
    a.p = sv.prob();
    a.p.tm = nullptr;
    a.rp = sv.rp; a.rpT = sv.rpT; a.ci = sv.ci; a.ciT = sv.ciT; a.vv = sv.vv; a.vvT = sv.vvT;
    a.x = sv.x; a.y = sv.y; a.xh = sv.xh; a.yh = sv.yh; a.gx = sv.gx; a.gty = sv.gty;
    a.gxh = sv.gxh; a.gtyh = sv.gtyh; a.x0 = sv.x0; a.y0 = sv.y0; a.gx0 = sv.gx0; a.gty0 = sv.gty0;
    a.xb = sv.xb; a.yb = sv.yb; a.gxb = sv.gxb; a.gtyb = sv.gtyb;
    a.xc = sv.xc; a.yc = sv.yc; a.gxc = sv.gxc; a.gtyc = sv.gtyc;
    a.xs = sv.xs; a.ys = sv.ys;
    for (int k = 0; k < 2; ++k) {
      a.tm[k] = sv.tm[k]; a.tn[k] = sv.tn[k]; a.um[k] = sv.um[k]; a.un[k] = sv.un[k];
      a.px[k] = sv.px[k]; a.py[k] = sv.py[k];
    }
    a.soc_rs = soc_rs; a.soc_cs = soc_cs; a.soc_rd = soc_rd; a.soc_cd = soc_cd;
    a.exp_rs = exp_rs; a.exp_cs = exp_cs; a.exp_risd = exp_risd; a.exp_cisd = exp_cisd;
    a.inst = dinst; a.order = dorder; a.count = n_queue; a.ctls = dctls; a.tmpl = dtmpl;
    a.queue = dqueue; a.times = dtimes; a.time_limit_s = time_limit;
    return a;
  }

  void launch(int32_t n_queue) {
    CK(cudaMemsetAsync(dqueue, 0, sizeof(unsigned int), sv.st));
    k_batch<T><<<grid, kBatchThreads, 0, sv.st>>>(args(n_queue));
    CK(cudaGetLastError());
  }

  // Lanes per row of the products, per size bucket (columns < 256, < 512,
  // < 1024, larger): a few instances of the bucket are solved for three check
  // periods with each candidate, and the fastest is kept.
  void autotune(const std::vector<int64_t>& nnz_i) {
    const int tiles[4] = {4, 8, 16, 32};
    const int64_t edges[4] = {256, 512, 1024, INT64_MAX};
    auto bucket = [&](int64_t i) {
      int b = 0;
      while (hinst[i].n >= edges[b]) ++b;
      return b;
    };
    Ctl short_tmpl = *sv.hctl;
    short_tmpl.max_iter = std::max<long long>(1, 3 * short_tmpl.check_freq);
    CK(cudaMemcpyAsync(dtmpl, &short_tmpl, sizeof(Ctl), cudaMemcpyHostToDevice, sv.st));
    int best[4] = {32, 32, 32, 32};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int b = 0; b < 4; ++b) {
      std::vector<int32_t> sample;
      for (int64_t q = 0; q < count && (int)sample.size() < 4; ++q)
        if (bucket(horder[q]) == b) sample.push_back(horder[q]);
      if (sample.empty()) continue;
      float best_ms = 1e30f;
      for (int t : tiles) {
        for (int32_t i : sample) hinst[i].tile = t;
        CK(cudaMemcpyAsync(dinst, hinst.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice, sv.st));
        CK(cudaMemcpyAsync(dorder, sample.data(), sizeof(int32_t) * sample.size(), cudaMemcpyHostToDevice, sv.st));
        CK(cudaEventRecord(e0, sv.st));
        launch((int32_t)sample.size());
        CK(cudaEventRecord(e1, sv.st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) { best_ms = ms; best[b] = t; }
      }
    }
    CK(cudaEventDestroy(e0));
    CK(cudaEventDestroy(e1));
    for (int64_t i = 0; i < count; ++i) hinst[i].tile = best[bucket(i)];
    CK(cudaMemcpyAsync(dinst, hinst.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice, sv.st));
    CK(cudaMemcpyAsync(dorder, horder.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, sv.st));
    CK(cudaMemcpyAsync(dtmpl, sv.hctl, sizeof(Ctl), cudaMemcpyHostToDevice, sv.st));
    CK(cudaStreamSynchronize(sv.st));
    for (int b = 0; b < 4; ++b) tile_of_bucket[b] = best[b];
  }
  int tile_of_bucket[4] = {32, 32, 32, 32};

  void solve(double* xo, double* yo, double* so, pdcs_result* res, double* finish_s) override {
    sv.order_after_user();
    launch((int32_t)count);
    const Prob<double> p = sv.prob();
    const int gmx = ew_grid(std::max(sv.m, sv.n));
    k_unscale<double><<<gmx, 256, 0, sv.st>>>(p, sv.xc, sv.yc, sv.gxc, sv.obuf_n, sv.obuf_m, sv.obuf_s);
    if (sv.ncol_rot) k_rotate_pairs<<<ew_grid(sv.ncol_rot), 256, 0, sv.st>>>(sv.obuf_n, sv.col_rot, sv.ncol_rot);
    if (sv.nrow_rot) {
      k_rotate_pairs<<<ew_grid(sv.nrow_rot), 256, 0, sv.st>>>(sv.obuf_m, sv.row_rot, sv.nrow_rot);
      k_rotate_pairs<<<ew_grid(sv.nrow_rot), 256, 0, sv.st>>>(sv.obuf_s, sv.row_rot, sv.nrow_rot);
    }
    CK(cudaGetLastError());
    if (xo) CK(cudaMemcpyAsync(xo, sv.obuf_n, sizeof(double) * sv.n, cudaMemcpyDefault, sv.st));
    if (yo && sv.m) CK(cudaMemcpyAsync(yo, sv.obuf_m, sizeof(double) * sv.m, cudaMemcpyDefault, sv.st));
    if (so && sv.m) CK(cudaMemcpyAsync(so, sv.obuf_s, sizeof(double) * sv.m, cudaMemcpyDefault, sv.st));
    std::vector<Ctl> hc((size_t)count);
    std::vector<unsigned long long> ht((size_t)(2 * count));
    CK(cudaMemcpyAsync(hc.data(), dctls, sizeof(Ctl) * count, cudaMemcpyDeviceToHost, sv.st));
    CK(cudaMemcpyAsync(ht.data(), dtimes, sizeof(unsigned long long) * 2 * count, cudaMemcpyDeviceToHost, sv.st));
    CK(cudaStreamSynchronize(sv.st));
    unsigned long long t0 = ~0ull;
    for (int64_t i = 0; i < count; ++i) t0 = std::min(t0, ht[2 * i]);
    for (int64_t i = 0; i < count; ++i) {
      const Ctl& c = hc[i];
      if (res) {
        pdcs_result& r = res[i];
        std::memset(&r, 0, sizeof(r));
        const PointStats& s3 = c.st[3];
        r.exit_code = c.status;
        r.pobj = s3.pobj;
        r.dobj = s3.dobj;
        r.err_rel_p = s3.inf_rel_p;
        r.err_rel_d = s3.inf_rel_d;
        r.err_rel_gap = s3.inf_rel_gap;
        r.err_abs_p = s3.inf_abs_p;
        r.err_abs_d = s3.inf_abs_d;
        r.err_abs_gap = s3.gap;
        r.iters = c.iter;
        r.attempts = c.kbar;
        r.restarts = c.restarts;
        r.solve_time_s = 1e-9 * (double)(ht[2 * i + 1] - ht[2 * i]);
      }
      if (finish_s) finish_s[i] = 1e-9 * (double)(ht[2 * i + 1] - t0);
    }
  }
};

}  // namespace pdcs

// ----------------------------------------------------------------- C ABI
extern "C" {

void pdcs_default_options(pdcs_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->rel_tol = 1e-6;
  o->abs_tol = 1e-6;
  o->time_limit = 1000.0;
  o->max_iter = INT64_MAX;
  o->use_preconditioner = 1;
  o->ruiz_iters = 10;
  o->pc_alpha = 1.0;
  o->method = 0;
  o->use_adaptive_restart = 1;
  o->check_freq = 64;
  o->precision = 0;
  o->require_abs = 0;
  o->bisect_rel_tol = 1e-3;
  o->verbose = 0;
  o->trace_capacity = 0;
  o->profile = 0;
  o->eager = 0;
  o->use_adaptive_step_size_weight = 1;
  o->use_duality_gap_restart = 1;
  o->use_kkt_restart = 0;
  o->overlap_launches = 0;
  o->kkt_restart_freq = 2000;
  o->print_freq = 2000;
  o->eps_primal_infeasible_low_acc = 1e-12;
  o->eps_dual_infeasible_low_acc = 1e-12;
  o->eps_primal_infeasible_high_acc = 1e-16;
  o->eps_dual_infeasible_high_acc = 1e-16;
}

const char* pdcs_last_error(void) { return g_last_error.c_str(); }

static int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

static int check_cones(const pdcs_cone* cl, int64_t k, int64_t expect, const char* what) {
  int64_t sum = 0;
  for (int64_t i = 0; i < k; ++i) {
    const pdcs_cone& c = cl[i];
    if (c.type < 0 || c.type > 5 || c.dim < 1) return fail(PDCS_ERR_INVALID, std::string("bad ") + what + " cone");
    if ((c.type == PDCS_CONE_EXP || c.type == PDCS_CONE_DUAL_EXP) && c.dim != 3)
      return fail(PDCS_ERR_INVALID, "exponential cone blocks have dimension 3");
    if (c.type == PDCS_CONE_RSOC && c.dim < 2) return fail(PDCS_ERR_INVALID, "RSOC needs dim >= 2");
    sum += c.dim;
  }
  if (sum != expect)
    return fail(PDCS_ERR_INVALID, std::string(what) + (what[0] == 'r' ? " cone dimensions must sum to m"
                                                                       : " cone dimensions must sum to n - nb"));
  return PDCS_OK;
}

int pdcs_setup(pdcs_handle** out, int64_t m, int64_t n, const int64_t* row_ptr,
               const int32_t* col_idx, const double* val, const double* h, const double* c,
               int64_t nb, const double* lb, const double* ub, const pdcs_cone* row_cones,
               int64_t n_row_cones, const pdcs_cone* col_cones, int64_t n_col_cones,
               const pdcs_options* opt, void* cuda_stream) {
  if (!out) return fail(PDCS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (m < 0 || n < 1) return fail(PDCS_ERR_INVALID, "need m >= 0 and n >= 1");
  if (nb < 0 || nb > n) return fail(PDCS_ERR_INVALID, "need 0 <= nb <= n");
  if (!row_ptr || (m > 0 && !h) || !c) return fail(PDCS_ERR_INVALID, "row_ptr, h and c are required");
  if (n_row_cones < 0 || n_col_cones < 0) return fail(PDCS_ERR_INVALID, "negative cone count");
  if ((n_row_cones > 0 && !row_cones) || (n_col_cones > 0 && !col_cones))
    return fail(PDCS_ERR_INVALID, "cone list is NULL");
  int rc_ = check_cones(row_cones, n_row_cones, m, "row");
  if (rc_ != PDCS_OK) return rc_;
  rc_ = check_cones(col_cones, n_col_cones, n - nb, "column");
  if (rc_ != PDCS_OK) return rc_;
  pdcs_options o;
  if (opt) o = *opt; else pdcs_default_options(&o);
  if (o.precision != 0 && o.precision != 1) return fail(PDCS_ERR_INVALID, "precision must be 0 or 1");
  if (o.check_freq < 1) return fail(PDCS_ERR_INVALID, "check_freq must be >= 1");
  if (o.use_kkt_restart && o.kkt_restart_freq < 1) return fail(PDCS_ERR_INVALID, "kkt_restart_freq must be >= 1");
  if (!(o.eps_primal_infeasible_low_acc >= 0) || !(o.eps_dual_infeasible_low_acc >= 0) ||
      !(o.eps_primal_infeasible_high_acc >= 0) || !(o.eps_dual_infeasible_high_acc >= 0))
    return fail(PDCS_ERR_INVALID, "infeasibility thresholds must be >= 0");
  if (o.method != 0 && o.method != 1) return fail(PDCS_ERR_INVALID, "method must be 0 or 1");
  if (o.max_iter < 1) return fail(PDCS_ERR_INVALID, "max_iter must be >= 1");
  if (o.ruiz_iters < 0) return fail(PDCS_ERR_INVALID, "ruiz_iters must be >= 0");
  if (!(o.bisect_rel_tol > 0.0)) return fail(PDCS_ERR_INVALID, "bisect_rel_tol must be > 0");
  if (o.trace_capacity < 0) return fail(PDCS_ERR_INVALID, "trace_capacity must be >= 0");
  std::vector<pdcs_cone> rcv(row_cones, row_cones + n_row_cones);
  std::vector<pdcs_cone> ccv(col_cones, col_cones + n_col_cones);
  pdcs_handle* hd = new pdcs_handle();
  try {
    CK(cudaGetDevice(&hd->device));
    if (o.precision == 0) {
      auto* s = new Solver<double>();
      hd->solver = s;
      s->setup(m, n, row_ptr, col_idx, val, h, c, nb, lb, ub, rcv, ccv, o, (cudaStream_t)cuda_stream);
    } else {
      auto* s = new Solver<float>();
      hd->solver = s;
      s->setup(m, n, row_ptr, col_idx, val, h, c, nb, lb, ub, rcv, ccv, o, (cudaStream_t)cuda_stream);
    }
  } catch (const Fail& f) {
    delete hd->solver;
    delete hd;
    return fail(f.code, f.msg);
  }
  *out = hd;
  g_last_error.clear();
  return PDCS_OK;
}

#define PDCS_API_BODY(call)                                   \
  if (!hd || !hd->solver) return fail(PDCS_ERR_INVALID, "handle is NULL"); \
  try {                                                       \
    CK(cudaSetDevice(hd->device));                            \
    call;                                                     \
  } catch (const Fail& f) {                                   \
    return fail(f.code, f.msg);                               \
  }                                                           \
  return PDCS_OK;

int pdcs_solve(pdcs_handle* hd, const double* x0, const double* y0, double* x, double* y,
               double* s, pdcs_result* res) {
  PDCS_API_BODY(hd->solver->solve(x0, y0, x, y, s, res))
}

int pdcs_kkt(pdcs_handle* hd, const double* x, const double* y, pdcs_result* res) {
  PDCS_API_BODY(hd->solver->evaluate(x, y, res))
}

int pdcs_resume(pdcs_handle* hd, int64_t max_iter, double* x, double* y, double* s,
                pdcs_result* res) {
  PDCS_API_BODY(hd->solver->resume(max_iter, x, y, s, res))
}

int pdcs_get_state(pdcs_handle* hd, pdcs_state* state, double* x, double* y, double* x0,
                   double* y0, double* xs, double* ys) {
  PDCS_API_BODY(hd->solver->get_state(state, x, y, x0, y0, xs, ys))
}

int pdcs_set_state(pdcs_handle* hd, const pdcs_state* state, const double* x, const double* y,
                   const double* x0, const double* y0, const double* xs, const double* ys) {
  if (!state || !x || !x0 || !xs || ((!y || !y0 || !ys) && hd && hd->solver && hd->solver->m > 0))
    return fail(PDCS_ERR_INVALID, "state and all six vectors are required");
  if (!(state->omega > 0) || !(state->eta_hat > 0) || state->iter < 0 || state->kbar < 0 ||
      state->k < 0)
    return fail(PDCS_ERR_INVALID, "state has a non-positive step / weight or negative counter");
  PDCS_API_BODY(hd->solver->set_state(state, x, y, x0, y0, xs, ys))
}

int pdcs_get_iterate(pdcs_handle* hd, int32_t which, double* x, double* y) {
  if (which < 0 || which > 3) return fail(PDCS_ERR_INVALID, "which must be 0..3");
  PDCS_API_BODY(hd->solver->get_iterate(which, x, y))
}

int pdcs_get_trace(pdcs_handle* hd, double* out, int64_t cap, int64_t* count) {
  if (cap > 0 && !out) return fail(PDCS_ERR_INVALID, "out is NULL");
  PDCS_API_BODY(const int64_t k = hd->solver->get_trace(out, cap); if (count) *count = k)
}

int pdcs_get_profile(pdcs_handle* hd, pdcs_profile* prof) {
  if (!prof) return fail(PDCS_ERR_INVALID, "prof is NULL");
  PDCS_API_BODY(hd->solver->get_profile(prof))
}

int pdcs_get_kernel_times(pdcs_handle* hd, double* seconds, int64_t* launches, int32_t cap,
                          int32_t* count) {
  int k = 0;
  PDCS_API_BODY(k = hd->solver->get_kernel_times(seconds, launches, cap); if (count) *count = k)
}

int pdcs_get_sizes(pdcs_handle* hd, int64_t* m, int64_t* n, int64_t* nnz) {
  if (!hd || !hd->solver) return fail(PDCS_ERR_INVALID, "handle is NULL");
  if (m) *m = hd->solver->m;
  if (n) *n = hd->solver->n;
  if (nnz) *nnz = hd->solver->nnz;
  return PDCS_OK;
}

int pdcs_setup_batch(pdcs_handle** out, const pdcs_instance* inst, int64_t count,
                     const pdcs_options* opt, void* cuda_stream) {
  if (!out) return fail(PDCS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (count < 1 || !inst) return fail(PDCS_ERR_INVALID, "need count >= 1 instances");
  for (int64_t i = 0; i < count; ++i) {
    const pdcs_instance& I = inst[i];
    if (I.m < 0 || I.n < 1 || I.nb < 0 || I.nb > I.n)
      return fail(PDCS_ERR_INVALID, "batch instance " + std::to_string(i) + ": bad sizes");
    if (!I.row_ptr || (I.m > 0 && !I.h) || !I.c || (I.nb > 0 && (!I.lb || !I.ub)))
      return fail(PDCS_ERR_INVALID, "batch instance " + std::to_string(i) + ": missing array");
    if ((I.n_row_cones > 0 && !I.row_cones) || (I.n_col_cones > 0 && !I.col_cones) ||
        I.n_row_cones < 0 || I.n_col_cones < 0)
      return fail(PDCS_ERR_INVALID, "batch instance " + std::to_string(i) + ": bad cone list");
    int rc_ = check_cones(I.row_cones, I.n_row_cones, I.m, "row");
    if (rc_ != PDCS_OK) return rc_;
    rc_ = check_cones(I.col_cones, I.n_col_cones, I.n - I.nb, "column");
    if (rc_ != PDCS_OK) return rc_;
  }
  pdcs_options o;
  if (opt) o = *opt; else pdcs_default_options(&o);
  if (o.precision != 0 && o.precision != 1) return fail(PDCS_ERR_INVALID, "precision must be 0 or 1");
  if (o.check_freq < 1 || o.max_iter < 1 || o.ruiz_iters < 0 || !(o.bisect_rel_tol > 0.0) ||
      (o.method != 0 && o.method != 1))
    return fail(PDCS_ERR_INVALID, "invalid options");
  pdcs_handle* hd = new pdcs_handle();
  try {
    CK(cudaGetDevice(&hd->device));
    if (o.precision == 0) {
      auto* b = new BatchSolver<double>();
      hd->batch = b;
      b->setup(inst, count, o, (cudaStream_t)cuda_stream);
    } else {
      auto* b = new BatchSolver<float>();
      hd->batch = b;
      b->setup(inst, count, o, (cudaStream_t)cuda_stream);
    }
  } catch (const Fail& f) {
    delete hd->batch;
    delete hd;
    return fail(f.code, f.msg);
  }
  *out = hd;
  return PDCS_OK;
}

int pdcs_solve_batch(pdcs_handle* hd, double* x, double* y, double* s, pdcs_result* res,
                     double* finish_s) {
  if (!hd || !hd->batch) return fail(PDCS_ERR_INVALID, "not a batch handle");
  try {
    CK(cudaSetDevice(hd->device));
    hd->batch->solve(x, y, s, res, finish_s);
  } catch (const Fail& f) {
    return fail(f.code, f.msg);
  }
  return PDCS_OK;
}

void pdcs_free(pdcs_handle* hd) {
  if (!hd) return;
  if (hd->solver || hd->batch) {
    cudaSetDevice(hd->device);
    delete hd->solver;
    delete hd->batch;
  }
  delete hd;
}

}  // extern "C"
