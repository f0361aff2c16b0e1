// Warm-start network: a fully connected ReLU network mapping a problem
// instance's parameters to a starting point (x0, y0) of the solver, trained on
// (parameter, solution) pairs the solver produces (include/pdcs.h,
// pdcs_mlp_*).  The paper has no such network; it is the learned warm start
// built around the solver.
//
// Layers l = 0 .. L-1 map d_l -> d_{l+1} features: H_{l+1} = relu(H_l W_l^T + b_l)
// for the hidden layers and Y = H_{L-1} W_{L-1}^T + b_{L-1} for the output.
// Weights W_l are stored [d_{l+1} x d_l] (row-major, inputs contiguous, rows
// padded to a multiple of 8 elements), so every product is C = A B^T with both
// operands K-major: the forward pass, dH_l = dPre_{l+1} W_l (with the
// transposed copy W_l^T) and dW_l = dPre_{l+1}^T H_l (with transposed
// activations), all on the tcgen05 GEMM of gemm_tc.cuh.  Activations and the
// GEMM operands are BF16, accumulation FP32; master weights, biases, gradients
// and the Adam moments are FP32.  Loss: mean squared error over the batch and
// the outputs.  Reductions (loss, bias gradients) have a fixed order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/pdcs.h"
#include "gemm_tc.cuh"

namespace pdcs {
extern thread_local std::string g_last_error;  // defined with the rest of the ABI
}

namespace {

using pdcs::tc::EpiArgs;

struct MlpFail {
  int code;
  std::string msg;
};

void ck(cudaError_t e, const char* what, int line) {
  if (e != cudaSuccess) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s failed (line %d): %s", what, line, cudaGetErrorString(e));
    throw MlpFail{e == cudaErrorMemoryAllocation ? PDCS_ERR_NOMEM : PDCS_ERR_CUDA, buf};
  }
}
#define MCK(call) ck((call), #call, __LINE__)

inline int64_t up8(int64_t v) { return (v + 7) / 8 * 8; }
inline unsigned grid_for(int64_t n, int threads = 256) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 148 * 32));
}

#define MLP_LOOP(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// SplitMix64 (Steele, Lea and Flood, 2014): a counter-based 64-bit generator.
__device__ inline uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// W (rows x cols, FP32) ~ U(-a, a) from counter (seed, layer, index).
__global__ void k_init_uniform(float* w, int64_t count, float a, uint64_t seed) {
  MLP_LOOP(i, count) {
    const uint64_t r = splitmix64(seed ^ splitmix64((uint64_t)i));
    const float u = (float)((r >> 40) * (1.0 / 16777216.0));  // [0, 1)
    w[i] = (2.0f * u - 1.0f) * a;
  }
}

__global__ void k_fill_f32(float* p, int64_t n, float v) {
  MLP_LOOP(i, n) p[i] = v;
}

// dst[r * ldd + c] = bf16(src[r * cols + c]) for a rows x cols FP32 matrix.
__global__ void k_to_bf16(const float* __restrict__ src, int64_t rows, int64_t cols,
                          __nv_bfloat16* __restrict__ dst, int64_t ldd) {
  MLP_LOOP(i, rows * cols) {
    const int64_t r = i / cols, c = i - r * cols;
    dst[r * ldd + c] = __float2bfloat16(src[i]);
  }
}

// dst[c * ldd + r] = src[r * lds + c] (rows x cols BF16), 32 x 32 tiles
// through shared memory.  Grid: (ceil(cols / 32), ceil(rows / 32)), 32 x 8 threads.
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ src, int64_t rows, int64_t cols,
                                 int64_t lds, __nv_bfloat16* __restrict__ dst, int64_t ldd) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int64_t r = r0 + j, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[j][threadIdx.x] = src[r * lds + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int64_t c = c0 + j, r = r0 + threadIdx.x;
    if (r < rows && c < cols) dst[c * ldd + r] = tile[threadIdx.x][j];
  }
}

// Loss and output gradient: e = Y - T, dY = 2 e / (B * out) (FP32 and BF16),
// per-CTA partial sums of e^2 (added in CTA order by k_loss_finish).
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ Y, const float* __restrict__ T,
                                             int64_t B, int64_t out, float* __restrict__ dY,
                                             __nv_bfloat16* __restrict__ dYb, int64_t lddb,
                                             double* __restrict__ part) {
  __shared__ double sh[256];
  const float scale = 2.0f / (float)((double)B * (double)out);
  double s = 0.0;
  MLP_LOOP(i, B * out) {
    const float e = Y[i] - T[i];
    s += (double)e * (double)e;
    const float g = scale * e;
    dY[i] = g;
    const int64_t r = i / out, c = i - r * out;
    dYb[r * lddb + c] = __float2bfloat16(g);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// One CTA of 256 threads: thread t adds partials t, t + 256, ... in order,
// then a fixed tree (deterministic).
__global__ void __launch_bounds__(256) k_loss_finish(const double* __restrict__ part, int nparts,
                                                     double denom, double* __restrict__ loss) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 256) s += part[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = sh[0] / denom;
}

// db[c] = sum over rows of G[r, c] (FP32 or BF16 G), rows in order.
template <typename G>
__global__ void k_colsum(const G* __restrict__ g, int64_t rows, int64_t cols, int64_t ld,
                         float* __restrict__ db) {
  MLP_LOOP(c, cols) {
    float s = 0.0f;
    for (int64_t r = 0; r < rows; ++r) s += (float)g[r * ld + c];
    db[c] = s;
  }
}

// Adam (Kingma and Ba, 2015, Algorithm 1) on FP32 parameters:
// m <- b1 m + (1 - b1) g; v <- b2 v + (1 - b2) g^2;
// p <- p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
// When wb is given, also writes the BF16 copy (row length cols, ld ldw).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t count, int64_t cols, float lr, float b1,
                       float b2, float eps, float c1, float c2, __nv_bfloat16* __restrict__ wb,
                       int64_t ldw) {
  MLP_LOOP(i, count) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (wb) {
      const int64_t r = i / cols, c = i - r * cols;
      wb[r * ldw + c] = __float2bfloat16(pi);
    }
  }
}

struct Layer {
  int64_t din = 0, dout = 0, ldin = 0, ldout = 0;  // ld* = up8(d*)
  float *w = nullptr, *b = nullptr;                 // master FP32 [dout x din], [dout]
  float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;
  float *gw = nullptr, *gb = nullptr;               // gradients
  __nv_bfloat16 *wb = nullptr, *wt = nullptr;       // BF16 [dout x ldin], transposed [din x ldout]
};

struct Mlp {
  pdcs_mlp_config cfg;
  cudaStream_t st = nullptr;
  std::vector<void*> allocs;
  std::vector<Layer> L;
  int64_t bmax = 0, bpad = 0;
  // activations: act[0] = X, act[l] = H_l (BF16, [bmax x ld_l]); Y, T, dY FP32
  std::vector<__nv_bfloat16*> act, actT, dpre;
  float *Y = nullptr, *T = nullptr, *dY = nullptr, *xin = nullptr;
  double *part = nullptr, *loss = nullptr;
  int* err = nullptr;
  int64_t step = 0;
  int nparts = 0;

  template <typename U>
  U* alloc(int64_t count) {
    void* p = nullptr;
    MCK(cudaMalloc(&p, (size_t)std::max<int64_t>(count, 1) * sizeof(U)));
    allocs.push_back(p);
    return static_cast<U*>(p);
  }

  ~Mlp() {
    for (void* p : allocs) cudaFree(p);
    if (st) cudaStreamDestroy(st);
  }

  void setup(const pdcs_mlp_config& c, cudaStream_t user) {
    cfg = c;
    MCK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    if (user) {
      cudaEvent_t ev;
      MCK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      MCK(cudaEventRecord(ev, user));
      MCK(cudaStreamWaitEvent(st, ev, 0));
      MCK(cudaEventDestroy(ev));
    }
    MCK(cudaFuncSetAttribute(pdcs::tc::k_gemm_bf16_tn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             pdcs::tc::kGemmSmem));
    std::vector<int64_t> dims;
    dims.push_back(c.in_dim);
    for (int i = 0; i < c.n_hidden; ++i) dims.push_back(c.hidden);
    dims.push_back(c.out_dim);
    bmax = c.max_batch;
    bpad = up8(bmax);
    L.resize(dims.size() - 1);
    for (size_t l = 0; l < L.size(); ++l) {
      Layer& y = L[l];
      y.din = dims[l];
      y.dout = dims[l + 1];
      y.ldin = up8(y.din);
      y.ldout = up8(y.dout);
      const int64_t nw = y.din * y.dout;
      y.w = alloc<float>(nw);
      y.mw = alloc<float>(nw);
      y.vw = alloc<float>(nw);
      y.gw = alloc<float>(nw);
      y.b = alloc<float>(y.dout);
      y.mb = alloc<float>(y.dout);
      y.vb = alloc<float>(y.dout);
      y.gb = alloc<float>(y.dout);
      y.wb = alloc<__nv_bfloat16>(y.dout * y.ldin);
      y.wt = alloc<__nv_bfloat16>(y.din * y.ldout);
      MCK(cudaMemsetAsync(y.wb, 0, sizeof(__nv_bfloat16) * y.dout * y.ldin, st));
      MCK(cudaMemsetAsync(y.wt, 0, sizeof(__nv_bfloat16) * y.din * y.ldout, st));
      // Glorot-uniform weights, zero biases
      const float a = (float)std::sqrt(6.0 / (double)(y.din + y.dout));
      k_init_uniform<<<grid_for(nw), 256, 0, st>>>(y.w, nw, a, c.seed * 1315423911ull + l);
      k_fill_f32<<<grid_for(y.dout), 256, 0, st>>>(y.b, y.dout, 0.0f);
    }
    reset_moments();
    for (size_t l = 0; l < L.size(); ++l) refresh_bf16((int)l);
    act.resize(dims.size() - 1);
    actT.resize(dims.size() - 1);
    dpre.resize(dims.size());
    for (size_t l = 0; l + 1 < dims.size(); ++l) {
      act[l] = alloc<__nv_bfloat16>(bmax * up8(dims[l]));
      actT[l] = alloc<__nv_bfloat16>(dims[l] * bpad);
      dpre[l + 1] = alloc<__nv_bfloat16>(bmax * up8(dims[l + 1]));
    }
    Y = alloc<float>(bmax * c.out_dim);
    T = alloc<float>(bmax * c.out_dim);
    dY = alloc<float>(bmax * c.out_dim);
    xin = alloc<float>(bmax * c.in_dim);
    nparts = (int)grid_for(bmax * c.out_dim);
    part = alloc<double>(nparts);
    loss = alloc<double>(1);
    err = alloc<int>(1);
    MCK(cudaMemsetAsync(err, 0, sizeof(int), st));
    MCK(cudaStreamSynchronize(st));
  }

  void reset_moments() {
    for (auto& y : L) {
      MCK(cudaMemsetAsync(y.mw, 0, sizeof(float) * y.din * y.dout, st));
      MCK(cudaMemsetAsync(y.vw, 0, sizeof(float) * y.din * y.dout, st));
      MCK(cudaMemsetAsync(y.mb, 0, sizeof(float) * y.dout, st));
      MCK(cudaMemsetAsync(y.vb, 0, sizeof(float) * y.dout, st));
    }
    step = 0;
  }

  // BF16 copy and transposed copy of layer l's master weights.
  void refresh_bf16(int l) {
    Layer& y = L[l];
    k_to_bf16<<<grid_for(y.din * y.dout), 256, 0, st>>>(y.w, y.dout, y.din, y.wb, y.ldin);
    transpose(y.wb, y.dout, y.din, y.ldin, y.wt, y.ldout);
  }

  void transpose(const __nv_bfloat16* src, int64_t rows, int64_t cols, int64_t lds,
                 __nv_bfloat16* dst, int64_t ldd) {
    dim3 g((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    k_transpose_bf16<<<g, dim3(32, 8), 0, st>>>(src, rows, cols, lds, dst, ldd);
  }

  // Split-K when the output has fewer tiles than SMs and K is long: about two
  // CTAs per SM in all, each slice at least 8 K blocks; the FP32 partial
  // tiles go to `splitws` and k_splitk_reduce applies the epilogue.
  float* splitws = nullptr;
  int64_t splitws_len = 0;

  void gemm(const __nv_bfloat16* A, const __nv_bfloat16* Bm, int64_t M, int64_t N, int64_t K,
            int64_t lda, int64_t ldb, EpiArgs ep) {
    const int64_t tn = (N + pdcs::tc::kTileN - 1) / pdcs::tc::kTileN;
    const int64_t tm = (M + pdcs::tc::kTileM - 1) / pdcs::tc::kTileM;
    const int64_t nkb = (K + pdcs::tc::kTileK - 1) / pdcs::tc::kTileK;
    CUtensorMap ta, tb;
    if (!pdcs::tc::make_kmajor_map(&ta, A, M, K, lda) || !pdcs::tc::make_kmajor_map(&tb, Bm, N, K, ldb))
      throw MlpFail{PDCS_ERR_CUDA, "cuTensorMapEncodeTiled refused a GEMM operand"};
    int64_t splits = 1;
    if (tn * tm < 148 && nkb >= 16) splits = std::min<int64_t>(nkb / 8, (2 * 148 + tn * tm - 1) / (tn * tm));
    // stages: as many as a CTA has K blocks, up to the maximum; grids of two
    // or more CTAs per SM take at most two, so three CTAs fit on an SM
    auto stages = [&](int64_t nk_cta, int64_t ctas) {
      const int64_t cap = ctas >= 2 * 148 ? 2 : pdcs::tc::kStages;
      return (int)std::max<int64_t>(1, std::min<int64_t>(nk_cta, cap));
    };
    if (splits <= 1) {
      const int nst = stages(nkb, tn * tm);
      pdcs::tc::k_gemm_bf16_tn<<<dim3((unsigned)tn, (unsigned)tm), pdcs::tc::kThreads,
                                 pdcs::tc::gemm_smem(nst), st>>>(ta, tb, M, N, K, ep, err, 0, 0, nst);
      return;
    }
    const int64_t kchunk = (nkb + splits - 1) / splits * pdcs::tc::kTileK;
    splits = (K + kchunk - 1) / kchunk;
    const int nst = stages(kchunk / pdcs::tc::kTileK, tn * tm * splits);
    const int64_t zstride = M * N;
    if (splits * zstride > splitws_len) {
      splitws_len = splits * zstride;
      splitws = alloc<float>(splitws_len);
    }
    EpiArgs part{pdcs::tc::EPI_F32, splitws, N, nullptr, nullptr, 0};
    pdcs::tc::k_gemm_bf16_tn<<<dim3((unsigned)tn, (unsigned)tm, (unsigned)splits), pdcs::tc::kThreads,
                               pdcs::tc::gemm_smem(nst), st>>>(ta, tb, M, N, K, part, err, kchunk, zstride,
                                                               nst);
    pdcs::tc::k_splitk_reduce<<<grid_for(M * N), 256, 0, st>>>(splitws, (int)splits, M, N, zstride, ep);
  }

  void check_err() {
    int h = 0;
    MCK(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    if (h) {
      MCK(cudaMemsetAsync(err, 0, sizeof(int), st));
      throw MlpFail{PDCS_ERR_TIMEOUT, "a tensor-core GEMM wait gave up"};
    }
  }

  // Inputs (FP32, host or device, batch x in_dim) -> act[0] (BF16).
  void load_inputs(const float* X, int64_t B) {
    MCK(cudaMemcpyAsync(xin, X, sizeof(float) * B * cfg.in_dim, cudaMemcpyDefault, st));
    k_to_bf16<<<grid_for(B * cfg.in_dim), 256, 0, st>>>(xin, B, cfg.in_dim, act[0], up8(cfg.in_dim));
  }

  void forward(int64_t B) {
    const int nl = (int)L.size();
    for (int l = 0; l < nl; ++l) {
      Layer& y = L[l];
      if (l + 1 < nl) {
        EpiArgs ep{pdcs::tc::EPI_BF16_BIAS_RELU, act[l + 1], y.ldout, y.b, nullptr, 0};
        gemm(act[l], y.wb, B, y.dout, y.din, y.ldin, y.ldin, ep);
      } else {
        EpiArgs ep{pdcs::tc::EPI_F32_BIAS, Y, y.dout, y.b, nullptr, 0};
        gemm(act[l], y.wb, B, y.dout, y.din, y.ldin, y.ldin, ep);
      }
    }
  }

  // Forward, loss and every gradient (no update).
  void gradients(const float* X, const float* Tt, int64_t B) {
    load_inputs(X, B);
    MCK(cudaMemcpyAsync(T, Tt, sizeof(float) * B * cfg.out_dim, cudaMemcpyDefault, st));
    forward(B);
    const int nl = (int)L.size();
    const int np = (int)grid_for(B * cfg.out_dim);
    k_mse<<<np, 256, 0, st>>>(Y, T, B, cfg.out_dim, dY, dpre[nl], up8(cfg.out_dim), part);
    k_loss_finish<<<1, 256, 0, st>>>(part, np, (double)B * (double)cfg.out_dim, loss);
    for (int l = nl - 1; l >= 0; --l) {
      Layer& y = L[l];
      const __nv_bfloat16* Gb = dpre[l + 1];  // dLoss / d(pre-activation of layer l), B x dout
      // dW_l = G^T H_l: A = G^T [dout x B], B-operand = H_l^T [din x B], K = B
      transpose(act[l], B, y.din, y.ldin, actT[l], bpad);
      __nv_bfloat16* Gt = gt_buffer(l);
      transpose(Gb, B, y.dout, y.ldout, Gt, bpad);
      EpiArgs ew{pdcs::tc::EPI_F32, y.gw, y.din, nullptr, nullptr, 0};
      gemm(Gt, actT[l], y.dout, y.din, B, bpad, bpad, ew);
      if (l == nl - 1) k_colsum<float><<<grid_for(y.dout), 256, 0, st>>>(dY, B, y.dout, y.dout, y.gb);
      else k_colsum<__nv_bfloat16><<<grid_for(y.dout), 256, 0, st>>>(Gb, B, y.dout, y.ldout, y.gb);
      if (l > 0) {
        // dPre_l = (G W_l) o [H_l > 0]: A = G [B x dout], B-operand = W_l^T [din x dout]
        EpiArgs eh{pdcs::tc::EPI_BF16_RELU_MASK, dpre[l], y.ldin, nullptr, act[l], y.ldin};
        gemm(Gb, y.wt, B, y.din, y.dout, y.ldout, y.ldout, eh);
      }
    }
  }

  // Transposed-gradient scratch: G_l^T has dout_l rows of bpad.
  std::vector<__nv_bfloat16*> gtb;
  __nv_bfloat16* gt_buffer(int l) {
    if (gtb.empty()) {
      gtb.resize(L.size());
      for (size_t i = 0; i < L.size(); ++i) gtb[i] = alloc<__nv_bfloat16>(L[i].dout * bpad);
    }
    return gtb[l];
  }

  void adam_update() {
    ++step;
    const double c1 = 1.0 - std::pow(cfg.beta1, (double)step), c2 = 1.0 - std::pow(cfg.beta2, (double)step);
    for (size_t l = 0; l < L.size(); ++l) {
      Layer& y = L[l];
      k_adam<<<grid_for(y.din * y.dout), 256, 0, st>>>(y.w, y.gw, y.mw, y.vw, y.din * y.dout, y.din,
                                                       (float)cfg.lr, (float)cfg.beta1, (float)cfg.beta2,
                                                       (float)cfg.eps, (float)c1, (float)c2, y.wb, y.ldin);
      k_adam<<<grid_for(y.dout), 256, 0, st>>>(y.b, y.gb, y.mb, y.vb, y.dout, y.dout, (float)cfg.lr,
                                               (float)cfg.beta1, (float)cfg.beta2, (float)cfg.eps,
                                               (float)c1, (float)c2, nullptr, 0);
      transpose(y.wb, y.dout, y.din, y.ldin, y.wt, y.ldout);
    }
  }
};

int mlp_fail(int code, const std::string& msg) {
  pdcs::g_last_error = msg;
  return code;
}

#define MLP_BODY(call)                                         \
  if (!net) return mlp_fail(PDCS_ERR_INVALID, "network is NULL"); \
  try {                                                        \
    call;                                                      \
  } catch (const MlpFail& f) {                                 \
    return mlp_fail(f.code, f.msg);                            \
  }                                                            \
  return PDCS_OK;

}  // namespace

struct pdcs_mlp {
  int device = 0;
  Mlp* net = nullptr;
};

extern "C" {

void pdcs_mlp_default_config(pdcs_mlp_config* c) {
  if (!c) return;
  c->in_dim = 0;
  c->hidden = 512;
  c->n_hidden = 3;
  c->pad = 0;
  c->out_dim = 0;
  c->max_batch = 256;
  c->lr = 1e-3;
  c->beta1 = 0.9;
  c->beta2 = 0.999;
  c->eps = 1e-8;
  c->seed = 20260105ull;
}

int pdcs_mlp_create(pdcs_mlp** out, const pdcs_mlp_config* cfg, void* cuda_stream) {
  if (!out || !cfg) return mlp_fail(PDCS_ERR_INVALID, "pdcs_mlp_create: NULL argument");
  *out = nullptr;
  if (cfg->in_dim < 1 || cfg->out_dim < 1 || cfg->hidden < 1 || cfg->n_hidden < 1 ||
      cfg->max_batch < 1)
    return mlp_fail(PDCS_ERR_INVALID, "pdcs_mlp_create: dimensions and max_batch must be >= 1");
  if (!(cfg->lr > 0) || !(cfg->beta1 >= 0 && cfg->beta1 < 1) || !(cfg->beta2 >= 0 && cfg->beta2 < 1) ||
      !(cfg->eps > 0))
    return mlp_fail(PDCS_ERR_INVALID, "pdcs_mlp_create: invalid Adam parameters");
  auto* h = new pdcs_mlp;
  try {
    ck(cudaGetDevice(&h->device), "cudaGetDevice", __LINE__);
    h->net = new Mlp;
    h->net->setup(*cfg, static_cast<cudaStream_t>(cuda_stream));
  } catch (const MlpFail& f) {
    delete h->net;
    delete h;
    return mlp_fail(f.code, f.msg);
  }
  *out = h;
  return PDCS_OK;
}

int pdcs_mlp_train_step(pdcs_mlp* h, const float* X, const float* T, int64_t batch, double* loss) {
  Mlp* net = h ? h->net : nullptr;
  if (net && (!X || !T || batch < 1 || batch > net->bmax))
    return mlp_fail(PDCS_ERR_INVALID, "pdcs_mlp_train_step: NULL data or batch outside [1, max_batch]");
  MLP_BODY(ck(cudaSetDevice(h->device), "cudaSetDevice", __LINE__); net->gradients(X, T, batch);
           net->adam_update();
           if (loss) ck(cudaMemcpyAsync(loss, net->loss, sizeof(double), cudaMemcpyDefault, net->st),
                        "copy loss", __LINE__);
           net->check_err())
}

int pdcs_mlp_gradients(pdcs_mlp* h, const float* X, const float* T, int64_t batch, int32_t layer,
                       float* dW, float* db, double* loss) {
  Mlp* net = h ? h->net : nullptr;
  if (net && (!X || !T || batch < 1 || batch > net->bmax || layer < 0 || layer >= (int)net->L.size()))
    return mlp_fail(PDCS_ERR_INVALID, "pdcs_mlp_gradients: bad data, batch or layer");
  MLP_BODY(ck(cudaSetDevice(h->device), "cudaSetDevice", __LINE__); net->gradients(X, T, batch);
           const Layer& y = net->L[layer];
           if (dW) ck(cudaMemcpyAsync(dW, y.gw, sizeof(float) * y.din * y.dout, cudaMemcpyDefault, net->st),
                      "copy dW", __LINE__);
           if (db) ck(cudaMemcpyAsync(db, y.gb, sizeof(float) * y.dout, cudaMemcpyDefault, net->st),
                      "copy db", __LINE__);
           if (loss) ck(cudaMemcpyAsync(loss, net->loss, sizeof(double), cudaMemcpyDefault, net->st),
                        "copy loss", __LINE__);
           net->check_err())
}

int pdcs_mlp_predict(pdcs_mlp* h, const float* X, int64_t batch, float* Y) {
  Mlp* net = h ? h->net : nullptr;
  if (net && (!X || !Y || batch < 1 || batch > net->bmax))
    return mlp_fail(PDCS_ERR_INVALID, "pdcs_mlp_predict: NULL data or batch outside [1, max_batch]");
  MLP_BODY(ck(cudaSetDevice(h->device), "cudaSetDevice", __LINE__); net->load_inputs(X, batch);
           net->forward(batch);
           ck(cudaMemcpyAsync(Y, net->Y, sizeof(float) * batch * net->cfg.out_dim, cudaMemcpyDefault,
                              net->st),
              "copy Y", __LINE__);
           net->check_err())
}

int pdcs_mlp_get_layer(pdcs_mlp* h, int32_t layer, float* W, float* b) {
  Mlp* net = h ? h->net : nullptr;
  if (net && (layer < 0 || layer >= (int)net->L.size()))
    return mlp_fail(PDCS_ERR_INVALID, "pdcs_mlp_get_layer: bad layer");
  MLP_BODY(ck(cudaSetDevice(h->device), "cudaSetDevice", __LINE__); const Layer& y = net->L[layer];
           if (W) ck(cudaMemcpyAsync(W, y.w, sizeof(float) * y.din * y.dout, cudaMemcpyDefault, net->st),
                     "copy W", __LINE__);
           if (b) ck(cudaMemcpyAsync(b, y.b, sizeof(float) * y.dout, cudaMemcpyDefault, net->st),
                     "copy b", __LINE__);
           ck(cudaStreamSynchronize(net->st), "sync", __LINE__))
}

int pdcs_mlp_set_layer(pdcs_mlp* h, int32_t layer, const float* W, const float* b) {
  Mlp* net = h ? h->net : nullptr;
  if (net && (layer < 0 || layer >= (int)net->L.size() || !W || !b))
    return mlp_fail(PDCS_ERR_INVALID, "pdcs_mlp_set_layer: bad layer or NULL data");
  MLP_BODY(ck(cudaSetDevice(h->device), "cudaSetDevice", __LINE__); Layer& y = net->L[layer];
           ck(cudaMemcpyAsync(y.w, W, sizeof(float) * y.din * y.dout, cudaMemcpyDefault, net->st),
              "copy W", __LINE__);
           ck(cudaMemcpyAsync(y.b, b, sizeof(float) * y.dout, cudaMemcpyDefault, net->st), "copy b",
              __LINE__);
           net->refresh_bf16(layer); net->reset_moments();
           ck(cudaStreamSynchronize(net->st), "sync", __LINE__))
}

void pdcs_mlp_free(pdcs_mlp* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  delete h->net;
  delete h;
}

}  // extern "C"
