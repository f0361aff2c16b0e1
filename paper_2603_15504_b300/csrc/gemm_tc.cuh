// BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a):
//   C[M x N] = A[M x K] * B[N x K]^T   (A and B row-major with K contiguous),
// FP32 accumulation in tensor memory (TMEM), with a fused epilogue.
//
// One CTA of 128 threads (4 warps) computes a 128 x 128 tile of C.  K is
// walked in blocks of 64: the threads copy the A and B blocks from global
// memory into shared memory in the canonical K-major layout without swizzle
// (8-row x 16-byte core matrices; core matrices adjacent along K are 128 bytes
// apart, along M / N 1024 bytes apart), two stages deep; one thread issues the
// four 128 x 128 x 16 MMAs of a block and commits them to the stage's
// mbarrier, which the threads wait on before they overwrite that stage.  The
// accumulator tile occupies 128 TMEM columns; at the end warp w reads lanes
// 32w .. 32w + 31 (rows of C) with tcgen05.ld and applies the epilogue.
// Every mbarrier wait is bounded: on expiry the kernel records an error,
// stops issuing work, waits (bounded) for its last commit and still frees its
// TMEM.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pdcs {
namespace tc {

constexpr int kTileM = 128, kTileN = 128, kTileK = 64, kThreads = 128;
constexpr int kStageBytes = kTileM * kTileK * 2;  // 16 KB per operand per stage
constexpr uint32_t kLBO = 128, kSBO = 1024;        // canonical no-swizzle K-major layout
constexpr unsigned long long kSpinLimit = 1ull << 26;

// Epilogues.  out[r * ldc + c] for r < M, c < N:
enum Epi : int {
  EPI_F32 = 0,        // v (FP32)
  EPI_BF16_BIAS_RELU, // bf16(max(v + bias[c], 0))
  EPI_F32_BIAS,       // v + bias[c] (FP32)
  EPI_BF16_RELU_MASK  // bf16(v * (mask[r * ldm + c] > 0)): ReLU backward
};

struct EpiArgs {
  int kind;
  void* out;
  int64_t ldc;
  const float* bias;
  const __nv_bfloat16* mask;
  int64_t ldm;
};

// Shared-memory matrix descriptor (tcgen05): start address >> 4 in bits 0-13,
// leading byte offset >> 4 in 16-29, stride byte offset >> 4 in 32-45, the
// descriptor version 1 in bits 46-47, no swizzle (bits 61-63 = 0).
__host__ __device__ inline uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ inline uint32_t instr_desc_bf16(int m, int n) {
  uint32_t d = 0;
  d |= 1u << 4;
  d |= 1u << 7;
  d |= 1u << 10;
  d |= (uint32_t)(n >> 3) << 17;
  d |= (uint32_t)(m >> 4) << 24;
  return d;
}

// Byte offset of element (row r, k) of a 128 x 64 block in the canonical layout.
__host__ __device__ inline uint32_t canon_off(int r, int k) {
  return (uint32_t)((r >> 3) * kSBO + (k >> 3) * kLBO + (r & 7) * 16 + (k & 7) * 2);
}

#ifdef __CUDA_ARCH__
__device__ inline uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Bounded wait for the phase with the given parity; false on expiry.
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (unsigned long long i = 0; i < kSpinLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ inline void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ inline void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ inline void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ inline void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                              uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ inline void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ inline void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Copy rows [row0, row0 + 128) x columns [k0, k0 + 64) of a row-major
// rows x K BF16 matrix (leading dimension ld, a multiple of 8) into the
// canonical layout at dst; out-of-range elements are zero.  Thread t copies
// 16-byte pieces v = t, t + 128, ...: chunk c = v / 128 (8 elements of K),
// row r = v % 128, so a warp's stores fill 512 contiguous bytes.
__device__ inline void load_block(uint8_t* dst, const __nv_bfloat16* __restrict__ src, int64_t rows,
                                  int64_t K, int64_t ld, int64_t row0, int64_t k0) {
#pragma unroll
  for (int i = 0; i < (kTileM * kTileK / 8) / kThreads; ++i) {
    const int v = threadIdx.x + i * kThreads;
    const int c = v / kTileM, r = v % kTileM;
    const int64_t gr = row0 + r, gk = k0 + c * 8;
    uint4 val = make_uint4(0u, 0u, 0u, 0u);
    if (gr < rows && gk < K) {
      const __nv_bfloat16* p = src + gr * ld + gk;
      if (gk + 8 <= K) {
        val = __ldg(reinterpret_cast<const uint4*>(p));
      } else {
        __nv_bfloat16 tmp[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) tmp[e] = gk + e < K ? p[e] : __float2bfloat16(0.0f);
        val = *reinterpret_cast<uint4*>(tmp);
      }
    }
    *reinterpret_cast<uint4*>(dst + canon_off(r, c * 8)) = val;
  }
}
#endif

// C = A * B^T with the epilogue; A: M x K (lda), B: N x K (ldb), K, lda, ldb
// multiples of 8, A and B 16-byte aligned.  Grid: (ceil(N / 128), ceil(M / 128),
// splits).  Split-K (kchunk > 0, a multiple of 64): CTA z multiplies the K
// slice [z kchunk, (z + 1) kchunk) and writes its FP32 partial tile (EPI_F32)
// at ep.out + z * zstride floats; k_splitk_reduce adds the slices.
// err: set to 1 if an mbarrier wait expired (the tile is then not written).
__global__ void __launch_bounds__(kThreads) k_gemm_bf16_tn(const __nv_bfloat16* __restrict__ A,
                                                           const __nv_bfloat16* __restrict__ B,
                                                           int64_t M, int64_t N, int64_t K,
                                                           int64_t lda, int64_t ldb, EpiArgs ep,
                                                           int* err, int64_t kchunk, int64_t zstride) {
#ifdef __CUDA_ARCH__
  if (kchunk > 0) {
    const int64_t kz = (int64_t)blockIdx.z * kchunk;
    A += kz;
    B += kz;
    K = K - kz < kchunk ? K - kz : kchunk;
    ep.out = reinterpret_cast<float*>(ep.out) + (int64_t)blockIdx.z * zstride;
  }
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte aligned stages: A0 B0 A1 B1
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sa[2] = {base, base + 2 * kStageBytes};
  uint8_t* sb[2] = {base + kStageBytes, base + 3 * kStageBytes};
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t m0 = (int64_t)blockIdx.y * kTileM, n0 = (int64_t)blockIdx.x * kTileN;
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(kTileN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = instr_desc_bf16(kTileM, kTileN);
  const int nk = (int)((K + kTileK - 1) / kTileK);
  int issued = 0;  // commits issued (thread 0's count; the same for all threads)
  for (int kb = 0; kb < nk; ++kb) {
    const int s = kb & 1;
    if (kb >= 2) {
      // the MMAs that read this stage (block kb - 2) must have completed
      if (!mbar_wait(&bar[s], (uint32_t)(((kb - 2) >> 1) & 1))) atomicExch(&failed, 1);
    }
    __syncthreads();
    if (failed) break;  // uniform after the barrier
    load_block(sa[s], A, M, K, lda, m0, (int64_t)kb * kTileK);
    load_block(sb[s], B, N, K, ldb, n0, (int64_t)kb * kTileK);
    fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sa[s]), b0 = smem_u32(sb[s]);
#pragma unroll
      for (int j = 0; j < kTileK / 16; ++j) {
        // 16 elements of K = two core matrices = 2 * LBO bytes
        tc_mma(tmem, smem_desc(a0 + j * 2 * kLBO, kLBO, kSBO), smem_desc(b0 + j * 2 * kLBO, kLBO, kSBO),
               idesc, (kb > 0 || j > 0) ? 1u : 0u);
      }
      tc_commit(&bar[s]);
    }
    ++issued;
  }
  // wait for the last commit (it tracks every MMA issued before it)
  if (issued > 0) {
    const int kl = issued - 1;
    if (!mbar_wait(&bar[kl & 1], (uint32_t)((kl >> 1) & 1))) atomicExch(&failed, 1);
  }
  __syncthreads();
  tc_fence_after();
  if (!failed && issued == nk && nk > 0) {
    const int64_t r = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < kTileN; c0 += 16) {
      float v[16];
      tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (r >= M) continue;
      const int64_t cb = n0 + c0;
      if (ep.kind == EPI_F32 || ep.kind == EPI_F32_BIAS) {
        float* o = reinterpret_cast<float*>(ep.out) + r * ep.ldc;
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (cb + i < N) o[cb + i] = v[i] + (ep.kind == EPI_F32_BIAS ? ep.bias[cb + i] : 0.0f);
      } else {
        __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(ep.out) + r * ep.ldc;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          if (cb + i >= N) continue;
          float x = v[i];
          if (ep.kind == EPI_BF16_BIAS_RELU) x = fmaxf(x + ep.bias[cb + i], 0.0f);
          else if (__bfloat162float(ep.mask[r * ep.ldm + cb + i]) <= 0.0f) x = 0.0f;
          o[cb + i] = __float2bfloat16(x);
        }
      }
    }
  }
  if (failed && t == 0) atomicExch(err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTileN)
                 : "memory");
  }
#endif
}

// Split-K epilogue: v = sum over the slices z (in order) of part[z][r][c], then
// the epilogue of ep (r < M, c < N; the slices have leading dimension N).
__global__ void k_splitk_reduce(const float* __restrict__ part, int splits, int64_t M, int64_t N,
                                int64_t zstride, EpiArgs ep) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M * N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / N, c = i - r * N;
    float v = 0.0f;
    for (int z = 0; z < splits; ++z) v += part[z * zstride + i];
    if (ep.kind == EPI_F32) {
      reinterpret_cast<float*>(ep.out)[r * ep.ldc + c] = v;
    } else if (ep.kind == EPI_F32_BIAS) {
      reinterpret_cast<float*>(ep.out)[r * ep.ldc + c] = v + ep.bias[c];
    } else {
      if (ep.kind == EPI_BF16_BIAS_RELU) v = fmaxf(v + ep.bias[c], 0.0f);
      else if (__bfloat162float(ep.mask[r * ep.ldm + c]) <= 0.0f) v = 0.0f;
      reinterpret_cast<__nv_bfloat16*>(ep.out)[r * ep.ldc + c] = __float2bfloat16(v);
    }
  }
}

// Dynamic shared memory of k_gemm_bf16_tn (two stages of A and B, plus the
// 1024-byte alignment slack).
constexpr int kGemmSmem = 4 * kStageBytes + 1024;

}  // namespace tc
}  // namespace pdcs
