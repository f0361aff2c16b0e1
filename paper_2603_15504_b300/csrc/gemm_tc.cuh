// BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a):
//   C[M x N] = A[M x K] * B[N x K]^T   (A and B row-major with K contiguous),
// FP32 accumulation in tensor memory (TMEM), with a fused epilogue.
//
// One CTA of 128 threads (4 warps) computes a 128 x 128 tile of C, walking K
// in blocks of 64 through a ring of kStages shared-memory stages:
//   * lane 0 of warp 0 is the producer: per block it waits until the MMAs
//     have released the stage, announces 32 KB on the stage's "full"
//     mbarrier and issues two TMA tile loads (cp.async.bulk.tensor.2d) of the
//     128 x 64 A and B boxes, which land 128-byte swizzled (the K-major
//     SWIZZLE_128B layout of the MMA: 8-row x 128-byte atoms, 1024 bytes
//     apart along M / N); rows past M / N and columns past K arrive as zeros;
//   * lane 0 of warp 1 issues the four 128 x 128 x 16 MMAs of a block once its
//     stage is full and commits them to the stage's "empty" mbarrier, and
//     after the last block to a "done" mbarrier;
//   * then warp w reads TMEM lanes 32w .. 32w + 31 (rows of C) with
//     tcgen05.ld into shared memory, and the threads write the tile back
//     column by column (coalesced rows) through the epilogue.
// Every mbarrier wait is bounded: on expiry the kernel records an error,
// stops issuing, waits (bounded) for the loads and MMAs it has in flight and
// still frees its TMEM.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pdcs {
namespace tc {

constexpr int kTileM = 128, kTileN = 128, kTileK = 64, kThreads = 128;
constexpr int kStages = 4;
constexpr int kStageBytes = kTileM * kTileK * 2;  // 16 KB per operand per stage
constexpr uint32_t kSBO = 1024;                    // 8 rows x 128 B: one swizzle atom
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

// Shared-memory matrix descriptor (tcgen05) of a K-major operand in the
// 128-byte swizzle layout: start address >> 4 in bits 0-13, leading byte
// offset >> 4 in 16-29 (unused for this layout: one 16-element K step stays
// inside a 128-byte row; set to 16 bytes), stride byte offset >> 4 in 32-45
// (1024: the next 8-row atom), descriptor version 1 in bits 46-47, base
// offset 0 (atoms 1024-byte aligned), swizzle mode 2 (128-byte) in bits 61-63.
// The K step j of a 64-wide block starts 32 j bytes into the atom; the swizzle
// is applied from the address bits, so the start address simply advances.
__host__ __device__ inline uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)((kSBO & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
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

// Tensor map of a row-major rows x K BF16 matrix (leading dimension ld
// elements) for 64 x 128 (K x rows) boxes with the 128-byte swizzle; zeros
// outside the matrix.  Needs base 16-byte aligned and ld a multiple of 8.
// Returns false if the driver refuses the map.
inline bool make_kmajor_map(CUtensorMap* map, const void* base, int64_t rows, int64_t K,
                            int64_t ld) {
  typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                               const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                               const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                               CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn encode = nullptr;
  if (encode == nullptr) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || fn == nullptr)
      return false;
    encode = reinterpret_cast<EncodeFn>(fn);
  }
  if (((uintptr_t)base & 15u) != 0 || (ld & 7) != 0 || rows <= 0 || K <= 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kTileK, (cuuint32_t)kTileM};
  const cuuint32_t estr[2] = {1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
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

// Announce the bytes the stage's loads will deliver (counts as the one arrival).
__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// TMA load of the box at (x = k, y = row) of the map into dst, completing on bar.
__device__ inline void tma_load_2d(void* dst, const CUtensorMap* map, int32_t x, int32_t y,
                                   uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
#endif

// C = A * B^T with the epilogue; A: M x K, B: N x K, given as tensor maps
// (make_kmajor_map).  Grid: (ceil(N / 128), ceil(M / 128), splits).  Split-K
// (kchunk > 0, a multiple of 64): CTA z multiplies the K slice
// [z kchunk, (z + 1) kchunk) and writes its FP32 partial tile (EPI_F32) at
// ep.out + z * zstride floats; k_splitk_reduce adds the slices.
// err: set to 1 if an mbarrier wait expired (the tile is then not written).
// nst (1 .. kStages): stages in the ring; dynamic shared memory gemm_smem(nst).
__global__ void __launch_bounds__(kThreads) k_gemm_bf16_tn(const __grid_constant__ CUtensorMap tmA,
                                                           const __grid_constant__ CUtensorMap tmB,
                                                           int64_t M, int64_t N, int64_t K,
                                                           EpiArgs ep, int* err, int64_t kchunk,
                                                           int64_t zstride, int nst) {
#ifdef __CUDA_ARCH__
  int64_t kbeg = 0;
  if (kchunk > 0) {
    kbeg = (int64_t)blockIdx.z * kchunk;
    K = K - kbeg < kchunk ? K - kbeg : kchunk;
    ep.out = reinterpret_cast<float*>(ep.out) + (int64_t)blockIdx.z * zstride;
  }
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte aligned stages (swizzle atoms): A0 B0 A1 B1 ...
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
  __shared__ uint32_t tmem_base;
  __shared__ int failed, n_loads, n_mma;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t m0 = (int64_t)blockIdx.y * kTileM, n0 = (int64_t)blockIdx.x * kTileN;
  const int nk = (int)((K + kTileK - 1) / kTileK);
  if (t == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    failed = 0;
    n_loads = 0;
    n_mma = 0;
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
  volatile int* vfailed = &failed;
  if (warp == 0 && lane == 0) {
    // producer
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % nst;
      if (kb >= nst && !mbar_wait(&empty[s], (uint32_t)(((kb / nst) - 1) & 1))) {
        *vfailed = 1;
        break;
      }
      if (*vfailed) break;
      uint8_t* sa = base + (size_t)s * 2 * kStageBytes;
      mbar_expect_tx(&full[s], 2 * kStageBytes);
      const int32_t kx = (int32_t)(kbeg + (int64_t)kb * kTileK);
      tma_load_2d(sa, &tmA, kx, (int32_t)m0, &full[s]);
      tma_load_2d(sa + kStageBytes, &tmB, kx, (int32_t)n0, &full[s]);
      ++issued;
    }
    n_loads = issued;
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = instr_desc_bf16(kTileM, kTileN);
    int used = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % nst;
      if (!mbar_wait(&full[s], (uint32_t)((kb / nst) & 1))) {
        *vfailed = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a0 = smem_u32(base + (size_t)s * 2 * kStageBytes), b0 = a0 + kStageBytes;
#pragma unroll
      for (int j = 0; j < kTileK / 16; ++j)
        tc_mma(tmem, smem_desc_sw128(a0 + 32 * j), smem_desc_sw128(b0 + 32 * j), idesc,
               (kb > 0 || j > 0) ? 1u : 0u);
      tc_commit(&empty[s]);
      ++used;
    }
    tc_commit(&done);  // tracks every MMA this thread issued
    n_mma = used;
  }
  __syncthreads();
  // ReLU-mask epilogue: while the last MMAs run, thread (warp w, lane l)
  // turns the mask of its row 32 w + l into 128 keep bits
  const int rl = warp * 32 + lane;
  uint32_t keep[4] = {0u, 0u, 0u, 0u};
  if (ep.kind == EPI_BF16_RELU_MASK && m0 + rl < M) {
    const __nv_bfloat16* mp = ep.mask + (m0 + rl) * ep.ldm + n0;
    if (n0 + kTileN <= N && ((uintptr_t)mp & 15u) == 0) {
      uint4 q[kTileN / 8];
#pragma unroll
      for (int j = 0; j < kTileN / 8; ++j) q[j] = __ldg(reinterpret_cast<const uint4*>(mp) + j);
#pragma unroll
      for (int j = 0; j < kTileN / 8; ++j) {
        const uint32_t w[4] = {q[j].x, q[j].y, q[j].z, q[j].w};
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const uint16_t b = (uint16_t)(w[e >> 1] >> (16 * (e & 1)));
          if (__bfloat162float(__ushort_as_bfloat16(b)) > 0.0f) keep[(8 * j + e) >> 5] |= 1u << ((8 * j + e) & 31);
        }
      }
    } else {
#pragma unroll
      for (int w = 0; w < 4; ++w)
        for (int j = 0; j < 32 && n0 + 32 * w + j < N; ++j)
          if (__bfloat162float(mp[32 * w + j]) > 0.0f) keep[w] |= 1u << j;
    }
  }
  // the accumulator is complete once "done" fires; a failed run still waits
  // for the MMAs and loads it has in flight before the memory is released
  if (t == 0) {
    if (!mbar_wait(&done, 0u)) failed = 1;
    for (int kb = n_mma; kb < n_loads; ++kb)
      if (!mbar_wait(&full[kb % nst], (uint32_t)((kb / nst) & 1))) failed = 1;
  }
  __syncthreads();
  tc_fence_after();
  if (!failed && n_mma == nk && nk > 0) {
    // the accumulator goes through shared memory (the stages are free now):
    // thread (warp w, lane l) holds row 32 w + l; rows are stored 129 floats
    // apart so the column-wise writes hit distinct banks, then each thread
    // takes one column and walks the rows, so a warp stores 32 consecutive
    // columns of a row per step (coalesced)
    float* stage = reinterpret_cast<float*>(base);
    constexpr int kLd = kTileN + 1;
    fence_proxy_async_smem();  // the stages were last touched by the async proxy
    const bool masked = ep.kind == EPI_BF16_RELU_MASK;
#pragma unroll
    for (int c0 = 0; c0 < kTileN; c0 += 16) {
      float v[16];
      tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int cc = c0 + i;
        stage[rl * kLd + cc] = (masked && !((keep[cc >> 5] >> (cc & 31)) & 1u)) ? 0.0f : v[i];
      }
    }
    __syncthreads();
    const int64_t c = n0 + t;
    if (c < N) {
      const float bc = (ep.kind == EPI_F32_BIAS || ep.kind == EPI_BF16_BIAS_RELU) ? ep.bias[c] : 0.0f;
      const int rmax = (int)(M - m0 < kTileM ? M - m0 : kTileM);
      // eight rows at a time: their shared-memory loads before the stores
      for (int r0 = 0; r0 < rmax; r0 += 8) {
        float x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = r0 + i < rmax ? stage[(r0 + i) * kLd + t] + bc : 0.0f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (r0 + i >= rmax) break;
          const int64_t gr = m0 + r0 + i;
          if (ep.kind == EPI_F32 || ep.kind == EPI_F32_BIAS) {
            reinterpret_cast<float*>(ep.out)[gr * ep.ldc + c] = x[i];
          } else {
            const float y = ep.kind == EPI_BF16_BIAS_RELU ? fmaxf(x[i], 0.0f) : x[i];
            reinterpret_cast<__nv_bfloat16*>(ep.out)[gr * ep.ldc + c] = __float2bfloat16(y);
          }
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

// Dynamic shared memory of k_gemm_bf16_tn with nst stages: the ring of A and
// B stages or the epilogue's 128 x 129 FP32 staging tile, whichever is
// larger, plus the 1024-byte alignment slack.
constexpr int gemm_smem(int nst) {
  return (2 * nst * kStageBytes > kTileM * (kTileN + 1) * 4 ? 2 * nst * kStageBytes
                                                            : kTileM * (kTileN + 1) * 4) +
         1024;
}
constexpr int kGemmSmem = gemm_smem(kStages);

}  // namespace tc
}  // namespace pdcs
