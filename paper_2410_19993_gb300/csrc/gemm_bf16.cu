// gemm_bf16.cu -- BF16 x BF16 -> FP32 products on the tensor cores (tcgen05 kind::f16), the
// building block of the surrogate's training and inference kernels.
//
//   C[m][n] = sum_k A(m, k) B(n, k),   A(m, k) = A[m*sAm + k*sAk],   B(n, k) = B[n*sBn + k*sBk]
//
// Operands are staged into shared memory by the threads of the block (16-byte loads along
// whichever index is contiguous), so forward products (X W^T), input gradients (dZ W) and weight
// gradients (dZ^T X, split over K with atomic accumulation) use one kernel.  Tiles: 128 rows x
// 128 columns per block, K in chunks of 64 (four K=16 MMAs), double-buffered; the accumulator
// lives in 128 columns of tensor memory.  Shapes must be multiples of the tiles (the callers pad):
// M % 128 == 0, N % 128 == 0, K % 64 == 0.
//
// Epilogues: EPI_STORE (FP32 C, or atomic add for split-K), EPI_BIAS_RELU (H = relu(C + bias) as
// BF16), EPI_MASK (D = C where mask > 0 else 0, as BF16: the ReLU derivative applied to a
// back-propagated gradient).
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "kernels.h"
#include "umma.cuh"

namespace xbar {

namespace g16 {

constexpr int kBM = 128, kBN = 128, kBK = 64, kThreads = 128;
constexpr uint32_t kTileBytes = kBM * kBK * 2;  // one operand tile (A or B) of a K chunk: 16 KB
constexpr uint32_t kLBO = (kBM / 8) * 128;        // K-direction stride between core matrices (2 KB)

// byte offset of element (row, k) of a [128 x 64] BF16 tile in the no-swizzle K-major core-matrix
// layout: core matrix (row/8, k/8) of 8 rows x 16 bytes, K-direction stride kLBO, row-group 128 B
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
  return (uint32_t)(k >> 3) * kLBO + (uint32_t)(row >> 3) * 128 + (uint32_t)(row & 7) * 16 + (uint32_t)(k & 7) * 2;
}

// Staging a [128 rows x 64 k] tile into the core-matrix layout.  A 16-byte store holds 8 k values
// of one row; its bank group is set by the row (r & 7), so a warp's stores are conflict-free when
// its 32 threads store 32 consecutive rows at one k group.  Each thread issues all of its loads
// before its shared-memory stores, so one chunk costs one memory latency.
static_assert(kThreads == kBM, "one thread per tile row");
constexpr int kKG = kBK / 8;  // k groups of 8 per chunk

// rotate the 8 entries of v left by rot (0..7) without dynamic register indexing
__device__ __forceinline__ void rotate8(uint4 (&v)[8], int rot) {
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int sh = 1 << b;
    if (rot & sh) {
      uint4 t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = v[(u + sh) & 7];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = t[u];
    }
  }
}

// op(r, k) = P[(r0 + r)*sR + (k0 + k)*sK]
__device__ __forceinline__ void stage(unsigned char* dst, const __nv_bfloat16* P, long sR, long sK, long r0,
                                      long k0, int tid) {
  uint4 v[8];
  if (sK == 1) {  // k contiguous: thread = row, eight 16-byte loads along its row
    const __nv_bfloat16* src = P + (r0 + tid) * sR + k0;
#pragma unroll
    for (int g = 0; g < kKG; ++g) v[g] = *reinterpret_cast<const uint4*>(src + g * 8);
#pragma unroll
    for (int g = 0; g < kKG; ++g) *reinterpret_cast<uint4*>(dst + tile_off(tid, g * 8)) = v[g];
  } else {        // rows contiguous (sR == 1): thread = 8 rows x 8 k block, transposed in registers
    const int rg = tid & 15, kg = tid >> 4;  // row group (16) x k group (8) = 128 blocks
    const __nv_bfloat16* src = P + (r0 + rg * 8) + (k0 + kg * 8) * sK;
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = *reinterpret_cast<const uint4*>(src + e * sK);  // 8 rows at k = e
    uint4 o[8];
    const __nv_bfloat16* in = reinterpret_cast<const __nv_bfloat16*>(v);
    __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(o);
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int e = 0; e < 8; ++e) out[u * 8 + e] = in[e * 8 + u];
    // store row (s + rg) & 7 at step s: a warp's 32 stores then cover all eight bank groups
    rotate8(o, rg & 7);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int u = (s + rg) & 7;
      *reinterpret_cast<uint4*>(dst + tile_off(rg * 8 + u, kg * 8)) = o[s];
    }
  }
}

}  // namespace g16

__global__ void __launch_bounds__(g16::kThreads, 1) gemm_bf16_kernel(GemmBf16Params p) {
  using namespace g16;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint64_t wlim = wait_limit(p.status);  // read once: the waits below sit on critical paths
  const long m0 = (long)blockIdx.x * kBM, n0 = (long)blockIdx.y * kBN;
  const int nks = p.K / kBK;                                  // K chunks of the whole product
  const int per = (nks + (int)gridDim.z - 1) / (int)gridDim.z;  // chunks of this split
  const int kc0 = (int)blockIdx.z * per, kc1 = min(nks, kc0 + per);

  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm);  // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 16);
  unsigned char* tiles = sm + 1024;                  // [2 buffers][A tile | B tile]

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"((uint32_t)kBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tslot;
  const uint32_t idesc = umma::idesc_bf16(kBM, kBN);
  bool ok = true;

  for (int kc = kc0; kc < kc1 && ok; ++kc) {
    const int it = kc - kc0, buf = it & 1;
    unsigned char* At = tiles + (size_t)buf * 2 * kTileBytes;
    unsigned char* Bt = At + kTileBytes;
    if (it >= 2)  // the MMAs that read this buffer two chunks ago are complete
      ok = mbar_spin_bounded(&bar[buf], (unsigned)(((it - 2) >> 1) & 1), p.status, wlim, 20);
    if (__syncthreads_or(!ok)) break;
    stage(At, p.A, p.sAm, p.sAk, m0, (long)kc * kBK, tid);
    stage(Bt, p.B, p.sBn, p.sBk, n0, (long)kc * kBK, tid);
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t ad = umma::sdesc(smem_addr(At), kLBO, 128), bd = umma::sdesc(smem_addr(Bt), kLBO, 128);
#pragma unroll
      for (int s = 0; s < kBK / 16; ++s)  // K = 16 per MMA: two 8-element core-matrix columns
        umma::mma_bf16(tbase, ad + (uint64_t)((2 * s * kLBO) >> 4), bd + (uint64_t)((2 * s * kLBO) >> 4), idesc,
                 (it > 0 || s > 0) ? 1u : 0u);
      umma::commit(&bar[buf]);
    }
  }
  if (ok && kc1 > kc0) {
    const int last = kc1 - kc0 - 1;
    ok = mbar_spin_bounded(&bar[last & 1], (unsigned)((last >> 1) & 1), p.status, wlim, 20);
  }
  ok = !__syncthreads_or(!ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // ---- epilogue: warp w owns accumulator rows 32w .. 32w+31 -----------------------------------
  if (ok && kc1 > kc0) {
    const long row = m0 + warp * 32 + lane;
    for (int cb = 0; cb < kBN; cb += 32) {
      float a[32];
      umma::ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, a);
      const long col = n0 + cb;
      if (p.mode == GEMM_EPI_STORE) {
        float* c = p.C + row * p.ldc + col;
        if (p.atomic) {
          for (int q = 0; q < 32; ++q) atomicAdd(c + q, a[q]);
        } else {
          for (int q = 0; q < 32; q += 4) *reinterpret_cast<float4*>(c + q) = make_float4(a[q], a[q + 1], a[q + 2], a[q + 3]);
        }
      } else {
        __nv_bfloat16* o = p.out + row * p.ldo + col;
        alignas(16) __nv_bfloat16 v[32];
        if (p.mode == GEMM_EPI_BIAS_RELU) {
          for (int q = 0; q < 32; ++q) v[q] = __float2bfloat16_rn(fmaxf(a[q] + p.bias[col + q], 0.0f));
        } else {  // GEMM_EPI_MASK
          const __nv_bfloat16* mk = p.mask + row * p.ldm + col;
          for (int q = 0; q < 32; ++q) v[q] = __float2bfloat16_rn(__bfloat162float(mk[q]) > 0.0f ? a[q] : 0.0f);
        }
        for (int q = 0; q < 32; q += 8) *reinterpret_cast<uint4*>(o + q) = *reinterpret_cast<const uint4*>(v + q);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"((uint32_t)g16::kBN)
                 : "memory");
}

cudaError_t launch_gemm_bf16(const GemmBf16Params& p, int ksplit, cudaStream_t st) {
  if (p.M % g16::kBM || p.N % g16::kBN || p.K % g16::kBK || p.M <= 0 || p.N <= 0 || p.K <= 0)
    return cudaErrorInvalidValue;
  if (!(p.sAk == 1 || p.sAm == 1)) return cudaErrorInvalidValue;
  if (!(p.sBk == 1 || p.sBn == 1)) return cudaErrorInvalidValue;
  // 16-byte staging loads: the non-unit stride of each loaded operand is a multiple of 8 elements
  if ((p.sAk == 1 ? p.sAm : p.sAk) % 8) return cudaErrorInvalidValue;
  if ((p.sBk == 1 ? p.sBn : p.sBk) % 8) return cudaErrorInvalidValue;
  const int nks = p.K / g16::kBK;
  if (ksplit < 1) ksplit = 1;
  if (ksplit > nks) ksplit = nks;
  const size_t smem = 1024 + 4 * (size_t)g16::kTileBytes;
  cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(p.M / g16::kBM, p.N / g16::kBN, ksplit);
  gemm_bf16_kernel<<<grid, g16::kThreads, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace xbar
