// surrogate_infer.cu -- the surrogate's second and output layers for prediction, with the result
// formed in the same kernel.
//
// Row r = b*N + j (vector b, bit line j).  With the first layer split into a per-column part P_j
// and a per-vector part Q_b (surrogate.cu), the rest of the network for row r is
//   h1 = bf16(relu(P_j + Q_b + b1)),  h2 = bf16(relu(W2 h1 + b2)),  n = W3 h2 + b3,
// and the prediction I = I_line + I_ideal (mu + sigma n0) with the relative error estimate
// c sigma exp(n1) |I_ideal| / |I|; flag[b] = 1 when an estimate of vector b is above the bound.
//
// Persistent blocks (one per SM, 512 threads: four per tile row, each owning a quarter of the
// 256 hidden columns): W2 (256 x 256 BF16, 128 KB), pre-tiled in global
// memory in the B operand's layout whenever the weights change, is copied once into shared memory.  A tile is 128 rows = 8 vectors x 16 bit lines, so its operand
// h1 needs only 16 rows of P and 8 rows of Q (24 KB): they are copied into shared memory with
// cp.async while the previous tile's epilogue runs, and the threads build h1 (64 KB) from them
// (thread = row, a warp's 16-byte stores cover 32 consecutive rows: bank-conflict free).  One
// thread issues 16 MMAs (M = 128, N = 256, K = 16) into one of two 256-column tensor-memory
// accumulators; while the tensor core works on tile t, the threads drain tile t-1's accumulator
// (tcgen05.ld), apply b2, ReLU and the BF16 rounding of h2, reduce against W3 (four partial sums
// per row, combined through shared memory) and write the prediction.  Every wait is bounded; on expiry the block records XBAR_DEV_TIMEOUT, waits
// (bounded) for its own MMAs and frees its tensor memory.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "umma.cuh"

namespace xbar {

namespace si {

constexpr int kH = 256;         // hidden width (K and N of the product)
constexpr int kRows = 128;      // rows per tile (MMA M)
constexpr int kThreads = 512;   // tile row m = tid % 128, hidden-column quarter tid / 128
constexpr uint32_t kLA = (kRows / 8) * 128;  // A: K-direction stride between core matrices (2 KB)
constexpr uint32_t kLB = (kH / 8) * 128;     // B: same for 256 rows (4 KB)
constexpr uint32_t kBBytes = (kH / 8) * kLB;    // 128 KB
constexpr uint32_t kABytes = (kH / 8) * kLA;    // 64 KB
constexpr int kTJ = 16, kTB = kRows / kTJ;      // a tile: kTB vectors x kTJ bit lines
constexpr int kPPitch = kH + 4;                 // P rows in shared memory (bank offset 4 per row)
constexpr size_t kPBytes = (size_t)kTJ * kPPitch * 4, kQBytes = (size_t)kTB * kH * 4;
constexpr size_t kRedBytes = (size_t)4 * kRows * 2 * 4;  // partial W3 sums [quarter][row][2]
constexpr size_t kSmem = 1024 + kBBytes + kABytes + (size_t)(2 * kH + 2 * kH) * 4 + kPBytes + kQBytes + kRedBytes;
static_assert(kSmem <= 232448, "shared memory");

__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ uint32_t a_off(int m, int g) { return (uint32_t)g * kLA + (uint32_t)(m >> 3) * 128 + (uint32_t)(m & 7) * 16; }
__device__ __forceinline__ uint32_t b_off(int n, int g) { return (uint32_t)g * kLB + (uint32_t)(n >> 3) * 128 + (uint32_t)(n & 7) * 16; }

}  // namespace si

__global__ void __launch_bounds__(si::kThreads, 1) surrogate_infer_kernel(SurInferParams p) {
  using namespace si;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m = tid & (kRows - 1), cq = tid >> 7;  // tile row; quarter of the hidden columns
  const uint64_t wlim = wait_limit(p.status);  // read once: the waits below sit on critical paths
  const long Bv = p.rows / p.N;  // input vectors
  const long njt = (p.N + kTJ - 1) / kTJ, ntiles = ((Bv + kTB - 1) / kTB) * njt;

  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm);  // [2]: MMA of the tile in accumulator 0 / 1
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 16);
  unsigned char* Bs = sm + 1024;
  unsigned char* As = Bs + kBBytes;
  float* b1s = reinterpret_cast<float*>(As + kABytes);
  float* b2s = b1s + kH;
  float* w3s = b2s + kH;  // [2][kH]
  float* Ps = w3s + 2 * kH;          // [kTJ][kPPitch] rows of P of the tile's bit lines
  float* Qs = Ps + kTJ * kPPitch;    // [kTB][kH] rows of Q of the tile's vectors
  float2* red = reinterpret_cast<float2*>(Qs + kTB * kH);  // [4][kRows] partial (s0, s1)
  // rows of P and Q of tile t into Ps, Qs (16-byte cp.async, zero fill past N or B)
  auto stage_rows = [&](long t) {
    const long b0 = (t / njt) * kTB, j0 = (t % njt) * kTJ;
#pragma unroll
    for (int u = 0; u < kTJ * (kH / 4) / kThreads; ++u) {
      const int id = tid + kThreads * u, rr = id / (kH / 4), c = id % (kH / 4);
      const long j = j0 + rr;
      cp_async16(Ps + rr * kPPitch + 4 * c, p.P + (j < p.N ? j : 0) * kH + 4 * c, j < p.N ? 16u : 0u);
    }
#pragma unroll
    for (int u = 0; u < kTB * (kH / 4) / kThreads; ++u) {
      const int id = tid + kThreads * u, qq = id / (kH / 4), c = id % (kH / 4);
      const long b = b0 + qq;
      cp_async16(Qs + qq * kH + 4 * c, p.Q + (b < Bv ? b : 0) * kH + 4 * c, b < Bv ? 16u : 0u);
    }
    cp_async_commit();
  };

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  if (warp == 0) umma::alloc(tslot, 2 * kH);
  // W2, already in the B layout (launch_surrogate_w2_tile): 16-byte copies, all in flight at once
  for (uint32_t x = tid; x < kBBytes / 16; x += kThreads)
    cp_async16(Bs + 16 * x, reinterpret_cast<const unsigned char*>(p.W2) + 16 * x, 16u);
  cp_async_commit();
  for (int k = tid; k < kH; k += kThreads) {
    b1s[k] = p.b1[k];
    b2s[k] = p.b2[k];
    w3s[k] = p.W3[k];
    w3s[kH + k] = p.W3[kH + k];
  }
  cp_async_wait_all();
  fence_proxy_async_smem();
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t idesc = umma::idesc_bf16(kRows, kH);
  const uint64_t adesc = umma::sdesc(smem_addr(As), kLA, 128), bdesc = umma::sdesc(smem_addr(Bs), kLB, 128);

  bool ok = true;
  int issued = 0;  // tiles whose MMAs this block committed
  long prev = -1;
  // drain accumulator `buf` (tile t): b2, ReLU, BF16 rounding, W3, prediction
  // (every thread takes part: the quarters' partial sums meet in shared memory)
  auto epilogue = [&](long t, int buf) {
    const long b = (t / njt) * kTB + (m >> 4), j = (t % njt) * kTJ + (m & 15);
    const bool real = b < Bv && j < p.N;
    const long r = b * p.N + j;
    // the row's ideal and line-model currents, loaded before the accumulator reads so that their
    // latency overlaps them
    double ii = 0.0, il = 0.0;
    if (cq == 0 && real) {
      ii = p.Iid[r];
      il = p.Iln[r];
    }
    float s0 = 0.0f, s1 = 0.0f;
#pragma unroll 1
    for (int cb = 64 * cq; cb < 64 * cq + 64; cb += 32) {
      float a[32];
      // warp w reads tensor-memory lanes 32 (w % 4) ..: rows m of this thread
      umma::ld32(tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(buf * kH + cb), a);
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const float h = __bfloat162float(__float2bfloat16_rn(fmaxf(a[q] + b2s[cb + q], 0.0f)));
        s0 = fmaf(w3s[cb + q], h, s0);
        s1 = fmaf(w3s[kH + cb + q], h, s1);
      }
    }
    red[cq * kRows + m] = make_float2(s0, s1);
    __syncthreads();
    if (cq == 0) {
#pragma unroll
      for (int u = 1; u < 4; ++u) {
        const float2 v = red[u * kRows + m];
        s0 += v.x;
        s1 += v.y;
      }
    }
    if (cq == 0 && real) {
      const float n0 = s0 + p.b3[0], n1 = s1 + p.b3[1];
      const double Ir = il + ii * (p.mu + p.sigma * (double)n0);
      const double e = p.cal * p.sigma * (double)expf(n1) * fabs(ii) / fmax(fabs(Ir), 1e-300);
      p.I[r] = Ir;
      if (p.est) p.est[r] = e;
      if (p.flag && !(e <= p.bound)) p.flag[b] = 1;
    }
  };

  if (blockIdx.x < ntiles) stage_rows(blockIdx.x);
  for (long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    const int buf = issued & 1;
    // the previous tile's MMAs read the operand buffer: wait for them before regenerating it
    if (issued >= 1 && tid == 0)
      ok = mbar_spin_bounded(&bar[(issued - 1) & 1], (unsigned)(((issued - 1) >> 1) & 1), p.status,
                             wlim, 20);
    cp_async_wait_all();  // this thread's copies of tile t's rows; the barrier shows everyone's
    if (__syncthreads_or(!ok)) break;
    umma::fence_after();
    {  // operand of tile t: row m = (vector m / 16, bit line m % 16), core-matrix columns of this
       // thread's quarter, from the staged rows
      const long b = (t / njt) * kTB + (m >> 4), j = (t % njt) * kTJ + (m & 15);
      const bool real = b < Bv && j < p.N;
      const float4* P4 = reinterpret_cast<const float4*>(Ps + (m & 15) * kPPitch);
      const float4* Q4 = reinterpret_cast<const float4*>(Qs + (m >> 4) * kH);
      const float4* C4 = reinterpret_cast<const float4*>(b1s);
#pragma unroll
      for (int g0 = 8 * cq; g0 < 8 * cq + 8; g0 += 4) {
        float4 pa[8], qa[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          pa[u] = P4[2 * g0 + u];
          qa[u] = Q4[2 * g0 + u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int g = g0 + u;
          const float4 a0 = pa[2 * u], a1 = pa[2 * u + 1], e0 = qa[2 * u], e1 = qa[2 * u + 1];
          const float4 c0 = C4[2 * g], c1 = C4[2 * g + 1];
          const float z[8] = {a0.x + e0.x + c0.x, a0.y + e0.y + c0.y, a0.z + e0.z + c0.z, a0.w + e0.w + c0.w,
                              a1.x + e1.x + c1.x, a1.y + e1.y + c1.y, a1.z + e1.z + c1.z, a1.w + e1.w + c1.w};
          alignas(16) __nv_bfloat16 v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = __float2bfloat16_rn(real ? fmaxf(z[e], 0.0f) : 0.0f);
          *reinterpret_cast<uint4*>(As + a_off(m, g)) = *reinterpret_cast<const uint4*>(v);
        }
      }
    }
    fence_proxy_async_smem();
    umma::fence_before();
    __syncthreads();  // operand written; the previous epilogue's TMEM reads are done
    if (tid == 0) {
      umma::fence_after();
#pragma unroll
      for (int s = 0; s < kH / 16; ++s)  // K = 16 per MMA: two core-matrix columns
        umma::mma_bf16(tbase + (uint32_t)(buf * kH), adesc + (uint64_t)((2 * s * kLA) >> 4),
                       bdesc + (uint64_t)((2 * s * kLB) >> 4), idesc, s > 0 ? 1u : 0u);
      umma::commit(&bar[buf]);
    }
    ++issued;
    // the next tile's rows: Ps and Qs were last read before the barrier above
    if (t + gridDim.x < ntiles) stage_rows(t + gridDim.x);
    if (prev >= 0) epilogue(prev, (issued - 2) & 1);  // overlaps the MMAs just issued
    umma::fence_before();
    prev = t;
  }
  if (ok && prev >= 0) {
    if (tid == 0)
      ok = mbar_spin_bounded(&bar[(issued - 1) & 1], (unsigned)(((issued - 1) >> 1) & 1), p.status,
                             wlim, 20);
    ok = !__syncthreads_or(!ok);
    umma::fence_after();
    if (ok) epilogue(prev, (issued - 1) & 1);
  }
  cp_async_wait_all();  // no copy may still be in flight when the block exits
  if (!ok && issued >= 1 && tid == 0)  // the last commit covers every MMA of this block (bounded wait)
    mbar_spin_bounded(&bar[(issued - 1) & 1], (unsigned)(((issued - 1) >> 1) & 1), p.status, wlim, 20);
  umma::fence_before();
  __syncthreads();
  if (warp == 0) umma::dealloc(tbase, 2 * kH);
}

// W2 (row n = output unit, column k = input unit, BF16 [256][256]) -> the kernel's B-operand layout
// (core matrices of 8 rows x 16 bytes, K-direction stride kLB): 16 bytes per thread
__global__ void surrogate_w2_tile_kernel(const __nv_bfloat16* __restrict__ W2, unsigned char* __restrict__ W2t) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;  // (n, g): 8 consecutive k of row n
  if (x >= si::kH * (si::kH / 8)) return;
  const int n = x / (si::kH / 8), g = x % (si::kH / 8);
  *reinterpret_cast<uint4*>(W2t + si::b_off(n, g)) = reinterpret_cast<const uint4*>(W2 + (size_t)n * si::kH)[g];
}

cudaError_t launch_surrogate_w2_tile(const __nv_bfloat16* W2, void* W2t, cudaStream_t st) {
  const int n = si::kH * (si::kH / 8);
  surrogate_w2_tile_kernel<<<(n + 255) / 256, 256, 0, st>>>(W2, static_cast<unsigned char*>(W2t));
  return cudaGetLastError();
}

cudaError_t launch_surrogate_infer(const SurInferParams& p, int nsm, cudaStream_t st) {
  if (p.rows <= 0) return cudaSuccess;
  if (p.N < 1 || !p.P || !p.Q || !p.W2 || !p.I) return cudaErrorInvalidValue;
  const long ntiles = ((p.rows / p.N + si::kTB - 1) / si::kTB) * ((p.N + si::kTJ - 1) / si::kTJ);
  const int grid = (int)std::min<long>(ntiles, nsm > 0 ? nsm : 1);
  cudaError_t e = cudaFuncSetAttribute(surrogate_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)si::kSmem);
  if (e != cudaSuccess) return e;
  surrogate_infer_kernel<<<grid, si::kThreads, si::kSmem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace xbar
