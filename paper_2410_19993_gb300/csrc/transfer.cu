// transfer.cu -- currents-only transfer-matrix mode: the unit-input right-hand sides that give
// G_eff, and the FP64 product I = V G_eff.
//
// The nodal system (Sec. II, Eqs. 1-7) is linear in the source voltages, so the bit-line currents of
// any input vector are I = V G_eff with G_eff[i][j] = dI_j / dV_i, the current of bit line j for a
// unit voltage on word line i alone.  G_eff (M x N) comes from M unit-input solves of the current
// factorization (the handle's own solve, so its accuracy is the solve's certified per-current
// accuracy); every further input vector then costs one row of an FP64 matrix product, 2MN flops,
// instead of a sweep through all 2N - 1 column blocks.  For non-negative inputs every term V_i G_eff
// [i][j] is non-negative (A^-1 > 0 entrywise), so the relative error of each current is at most that
// of the G_eff entries plus the FP64 rounding of an M-term sum.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace xbar {

namespace {

// 32 x 64 output tiles, 2 x 4 per thread: the FP64 pipe (2 DFMA per SM and cycle on this part)
// bounds the product, so the tile is sized for balance rather than reuse -- at 256 x 256 with 8192
// vectors 1024 tiles give the busiest SM 7 against an average of 6.7 (64 x 64 tiles: 4 against
// 3.4, a 16% tail)
constexpr int kTileR = 32;   // output rows (input vectors) per block
constexpr int kTileC = 64;   // output columns (bit lines) per block
constexpr int kKStep = 16;   // K per shared-memory stage
constexpr int kGemmThreads = 256;

__global__ void eye_kernel(double* E, int M) {
  const size_t n = (size_t)M * M;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    E[t] = (t / M == t % M) ? 1.0 : 0.0;
}

// C[R x N] = A[R x K] . Bm[K x N], FP64, all row-major.  One kTileR x kTileC tile of C per block,
// 2 x 4 per thread, K in steps of 16 through shared memory; each output is one FMA chain over k in
// order.
__global__ void __launch_bounds__(kGemmThreads) gemm_f64_kernel(const double* __restrict__ A,
                                                                const double* __restrict__ Bm, double* __restrict__ C,
                                                                int R, int K, int N) {
  constexpr int PR = kTileR * kTileC / kGemmThreads / 4;  // rows per thread (2)
  __shared__ double As[kKStep][kTileR + 1];  // As[k][row]
  __shared__ double Bs[kKStep][kTileC + 1];  // Bs[k][col]
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  const int r0 = blockIdx.y * kTileR, c0 = blockIdx.x * kTileC;
  double acc[PR][4];
#pragma unroll
  for (int a = 0; a < PR; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k0 = 0; k0 < K; k0 += kKStep) {
#pragma unroll
    for (int u = 0; u < kTileR * kKStep / kGemmThreads; ++u) {  // A: 16 consecutive k of one row per 16 threads
      const int idx = t + u * kGemmThreads;
      const int ar = idx / kKStep, ak = idx % kKStep;
      const int r = r0 + ar, k = k0 + ak;
      As[ak][ar] = (r < R && k < K) ? A[(size_t)r * K + k] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kTileC * kKStep / kGemmThreads; ++u) {  // Bm: 64 consecutive columns of one k
      const int idx = t + u * kGemmThreads;
      const int bk = idx / kTileC, bc = idx % kTileC;
      const int kb = k0 + bk, c = c0 + bc;
      Bs[bk][bc] = (kb < K && c < N) ? Bm[(size_t)kb * N + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kKStep; ++kk) {
      double a[PR], b[4];
#pragma unroll
      for (int q = 0; q < PR; ++q) a[q] = As[kk][ty * PR + q];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Bs[kk][tx * 4 + q];
#pragma unroll
      for (int p = 0; p < PR; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < PR; ++p) {
    const int r = r0 + ty * PR + p;
    if (r >= R) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + tx * 4 + q;
      if (c < N) C[(size_t)r * N + c] = acc[p][q];
    }
  }
}

}  // namespace

cudaError_t launch_eye(double* E, int M, cudaStream_t st) {
  if (M <= 0) return cudaSuccess;
  const size_t n = (size_t)M * M;
  const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 4096);
  eye_kernel<<<blocks, 256, 0, st>>>(E, M);
  return cudaGetLastError();
}

cudaError_t launch_gemm_f64(const double* A, const double* Bm, double* C, int R, int K, int N, cudaStream_t st) {
  if (R <= 0 || N <= 0) return cudaSuccess;
  if (K <= 0 || !A || !Bm || !C) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((N + kTileC - 1) / kTileC), (unsigned)((R + kTileR - 1) / kTileR));
  if (grid.y > 65535u) return cudaErrorInvalidValue;
  gemm_f64_kernel<<<grid, kGemmThreads, 0, st>>>(A, Bm, C, R, K, N);
  return cudaGetLastError();
}

}  // namespace xbar
