// gemm_jobs.cu -- batched dense kernels of the cyclic-reduction factor and substitution on the
// CUDA cores: job-list GEMMs (FP32 or FP64) and Gauss-Jordan inversion of symmetric M-matrices.
//
// Every level of block cyclic reduction over the columns is a batch of independent dense M x M
// operations on different column blocks: inverses of the blocks it eliminates and products
// that form the couplings and Schur complements of the blocks it keeps.  A launch processes one
// list of such jobs; the host builds the lists once per factorization plan.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace xbar {

// ---------------------------------------------------------------------------------------------
// Job-list GEMM, 64 x TN output tiles (TN = 64, or 16 for narrow right-hand sides such as a few
// input vectors), 256 threads: thread (ty, tx) computes rows ty + 16 r (r < 4) and columns
// tx + 16 c (c < TN / 16); K is staged through shared memory in slabs of 16.
// ---------------------------------------------------------------------------------------------
constexpr int kGT = 64, kGK = 16;

template <typename T, int TN>
__global__ void __launch_bounds__(256) gemm_jobs_kernel(const GemmJob<T>* __restrict__ jobs, int m, int n,
                                                        int tiles_n) {
  constexpr int CW = TN / 16;
  __shared__ T As[kGK][kGT + 1];
  __shared__ T Bs[kGK][TN + 4];
  const GemmJob<T>& jb = jobs[blockIdx.y];
  const int i0 = (blockIdx.x / tiles_n) * kGT, j0 = (blockIdx.x % tiles_n) * TN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[4][CW];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < CW; ++c) acc[r][c] = (T)0;

  const int nseg = jb.nseg;
  for (int s = 0; s < nseg; ++s) {
    const T* A = jb.A[s];
    const T* B = jb.B[s];
    const int lda = jb.lda[s], ldb = jb.ldb[s], K = jb.k[s], ta = jb.ta[s], tb = jb.tb[s];
    for (int k0 = 0; k0 < K; k0 += kGK) {
      // A slab: rows i0..i0+63, k k0..k0+15 -> As[kk][i]
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int t = tid + 256 * u;
        int i, kk;
        if (ta) { kk = t >> 6; i = t & 63; }   // A[kk][i]: consecutive threads along i
        else { i = t >> 4; kk = t & 15; }      // A[i][kk]: consecutive threads along kk
        const int gi = i0 + i, gk = k0 + kk;
        T v = (T)0;
        if (gi < m && gk < K) v = ta ? A[(size_t)gk * lda + gi] : A[(size_t)gi * lda + gk];
        As[kk][i] = v;
      }
      // B slab: k k0..k0+15, columns j0..j0+TN-1 -> Bs[kk][j]
#pragma unroll
      for (int u = 0; u < CW; ++u) {
        const int t = tid + 256 * u;
        int j, kk;
        if (tb) { j = t >> 4; kk = t & 15; }       // B[j][kk]
        else { kk = t / TN; j = t % TN; }          // B[kk][j]
        const int gj = j0 + j, gk = k0 + kk;
        T v = (T)0;
        if (gj < n && gk < K) v = tb ? B[(size_t)gj * ldb + gk] : B[(size_t)gk * ldb + gj];
        Bs[kk][j] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < kGK; ++kk) {
        T a[4], b[CW];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
        for (int c = 0; c < CW; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < CW; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
      }
      __syncthreads();
    }
  }
  const T alpha = jb.alpha;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int gi = i0 + ty + 16 * r;
    if (gi >= m) continue;
#pragma unroll
    for (int c = 0; c < CW; ++c) {
      const int gj = j0 + tx + 16 * c;
      if (gj >= n) continue;
      T v = alpha * acc[r][c];
      if (jb.Cin) v += jb.Cin[(size_t)gi * jb.ldcin + gj];
      jb.C[(size_t)gi * jb.ldc + gj] = v;
    }
  }
}

template <typename T>
cudaError_t launch_gemm_jobs(const GemmJob<T>* jobs_dev, int njobs, int m, int n, unsigned* status,
                             cudaStream_t st) {
  (void)status;
  if (njobs <= 0 || m <= 0 || n <= 0) return cudaSuccess;
  if (njobs > 65535) return cudaErrorInvalidValue;
  const int tm = (m + kGT - 1) / kGT;
  if (n <= 16) {
    gemm_jobs_kernel<T, 16><<<dim3(tm, njobs), 256, 0, st>>>(jobs_dev, m, n, 1);
  } else {
    const int tn = (n + kGT - 1) / kGT;
    gemm_jobs_kernel<T, 64><<<dim3(tm * tn, njobs), 256, 0, st>>>(jobs_dev, m, n, tn);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Gauss-Jordan inversion in registers.  The matrix (padded with the identity to NT x NT) is held
// by 4 NT threads: thread (ty, tx) owns rows ty + (NT/8) r (r < 8) and columns tx + 32 c
// (c < NT/32).  Step q replaces the matrix by the sweep operator at pivot q:
//     a_qq <- 1/a_qq,  a_qm <- a_qm/a_qq,  a_iq <- -a_iq/a_qq,  a_im <- a_im - a_iq a_qm / a_qq,
// after which all n steps leave the inverse in place.  No pivoting: the matrices are symmetric
// M-matrices (positive definite), so every pivot is positive.  The owners of row q and column q
// publish them through shared memory (double-buffered: one barrier per step).  Pivots run in the
// natural order q = rq + (NT/8) aq with aq the outer, unrolled loop, so every register index is a
// compile-time constant.
// ---------------------------------------------------------------------------------------------
template <typename T, int NT>
__global__ void __launch_bounds__(NT * 4) gj_kernel(const GjJob<T>* __restrict__ jobs, int n) {
  constexpr int RG = NT / 8;   // row groups = warps
  constexpr int CB = NT / 32;  // columns per lane
  __shared__ T prow[2][NT], pcol[2][NT];
  const GjJob<T> jb = jobs[blockIdx.x];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  T a[8][CB];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = ty + RG * r;
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      const int mm = tx + 32 * c;
      a[r][c] = (i < n && mm < n) ? jb.src[(size_t)i * jb.lds + mm] : (i == mm ? (T)1 : (T)0);
    }
  }
#pragma unroll
  for (int aq = 0; aq < 8; ++aq) {
    for (int rq = 0; rq < RG; ++rq) {
      const int q = rq + RG * aq;
      if (q >= n) break;  // uniform: identity padding needs no steps
      const int buf = q & 1, cq = q & 31, bq = q >> 5;
      if (ty == rq) {
#pragma unroll
        for (int c = 0; c < CB; ++c) prow[buf][tx + 32 * c] = a[aq][c];
      }
      if (tx == cq) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          T v = a[r][0];
#pragma unroll
          for (int c = 1; c < CB; ++c)
            if (c == bq) v = a[r][c];
          pcol[buf][ty + RG * r] = v;
        }
      }
      __syncthreads();
      const T inv = (T)1 / prow[buf][q];
      T rs[CB], cs[8];
#pragma unroll
      for (int c = 0; c < CB; ++c) rs[c] = prow[buf][tx + 32 * c] * inv;
#pragma unroll
      for (int r = 0; r < 8; ++r) cs[r] = pcol[buf][ty + RG * r];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < CB; ++c) a[r][c] = fma(-cs[r], rs[c], a[r][c]);
      if (ty == rq) {  // pivot row
#pragma unroll
        for (int c = 0; c < CB; ++c) a[aq][c] = rs[c];
      }
      if (tx == cq) {  // pivot column (and the pivot itself)
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int c = 0; c < CB; ++c)
            if (c == bq) a[r][c] = (ty == rq && r == aq) ? inv : -cs[r] * inv;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = ty + RG * r;
    if (i >= n) continue;
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      const int mm = tx + 32 * c;
      if (mm < n) jb.dst[(size_t)i * jb.ldd + mm] = a[r][c];
    }
  }
}

template <typename T>
cudaError_t launch_gj_inverse(const GjJob<T>* jobs_dev, int njobs, int n, unsigned* status, cudaStream_t st) {
  (void)status;
  if (njobs <= 0 || n <= 0) return cudaSuccess;
  if (n <= 32) gj_kernel<T, 32><<<njobs, 128, 0, st>>>(jobs_dev, n);
  else if (n <= 64) gj_kernel<T, 64><<<njobs, 256, 0, st>>>(jobs_dev, n);
  else if (n <= 128) gj_kernel<T, 128><<<njobs, 512, 0, st>>>(jobs_dev, n);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template cudaError_t launch_gemm_jobs<float>(const GemmJob<float>*, int, int, int, unsigned*, cudaStream_t);
template cudaError_t launch_gemm_jobs<double>(const GemmJob<double>*, int, int, int, unsigned*, cudaStream_t);
template cudaError_t launch_gj_inverse<float>(const GjJob<float>*, int, int, unsigned*, cudaStream_t);
template cudaError_t launch_gj_inverse<double>(const GjJob<double>*, int, int, unsigned*, cudaStream_t);

}  // namespace xbar
