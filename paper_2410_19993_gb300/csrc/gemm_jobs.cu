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

  // the K slabs of all segments in order; the next slab's values are loaded into registers while
  // the current one is multiplied
  T ra[4], rb[CW];
  auto load = [&](int s, int k0) {
    const T* A = jb.A[s];
    const T* B = jb.B[s];
    const int lda = jb.lda[s], ldb = jb.ldb[s], K = jb.k[s], ta = jb.ta[s], tb = jb.tb[s];
#pragma unroll
    for (int u = 0; u < 4; ++u) {  // A slab: rows i0..i0+63, k k0..k0+15
      const int t = tid + 256 * u;
      int i, kk;
      if (ta) { kk = t >> 6; i = t & 63; }   // A[kk][i]: consecutive threads along i
      else { i = t >> 4; kk = t & 15; }      // A[i][kk]: consecutive threads along kk
      const int gi = i0 + i, gk = k0 + kk;
      ra[u] = (gi < m && gk < K) ? (ta ? A[(size_t)gk * lda + gi] : A[(size_t)gi * lda + gk]) : (T)0;
    }
#pragma unroll
    for (int u = 0; u < CW; ++u) {  // B slab: k k0..k0+15, columns j0..j0+TN-1
      const int t = tid + 256 * u;
      int j, kk;
      if (tb) { j = t >> 4; kk = t & 15; }       // B[j][kk]
      else { kk = t / TN; j = t % TN; }          // B[kk][j]
      const int gj = j0 + j, gk = k0 + kk;
      rb[u] = (gj < n && gk < K) ? (tb ? B[(size_t)gj * ldb + gk] : B[(size_t)gk * ldb + gj]) : (T)0;
    }
  };
  auto store = [&](int s) {
    const int ta = jb.ta[s], tb = jb.tb[s];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = tid + 256 * u;
      if (ta) As[t >> 6][t & 63] = ra[u];
      else As[t & 15][t >> 4] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < CW; ++u) {
      const int t = tid + 256 * u;
      if (tb) Bs[t & 15][t >> 4] = rb[u];
      else Bs[t / TN][t % TN] = rb[u];
    }
  };
  const int nseg = jb.nseg;
  int s = 0, k0 = 0;
  if (nseg > 0 && jb.k[0] > 0) load(0, 0);
  while (s < nseg) {
    const int cs = s;
    store(cs);
    __syncthreads();
    k0 += kGK;  // advance to the next slab and prefetch it
    if (k0 >= jb.k[s]) {
      k0 = 0;
      ++s;
    }
    if (s < nseg) load(s, k0);
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
// Gauss-Jordan inversion in registers, eliminating panels of 8 pivots at a time.  The matrix
// (padded with the identity to NT x NT) is held by 32 NT / RPT threads: thread (ty, tx) owns rows
// ty + (NT/RPT) r (r < RPT) and columns tx + 32 c (c < NT/32).  For the panel of pivots P..P+7, with
// D = A[P:P+8, P:P+8], panel rows R = A[P:P+8, :] and panel columns C = A[:, P:P+8]:
//     R' = D^-1 R outside the pivot columns and D^-1 inside them,
//     A[i, :] <- A[i, :] - C[i, :] R' outside the pivot columns and -C[i, :] D^-1 inside them
// for the rows i outside the panel, which is the product of the 8 single-pivot sweep operators;
// after all panels the inverse is in place.  No pivoting: the matrices are symmetric M-matrices
// (positive definite), so every pivot is positive.  The owners publish R and C to shared memory,
// one warp forms R' there (8 dependent sweep steps on 8 rows), and every thread applies the rank-8
// update to its own elements; the shared buffers alternate between panels, so each panel costs
// two block barriers.  All register indices are compile-time constants (the panel loop is unrolled).
// ---------------------------------------------------------------------------------------------
template <typename T, int NT, int RPT>
__global__ void __launch_bounds__(NT / RPT * 32) gj_kernel(const GjJob<T>* __restrict__ jobs, int n) {
  constexpr int RG = NT / RPT;  // row groups = warps
  constexpr int CB = NT / 32;   // columns per lane
  constexpr int PW = 8;        // pivots per panel
  __shared__ __align__(16) T PR[2][PW][NT];   // panel rows, then R'
  __shared__ __align__(16) T PC[2][NT][PW];   // panel columns
  const GjJob<T> jb = jobs[blockIdx.x];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  T a[RPT][CB];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int i = ty + RG * r;
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      const int mm = tx + 32 * c;
      a[r][c] = (i < n && mm < n) ? jb.src[(size_t)i * jb.lds + mm] : (i == mm ? (T)1 : (T)0);
    }
  }
  // the panel loop is not unrolled (code size): registers of a runtime row or column index are
  // picked by short compare chains
#pragma unroll 1
  for (int pn = 0; pn < NT / PW; ++pn) {
    const int P0 = pn * PW;
    if (P0 >= n) break;  // uniform: identity padding needs no steps
    const int b = pn & 1;
    // (1) publish the panel rows and columns
#pragma unroll
    for (int k = 0; k < PW; ++k) {
      const int row = P0 + k;
      if (ty == row % RG) {
        const int rk = row / RG;
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          T v = a[0][c];
#pragma unroll
          for (int r = 1; r < RPT; ++r)
            if (r == rk) v = a[r][c];
          PR[b][k][tx + 32 * c] = v;
        }
      }
    }
    {
      const int ck = P0 / 32;  // the 8 panel columns lie in one 32-column block
      const int k = tx - (P0 & 31);
      if (k >= 0 && k < PW) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          T v = a[r][0];
#pragma unroll
          for (int c = 1; c < CB; ++c)
            if (c == ck) v = a[r][c];
          PC[b][ty + RG * r][k] = v;
        }
      }
    }
    __syncthreads();
    // (2) one warp: R' = D^-1 R (8 sweep steps on the panel rows, in registers; lane l holds
    // columns l + 32 c of the 8 rows, the pivot column's values come by shuffle from its lane)
    if (ty == 0) {
      T pr[PW][CB];
#pragma unroll
      for (int k = 0; k < PW; ++k)
#pragma unroll
        for (int c = 0; c < CB; ++c) pr[k][c] = PR[b][k][tx + 32 * c];
      const int ck = P0 / 32, src = P0 & 31;
#pragma unroll
      for (int k = 0; k < PW; ++k) {
        T f[PW];  // column P0 + k of the 8 rows (lane src + k, slot ck)
#pragma unroll
        for (int l = 0; l < PW; ++l) {
          T v = pr[l][0];
#pragma unroll
          for (int c = 1; c < CB; ++c)
            if (c == ck) v = pr[l][c];
          f[l] = __shfl_sync(0xffffffffu, v, src + k);
        }
        const T inv = (T)1 / f[k];
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          const bool piv = (tx == src + k) && (c == ck);
          const T rk = piv ? inv : pr[k][c] * inv;
#pragma unroll
          for (int l = 0; l < PW; ++l) {
            if (l == k) continue;
            pr[l][c] = piv ? -f[l] * inv : fma(-f[l], rk, pr[l][c]);
          }
          pr[k][c] = rk;
        }
      }
#pragma unroll
      for (int k = 0; k < PW; ++k)
#pragma unroll
        for (int c = 0; c < CB; ++c) PR[b][k][tx + 32 * c] = pr[k][c];
    }
    __syncthreads();
    // (3) every thread: rank-8 update of its elements; R' of its columns is read once per panel, the
    // panel-column values C[i, :] once per row (a shared-memory broadcast: i is uniform in a warp)
    T rp[PW][CB];
#pragma unroll
    for (int k = 0; k < PW; ++k)
#pragma unroll
      for (int c = 0; c < CB; ++c) rp[k][c] = PR[b][k][tx + 32 * c];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int i = ty + RG * r;
      if (i >= P0 && i < P0 + PW) {  // panel row: R'
        const int k = i - P0;
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          T v = rp[0][c];
#pragma unroll
          for (int kk = 1; kk < PW; ++kk)
            if (kk == k) v = rp[kk][c];
          a[r][c] = v;
        }
        continue;
      }
      T cr[PW];
#pragma unroll
      for (int k = 0; k < PW; ++k) cr[k] = PC[b][i][k];
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        const int mm = tx + 32 * c;
        T v = (mm >= P0 && mm < P0 + PW) ? (T)0 : a[r][c];
#pragma unroll
        for (int k = 0; k < PW; ++k) v = fma(-cr[k], rp[k][c], v);
        a[r][c] = v;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int i = ty + RG * r;
    if (i >= n) continue;
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      const int mm = tx + 32 * c;
      if (mm < n) jb.dst[(size_t)i * jb.ldd + mm] = a[r][c];
    }
  }
}

// Single-pivot variant for FP64 (its register budget does not allow the panel form at 128 rows; the
// FP64 inversion is bound by the FP64 FMA rate either way).  Thread (ty, tx) owns rows
// ty + (NT/8) r (r < 8) and columns tx + 32 c (c < NT/32); each step applies one sweep operator
// (a_qq <- 1/a_qq, a_qm <- a_qm/a_qq, a_iq <- -a_iq/a_qq, a_im <- a_im - a_iq a_qm/a_qq) with the
// pivot row and column published through double-buffered shared memory (one barrier per step).
template <typename T, int NT>
__global__ void __launch_bounds__(NT * 4) gj1_kernel(const GjJob<T>* __restrict__ jobs, int n) {
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
  if constexpr (sizeof(T) == 8) {  // FP64: single-pivot steps
    if (n <= 32) gj1_kernel<T, 32><<<njobs, 128, 0, st>>>(jobs_dev, n);
    else if (n <= 64) gj1_kernel<T, 64><<<njobs, 256, 0, st>>>(jobs_dev, n);
    else if (n <= 128) gj1_kernel<T, 128><<<njobs, 512, 0, st>>>(jobs_dev, n);
    else return cudaErrorInvalidValue;
  } else {
    if (n <= 32) gj_kernel<T, 32, 8><<<njobs, 128, 0, st>>>(jobs_dev, n);
    else if (n <= 64) gj_kernel<T, 64, 8><<<njobs, 256, 0, st>>>(jobs_dev, n);
    else if (n <= 128) gj_kernel<T, 128, 8><<<njobs, 512, 0, st>>>(jobs_dev, n);
    else return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template cudaError_t launch_gemm_jobs<float>(const GemmJob<float>*, int, int, int, unsigned*, cudaStream_t);
template cudaError_t launch_gemm_jobs<double>(const GemmJob<double>*, int, int, int, unsigned*, cudaStream_t);
template cudaError_t launch_gj_inverse<float>(const GjJob<float>*, int, int, unsigned*, cudaStream_t);
template cudaError_t launch_gj_inverse<double>(const GjJob<double>*, int, int, unsigned*, cudaStream_t);

}  // namespace xbar
