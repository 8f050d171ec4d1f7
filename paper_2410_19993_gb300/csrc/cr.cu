// cr.cu -- block cyclic reduction over the columns: a factorization whose dense work is batches
// of independent M x M products, and the matching substitution.
//
// The word-line system left after the bit lines are eliminated inside each column (assemble.cu)
// is block tridiagonal over the N columns (Sec. II-B ordering by column, Sec. II-C LU once per
// conductance map).  Written with non-negative coupling blocks,
//     D_j x_j - L_j x_prev(j) - U_j x_next(j) = r_j,      U_j = L_next(j)^T,
// with D_j the dense M x M column block and, initially, L_j, U_j the diagonal word-line couplings.
// Odd-even reduction eliminates every second block of the current set J: for an eliminated k with
// kept neighbours p < k < q,
//     x_k = D_k^-1 (r_k + L_k x_p + U_k x_q) = D_k^-1 r_k + P_k x_p + Q_k x_q,
//     P_k = D_k^-1 L_k,   Q_k = D_k^-1 U_k,
// and substituting it into rows p and q gives the next, half-sized block-tridiagonal system
//     D_p <- D_p - U_p P_k,   D_q <- D_q - U_k^T Q_k,   U_p <- U_p Q_k   (new coupling p -> q),
//     r_p <- r_p + P_k^T r_k, r_q <- r_q + Q_k^T r_k.
// After ceil(log2 N) levels one block (column 0) remains.  The factor stores D_k^-1, P_k and Q_k
// of every eliminated block; the substitution reduces the right-hand side level by level,
// solves the last block and recovers the eliminated blocks in reverse order.  Every level is a
// batch of independent dense products, so the whole GPU works on one conductance map (block
// Thomas instead walks N dependent steps).
//
// Subtraction-free diagonals.  The system is an M-matrix whose weighted row sums are small
// positive "grounded" conductances: K w = gamma with weights w = 1 (plain) or w = s^-1
// (equilibrated, K = S K0 S), gamma = s o (h_j + g_s [j = 0]) >= 0.  Eliminating blocks maps gamma
// like a right-hand side (gamma_p <- gamma_p + P_k^T gamma_k, all terms >= 0), so after every
// level each kept diagonal is set from its off-diagonal magnitudes instead of by subtraction:
//     D_p(i,i) = (gamma_p(i) + sum_{m != i} |D_p(i,m)| w_p(m) + (U_p w_q)(i) + (U_pp^T w_pp)(i)) / w_p(i),
// the idea of the GTH variant of Gaussian elimination for M-matrices (the same device the block
// Thomas factor uses).  All products of the factor have operands of one sign (D^-1, L, U, P, Q >= 0),
// so no product cancels either.
//
// Inverses.  Blocks of up to 128 rows are inverted by Gauss-Jordan in registers (gemm_jobs.cu).
// Larger blocks (M up to 256) use the 2 x 2 block form with A = D[0:128, 0:128]:
//     W = A^-1 B,  S = C - B^T W (its diagonal again from weighted row sums),
//     D^-1 = [A^-1 - W X21, X12; X21, S^-1],  X21 = -S^-1 W^T,  X12 = -W S^-1,
// so most of the flops of the inversion are products as well.
//
// FP32 factors run their products on the tensor cores (gemm_jobs_tc.cu, three-term BF16 split,
// FP32-level accuracy) when M >= 128, and on the CUDA cores otherwise; FP64 factors run on the
// CUDA cores.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "handle.h"
#include "kernels.h"

namespace xbar {

// blocks of up to 256 rows; grids put the column count in y/z (<= 65535)
bool cr_supported(int Mp, int N) { return Mp <= 256 && N <= 65535; }

template <typename T>
__device__ __forceinline__ T cr_warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- level 0 -------------------------------------------------------------------------------------
template <typename T>
struct CrInitParams {
  int M, Mp, N;
  double gs;
  const double* Coff;  // [N][Mp][Mp] off-diagonal of the column blocks (unscaled)
  const double* h;     // [N][Mp]
  const T* s;          // [N][Mp] equilibration in the factor's precision, or nullptr
  const T* e;          // [N][Mp] coupling column j -> j+1 (equilibrated if s is set)
  T *D, *gam, *om, *gD;
};

// D_j (scaled) with its subtraction-free diagonal; gamma, weights w and block leakage gD.
// Grid (ceil(Mp/8), N), warp per row.  The scales and weights are read in the factor's precision
// (s32 / its reciprocal for FP32; unscaled for FP64), so the inner loop has no FP64 division.
template <typename T>
__global__ void cr_init_kernel(CrInitParams<T> p) {
  const int j = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + warp;
  if (i >= p.Mp) return;
  const int M = p.M, Mp = p.Mp, N = p.N;
  const size_t vo = (size_t)j * Mp;
  const bool real = i < M;
  const T* s = p.s;  // nullptr: unscaled
  const T si = (real && s) ? s[vo + i] : (T)1;
  T* Drow = p.D + (vo + i) * Mp;
  const double* Crow = p.Coff + (vo + i) * Mp;
  T off = (T)0;
  for (int m = lane; m < Mp; m += 32) {
    if (m == i) continue;
    T v = (T)0;
    if (real && m < M) {
      const T sm = s ? s[vo + m] : (T)1;
      v = (T)Crow[m] * (si * sm);
      off += s ? fabs(v) / sm : fabs(v);
    }
    Drow[m] = v;
  }
  off = cr_warp_sum(off);
  if (lane == 0) {
    T gam = (T)1, om = (T)1, cpl = (T)0;
    if (real) {
      gam = si * (T)(p.h[vo + i] + (j == 0 ? p.gs : 0.0));
      om = s ? (T)1 / si : (T)1;
      if (j > 0) cpl += s ? p.e[vo - Mp + i] / s[vo - Mp + i] : p.e[vo - Mp + i];
      if (j + 1 < N) cpl += s ? p.e[vo + i] / s[vo + Mp + i] : p.e[vo + i];
    }
    p.gam[vo + i] = gam;
    p.om[vo + i] = om;
    p.gD[vo + i] = gam + cpl;
    Drow[i] = real ? (gam + cpl + off) / om : (T)1;
  }
}

// P_k = D_k^-1 diag(e_{k-1}), Q_k = D_k^-1 diag(e_k) for the odd blocks k = 2t+1.  Grid (Mp, n_elim).
template <typename T>
__global__ void cr_l0_pq_kernel(int Mp, int N, const T* __restrict__ e, const T* __restrict__ Dinv, T* P, T* Q) {
  const int i = blockIdx.x, k = 2 * blockIdx.y + 1;
  const size_t ro = ((size_t)k * Mp + i) * Mp;
  for (int m = threadIdx.x; m < Mp; m += blockDim.x) {
    const T d = Dinv[ro + m];
    P[ro + m] = d * e[(size_t)(k - 1) * Mp + m];
    Q[ro + m] = k + 1 < N ? d * e[(size_t)k * Mp + m] : (T)0;
  }
}

// Even blocks p = 2t: D_p -= diag(e_{p-1}) D_{p-1}^-1 diag(e_{p-1}) + diag(e_p) D_{p+1}^-1 diag(e_p)
// and the next level's coupling U_p = diag(e_p) D_{p+1}^-1 diag(e_{p+1}).  Grid (Mp, n_kept).
template <typename T>
__global__ void cr_l0_upd_kernel(int Mp, int N, const T* __restrict__ e, const T* __restrict__ Dinv, T* D,
                                 T* Unew) {
  const int i = blockIdx.x, p = 2 * blockIdx.y;
  const bool hl = p > 0, hr = p + 1 < N, hrr = p + 2 < N;
  const T eli = hl ? e[(size_t)(p - 1) * Mp + i] : (T)0;
  const T eri = hr ? e[(size_t)p * Mp + i] : (T)0;
  const size_t ro = ((size_t)p * Mp + i) * Mp;
  for (int m = threadIdx.x; m < Mp; m += blockDim.x) {
    T v = D[ro + m];
    if (hl) v -= eli * Dinv[((size_t)(p - 1) * Mp + i) * Mp + m] * e[(size_t)(p - 1) * Mp + m];
    T u = (T)0;
    if (hr) {
      const T d = Dinv[((size_t)(p + 1) * Mp + i) * Mp + m];
      v -= eri * d * e[(size_t)p * Mp + m];
      if (hrr) u = eri * d * e[(size_t)(p + 1) * Mp + m];
    }
    D[ro + m] = v;
    Unew[ro + m] = u;
  }
}

// ---- every level: leakage and diagonals of the kept blocks ----------------------------------------
// Grid (kept blocks, Mp / 64): a block of 1024 threads handles 64 rows i of one kept p (with left /
// right eliminated neighbours kl, kr and next / previous kept blocks pn, pp of the next level; -1
// where absent).  Column sums (gamma' and the left coupling's row sums) split the summation index
// 16 ways with every load of a thread independent; row sums use two warps per row.
constexpr int kGthThreads = 1024, kGthRows = 64, kGthParts = kGthThreads / kGthRows;
template <typename T>
__global__ void __launch_bounds__(kGthThreads) cr_gth_kernel(int Mp, const CrGthIdx* __restrict__ idx,
                                                             const T* __restrict__ P, const T* __restrict__ Q,
                                                             T* gam, const T* __restrict__ om, T* D,
                                                             const T* __restrict__ U, T* gD) {
  __shared__ T gpart[kGthParts][kGthRows], lpart[kGthParts][kGthRows], rpart[2][kGthRows], opart[2][kGthRows];
  const CrGthIdx x = idx[blockIdx.x];
  const int i0 = blockIdx.y * kGthRows;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const size_t MM = (size_t)Mp * Mp;
  {
    const int il = tid % kGthRows, part = tid / kGthRows, i = i0 + il;
    const int q = (Mp + kGthParts - 1) / kGthParts, m0 = part * q;
    T g = (T)0, lc = (T)0;
    if (i < Mp) {
      // blocks that do not exist are skipped, never read (their storage may hold anything)
      const bool hl = x.kl >= 0, hr = x.kr >= 0, hu = x.pp >= 0;
      const T* Qk = Q + (size_t)(hl ? x.kl : 0) * MM;
      const T* gl = gam + (size_t)(hl ? x.kl : 0) * Mp;
      const T* Pk = P + (size_t)(hr ? x.kr : 0) * MM;
      const T* gr = gam + (size_t)(hr ? x.kr : 0) * Mp;
      const T* Up = U + (size_t)(hu ? x.pp : 0) * MM;
      const T* wpp = om + (size_t)(hu ? x.pp : 0) * Mp;
      T sa = (T)0, sb = (T)0, sc = (T)0;
#pragma unroll
      for (int u = 0; u < 16; ++u) {  // fully unrolled: the loads are independent (Mp <= 256: q <= 16)
        const int m = m0 + u;
        if (u < q && m < Mp) {
          if (hl) sa = fma(Qk[(size_t)m * Mp + i], gl[m], sa);
          if (hr) sb = fma(Pk[(size_t)m * Mp + i], gr[m], sb);
          if (hu) sc = fma(Up[(size_t)m * Mp + i], wpp[m], sc);
        }
      }
      g = sa + sb;
      lc = sc;
    }
    gpart[part][il] = g;
    lpart[part][il] = lc;
  }
  // row sums: two warps per row (32 warps, 64 rows: 4 rows per warp pair)
  const T* wp = om + (size_t)x.p * Mp;
  const bool hn = x.pn >= 0;
  const T* wn = om + (size_t)(hn ? x.pn : 0) * Mp;
  const int half = warp & 1;
  for (int il = warp >> 1; il < kGthRows; il += kGthThreads / 64) {
    const int i = i0 + il;
    T off = (T)0, rc = (T)0;
    if (i < Mp) {
      const T* Drow = D + ((size_t)x.p * Mp + i) * Mp;
      const T* Urow = U + ((size_t)x.p * Mp + i) * Mp;
      T dv[4], uv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int m = half * 128 + lane + 32 * u;
        const bool in = m < Mp;
        dv[u] = (in && m != i) ? fabs(Drow[m]) * wp[m] : (T)0;
        uv[u] = (in && hn) ? Urow[m] * wn[m] : (T)0;
      }
      off = (dv[0] + dv[1]) + (dv[2] + dv[3]);
      rc = (uv[0] + uv[1]) + (uv[2] + uv[3]);
    }
    off = cr_warp_sum(off);
    rc = cr_warp_sum(rc);
    if (lane == 0) {
      opart[half][il] = off;
      rpart[half][il] = rc;
    }
  }
  __syncthreads();
  if (tid < kGthRows) {
    const int i = i0 + tid;
    if (i < Mp) {
      T gs = (T)0, ls = (T)0;
#pragma unroll
      for (int pt = 0; pt < kGthParts; ++pt) {
        gs += gpart[pt][tid];
        ls += lpart[pt][tid];
      }
      const T g = gam[(size_t)x.p * Mp + i] + gs;
      const T gd = g + ls + (rpart[0][tid] + rpart[1][tid]);
      const T off = opart[0][tid] + opart[1][tid];
      gam[(size_t)x.p * Mp + i] = g;
      gD[(size_t)x.p * Mp + i] = gd;
      D[((size_t)x.p * Mp + i) * Mp + i] = (gd + off) / wp[i];
    }
  }
}

// Diagonal of S = C - B^T W (2 x 2 block inversion of block k, W = A^-1 B <= 0):
// S w_c = gD_c - W^T gD_a.  Grid (eliminated blocks, c / 64): 64 rows of S per block of 1024
// threads; ks[jj] = k, W + jj h c.
template <typename T>
__global__ void __launch_bounds__(kGthThreads) cr_gth_s_kernel(int Mp, int h, const int* __restrict__ ks,
                                                               const T* __restrict__ W, T* Dinv,
                                                               const T* __restrict__ gD, const T* __restrict__ om) {
  __shared__ T gpart[kGthParts][kGthRows], opart[kGthRows];
  const int c = Mp - h, jj = blockIdx.x, k = ks[jj], i0 = blockIdx.y * kGthRows;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const T* Wk = W + (size_t)jj * h * c;
  const T* g = gD + (size_t)k * Mp;
  const T* w = om + (size_t)k * Mp + h;
  {
    const int il = tid % kGthRows, part = tid / kGthRows, i = i0 + il;
    const int q = (h + kGthParts - 1) / kGthParts, m0 = part * q;  // h <= 128: q <= 8
    T a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int m = m0 + u;
      a[u] = (i < c && u < q && m < h) ? Wk[(size_t)m * c + i] * g[m] : (T)0;
    }
    gpart[part][il] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  }
  T* S = Dinv + ((size_t)k * Mp + h) * Mp + h;
  for (int il = warp; il < kGthRows; il += kGthThreads / 32) {
    const int i = i0 + il;
    T off = (T)0;
    if (i < c) {
      T v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int m = lane + 32 * u;
        v[u] = (m < c && m != i) ? fabs(S[(size_t)i * Mp + m]) * w[m] : (T)0;
      }
      off = (v[0] + v[1]) + (v[2] + v[3]);
    }
    off = cr_warp_sum(off);
    if (lane == 0) opart[il] = off;
  }
  __syncthreads();
  if (tid < kGthRows) {
    const int i = i0 + tid;
    if (i < c) {
      T gs = (T)0;
#pragma unroll
      for (int pt = 0; pt < kGthParts; ++pt) gs += gpart[pt][tid];
      S[(size_t)i * Mp + i] = (g[h + i] - gs + opart[tid]) / w[i];
    }
  }
}

// ---- substitution kernels ----------------------------------------------------------------------------
// r_0 = src o V^T (initial mode: the right-hand side is non-zero in column 0 only)
template <typename T>
__global__ void cr_rhs_kernel(int M, int Mp, int B, int Bpad, const T* __restrict__ src, const double* __restrict__ V,
                              T* r0) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (b >= Bpad) return;
  r0[(size_t)i * Bpad + b] = (i < M && b < B) ? src[i] * (T)V[(size_t)b * M + i] : (T)0;
}

// zero the padding rows M..Mp-1 of every column block of a [N][Mp][Bpad] array
template <typename T>
__global__ void cr_zero_pad_kernel(int M, int Mp, int Bpad, T* r) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x, i = M + blockIdx.y, j = blockIdx.z;
  if (b < Bpad) r[((size_t)j * Mp + i) * Bpad + b] = (T)0;
}

// level 0, even p: r_p += e_{p-1} o y_{p-1} + e_p o y_{p+1}  (y_k = D_k^-1 r_k, held in x)
template <typename T>
__global__ void cr_l0_fwd_kernel(int Mp, int N, int Bpad, const T* __restrict__ e, const T* __restrict__ y, T* r) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y, p = 2 * blockIdx.z;
  if (b >= Bpad) return;
  const size_t col = (size_t)Mp * Bpad;
  const size_t o = ((size_t)p * Mp + i) * Bpad + b;
  T v = r[o];
  if (p > 0) v += e[(size_t)(p - 1) * Mp + i] * y[o - col];
  if (p + 1 < N) v += e[(size_t)p * Mp + i] * y[o + col];
  r[o] = v;
}

// currents I_j(b) = hs_j . x_j(:, b) (I = dI or I += dI with the max relative change)
template <typename T>
__global__ void cr_currents_kernel(int M, int Mp, int N, int B, int Bpad, const T* __restrict__ hs,
                                   const T* __restrict__ x, double* I, int accumulate, float* max_rel,
                                   unsigned* status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  float local = 0.0f;
  if (b < B) {
    T acc = (T)0;
    const T* hj = hs + (size_t)j * Mp;
    const T* xj = x + (size_t)j * Mp * Bpad + b;
    for (int i = 0; i < M; ++i) acc = fma(hj[i], xj[(size_t)i * Bpad], acc);
    const double dI = (double)acc;
    if (!isfinite(dI)) set_status(status, XBAR_DEV_NONFINITE);
    double* Ip = I + (size_t)b * N + j;
    if (accumulate) {
      const double In = *Ip + dI;
      *Ip = In;
      local = (float)(fabs(dI) / fmax(fabs(In), 1e-300));
    } else {
      *Ip = dI;
    }
  }
  if (max_rel) {
    for (int o = 16; o > 0; o >>= 1) local = fmaxf(local, __shfl_xor_sync(0xffffffffu, local, o));
    if ((threadIdx.x & 31) == 0 && local > 0.0f) atomic_max_nonneg(max_rel, local);
  }
}

// ---------------------------------------------------------------------------------------------------
// Host side: the level plan (built once per handle and precision), the factor and the substitution
// ---------------------------------------------------------------------------------------------------
namespace {

template <typename T>
cudaError_t upload(DevArena& A, Buf& b, const std::vector<T>& v, cudaStream_t st) {
  if (v.empty()) return cudaSuccess;
  cudaError_t e = ensure(A, b, v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);  // v is a host vector that goes out of scope
}

}  // namespace

template <typename T>
static void cr_levels(CrPlanBase& pl, int N) {
  pl.lv.clear();
  std::vector<int> J(N);
  for (int j = 0; j < N; ++j) J[j] = j;
  while (J.size() > 1) {
    CrLevel L;
    const int n = (int)J.size();
    for (int t = 1; t < n; t += 2) {
      L.ek.push_back(J[t]);
      L.ep.push_back(J[t - 1]);
      L.eq.push_back(t + 1 < n ? J[t + 1] : -1);
    }
    std::vector<int> K;
    for (int t = 0; t < n; t += 2) {
      CrGthIdx x;
      x.p = J[t];
      x.kl = t > 0 ? J[t - 1] : -1;
      x.kr = t + 1 < n ? J[t + 1] : -1;
      x.pn = t + 2 < n ? J[t + 2] : -1;
      x.pp = t >= 2 ? J[t - 2] : -1;
      L.kept.push_back(x);
      K.push_back(J[t]);
    }
    pl.lv.push_back(L);
    J.swap(K);
  }
  pl.root = J[0];
}

template <typename T>
static cudaError_t cr_build(xbar_s* hd, CrPlan<T>& pl, bool tensor) {
  const MapDev& m = hd->m;
  DevArena& A = hd->A;
  const int Mp = m.Mp, N = m.N;
  const size_t MM = (size_t)Mp * Mp;
  pl.M = m.M;
  pl.Mp = Mp;
  pl.N = N;
  pl.tensor = tensor;
  cr_levels<T>(pl, N);
  cudaError_t e;
#define CR_ENSURE(buf, bytes)                   \
  do {                                          \
    e = ensure(A, (buf), (bytes));              \
    if (e != cudaSuccess) return e;             \
  } while (0)
  CR_ENSURE(pl.D, N * MM * sizeof(T));
  CR_ENSURE(pl.Dinv, N * MM * sizeof(T));
  CR_ENSURE(pl.P, N * MM * sizeof(T));
  CR_ENSURE(pl.Q, N * MM * sizeof(T));
  CR_ENSURE(pl.U[0], N * MM * sizeof(T));
  CR_ENSURE(pl.U[1], N * MM * sizeof(T));
  CR_ENSURE(pl.gam, (size_t)N * Mp * sizeof(T));
  CR_ENSURE(pl.om, (size_t)N * Mp * sizeof(T));
  CR_ENSURE(pl.gD, (size_t)N * Mp * sizeof(T));
  const int h = 128, c = Mp - 128;
  const bool two = Mp > 128;
  if (two) CR_ENSURE(pl.W, (size_t)std::max(1, (N + 1) / 2) * h * c * sizeof(T));
#undef CR_ENSURE
  T* D = (T*)pl.D.p;
  T* Dinv = (T*)pl.Dinv.p;
  T* P = (T*)pl.P.p;
  T* Q = (T*)pl.Q.p;
  T* U[2] = {(T*)pl.U[0].p, (T*)pl.U[1].p};
  T* W = (T*)pl.W.p;

  std::vector<GemmJob<T>> jobs;
  std::vector<GjJob<T>> gjs;
  std::vector<CrGthIdx> gidx;
  std::vector<int> ks;
  pl.ops.clear();
  auto op = [&](int kind, int off, int cnt, int mm, int nn, int aux) {
    CrOp o;
    o.kind = kind;
    o.off = off;
    o.cnt = cnt;
    o.m = mm;
    o.n = nn;
    o.aux = aux;
    pl.ops.push_back(o);
  };
  auto gemm_op = [&](int off, int mm, int nn) {
    const int cnt = (int)jobs.size() - off;
    if (cnt <= 0) return;
    const bool tc = tensor && sizeof(T) == 4;
    op(CR_OP_GEMM, off, cnt, mm, nn, tc ? (nn > 128 ? 256 : 128) : 0);
  };
  auto job = [&](T* C, int ldc, const T* Cin, int ldcin, T alpha) {
    GemmJob<T> g;
    memset(&g, 0, sizeof(g));
    g.C = C;
    g.ldc = ldc;
    g.Cin = Cin;
    g.ldcin = ldcin;
    g.alpha = alpha;
    g.nseg = 0;
    jobs.push_back(g);
    return (int)jobs.size() - 1;
  };
  auto seg = [&](int jid, const T* Am, int lda, int ta, const T* Bm, int ldb, int tb, int k) {
    GemmJob<T>& g = jobs[jid];
    const int s = g.nseg++;
    g.A[s] = Am;
    g.lda[s] = lda;
    g.ta[s] = ta;
    g.B[s] = Bm;
    g.ldb[s] = ldb;
    g.tb[s] = tb;
    g.k[s] = k;
  };
  // inversion of the blocks `list` (Dinv_k = D_k^-1)
  auto inverse = [&](const std::vector<int>& list) {
    if (list.empty()) return;
    if (!two) {
      const int off = (int)gjs.size();
      for (int k : list) gjs.push_back(GjJob<T>{D + k * MM, Dinv + k * MM, Mp, Mp});
      op(CR_OP_GJ, off, (int)list.size(), Mp, Mp, 0);
      return;
    }
    int off = (int)gjs.size();
    for (int k : list) gjs.push_back(GjJob<T>{D + k * MM, Dinv + k * MM, Mp, Mp});  // A^-1 (leading 128)
    op(CR_OP_GJ, off, (int)list.size(), h, h, 0);
    int jo = (int)jobs.size();
    for (size_t t = 0; t < list.size(); ++t) {  // W = A^-1 B
      const int k = list[t];
      const int g = job(W + t * h * c, c, nullptr, 0, (T)1);
      seg(g, Dinv + k * MM, Mp, 0, D + k * MM + h, Mp, 0, h);
    }
    gemm_op(jo, h, c);
    jo = (int)jobs.size();
    for (size_t t = 0; t < list.size(); ++t) {  // S = C - B^T W
      const int k = list[t];
      const int g = job(Dinv + k * MM + (size_t)h * Mp + h, Mp, D + k * MM + (size_t)h * Mp + h, Mp, (T)-1);
      seg(g, D + k * MM + (size_t)h * Mp, Mp, 0, W + t * h * c, c, 0, h);
    }
    gemm_op(jo, c, c);
    const int ko = (int)ks.size();
    for (int k : list) ks.push_back(k);
    op(CR_OP_GTHS, ko, (int)list.size(), h, c, 0);
    off = (int)gjs.size();
    for (int k : list) {
      T* S = Dinv + k * MM + (size_t)h * Mp + h;
      gjs.push_back(GjJob<T>{S, S, Mp, Mp});
    }
    op(CR_OP_GJ, off, (int)list.size(), c, c, 0);
    jo = (int)jobs.size();
    for (size_t t = 0; t < list.size(); ++t) {  // X21 = -S^-1 W^T
      const int k = list[t];
      const int g = job(Dinv + k * MM + (size_t)h * Mp, Mp, nullptr, 0, (T)-1);
      seg(g, Dinv + k * MM + (size_t)h * Mp + h, Mp, 0, W + t * h * c, c, 1, c);
    }
    gemm_op(jo, c, h);
    jo = (int)jobs.size();
    for (size_t t = 0; t < list.size(); ++t) {  // X12 = -W S^-1
      const int k = list[t];
      const int g = job(Dinv + k * MM + h, Mp, nullptr, 0, (T)-1);
      seg(g, W + t * h * c, c, 0, Dinv + k * MM + (size_t)h * Mp + h, Mp, 0, c);
    }
    gemm_op(jo, h, c);
    jo = (int)jobs.size();
    for (size_t t = 0; t < list.size(); ++t) {  // A^-1 - W X21
      const int k = list[t];
      const int g = job(Dinv + k * MM, Mp, Dinv + k * MM, Mp, (T)-1);
      seg(g, W + t * h * c, c, 0, Dinv + k * MM + (size_t)h * Mp, Mp, 0, c);
    }
    gemm_op(jo, h, h);
  };

  op(CR_OP_INIT, 0, 0, 0, 0, 0);
  int ucur = -1;  // U buffer of the current level (-1: level 0, diagonal couplings)
  for (size_t l = 0; l < pl.lv.size(); ++l) {
    const CrLevel& L = pl.lv[l];
    inverse(L.ek);
    const int unew = ucur < 0 ? 0 : 1 - ucur;
    if (l == 0) {
      op(CR_OP_L0PQ, 0, (int)L.ek.size(), Mp, Mp, 0);
      op(CR_OP_L0UPD, 0, (int)L.kept.size(), Mp, Mp, unew);
    } else {
      int jo = (int)jobs.size();
      for (size_t t = 0; t < L.ek.size(); ++t) {  // P_k = D_k^-1 U_p^T, Q_k = D_k^-1 U_k
        const int k = L.ek[t], p = L.ep[t], q = L.eq[t];
        int g = job(P + k * MM, Mp, nullptr, 0, (T)1);
        seg(g, Dinv + k * MM, Mp, 0, U[ucur] + p * MM, Mp, 1, Mp);
        if (q >= 0) {
          g = job(Q + k * MM, Mp, nullptr, 0, (T)1);
          seg(g, Dinv + k * MM, Mp, 0, U[ucur] + k * MM, Mp, 0, Mp);
        }
      }
      gemm_op(jo, Mp, Mp);
      jo = (int)jobs.size();
      for (const CrGthIdx& x : L.kept) {  // D_p -= U_kl^T Q_kl + U_p P_kr ; U_p' = U_p Q_kr
        const int p = x.p;
        if (x.kl >= 0 || x.kr >= 0) {
          const int g = job(D + p * MM, Mp, D + p * MM, Mp, (T)-1);
          if (x.kl >= 0) seg(g, U[ucur] + x.kl * MM, Mp, 1, Q + x.kl * MM, Mp, 0, Mp);
          if (x.kr >= 0) seg(g, U[ucur] + p * MM, Mp, 0, P + x.kr * MM, Mp, 0, Mp);
        }
        if (x.kr >= 0 && x.pn >= 0) {
          const int g = job(U[unew] + p * MM, Mp, nullptr, 0, (T)1);
          seg(g, U[ucur] + p * MM, Mp, 0, Q + x.kr * MM, Mp, 0, Mp);
        }
      }
      gemm_op(jo, Mp, Mp);
    }
    const int go = (int)gidx.size();
    for (const CrGthIdx& x : L.kept) gidx.push_back(x);
    op(CR_OP_GTH, go, (int)L.kept.size(), Mp, Mp, unew);
    ucur = unew;
  }
  inverse(std::vector<int>{pl.root});

  e = upload(A, pl.jobs, jobs, hd->st);
  if (e == cudaSuccess) e = upload(A, pl.gj, gjs, hd->st);
  if (e == cudaSuccess) e = upload(A, pl.gidx, gidx, hd->st);
  if (e == cudaSuccess) e = upload(A, pl.ks, ks, hd->st);
  if (e != cudaSuccess) return e;
  pl.njobs_factor = (int)jobs.size();
  pl.built = 1;
  cr_clear_solve_cache(A, pl);
  return cudaSuccess;
}

template <typename T>
static cudaError_t cr_run_gemm(xbar_s* hd, const CrPlan<T>& pl, const GemmJob<T>* jobs, const CrOp& o) {
  if (o.aux && sizeof(T) == 4)
    return launch_gemm_jobs_tc(reinterpret_cast<const GemmJob<float>*>(jobs) + o.off, o.cnt, o.m, o.n, o.aux,
                               hd->nsm, hd->status, hd->st);
  return launch_gemm_jobs<T>(jobs + o.off, o.cnt, o.m, o.n, hd->status, hd->st);
}

template <typename T>
cudaError_t cr_prepare(xbar_s* hd, CrPlan<T>& pl, bool tensor) {
  const MapDev& m = hd->m;
  if (pl.built && pl.tensor == tensor && pl.Mp == m.Mp && pl.N == m.N && pl.M == m.M) return cudaSuccess;
  return cr_build<T>(hd, pl, tensor);
}

template <typename T>
cudaError_t cr_factor(xbar_s* hd, CrPlan<T>& pl, bool tensor, bool equilibrate) {
  const MapDev& m = hd->m;
  {
    cudaError_t e = cr_prepare<T>(hd, pl, tensor);
    if (e != cudaSuccess) return e;
  }
  const int Mp = m.Mp, N = m.N;
  const size_t MM = (size_t)Mp * Mp;
  cudaStream_t st = hd->st;
  T* D = (T*)pl.D.p;
  T* Dinv = (T*)pl.Dinv.p;
  // couplings in the factor's precision: FP32 factors are equilibrated, FP64 ones are not
  const T* e = sizeof(T) == 4 ? (const T*)(const void*)m.e32 : (const T*)(const void*)m.e_pl;
  if ((sizeof(T) == 4) != equilibrate) return cudaErrorInvalidValue;
  const GemmJob<T>* jobs = (const GemmJob<T>*)pl.jobs.p;
  const GjJob<T>* gjs = (const GjJob<T>*)pl.gj.p;
  for (const CrOp& o : pl.ops) {
    cudaError_t err = cudaSuccess;
    switch (o.kind) {
      case CR_OP_INIT: {
        CrInitParams<T> ip;
        ip.M = m.M;
        ip.Mp = Mp;
        ip.N = N;
        ip.gs = m.gs;
        ip.Coff = m.Coff;
        ip.h = m.h;
        ip.s = equilibrate ? (const T*)(const void*)m.s32 : nullptr;  // FP32 factors only
        ip.e = e;
        ip.D = D;
        ip.gam = (T*)pl.gam.p;
        ip.om = (T*)pl.om.p;
        ip.gD = (T*)pl.gD.p;
        cr_init_kernel<T><<<dim3((Mp + 7) / 8, N), 256, 0, st>>>(ip);
        err = cudaGetLastError();
        break;
      }
      case CR_OP_GJ:
        err = launch_gj_inverse<T>(gjs + o.off, o.cnt, o.m, hd->status, st);
        break;
      case CR_OP_GEMM:
        err = cr_run_gemm<T>(hd, pl, jobs, o);
        break;
      case CR_OP_L0PQ:
        cr_l0_pq_kernel<T><<<dim3(Mp, o.cnt), 128, 0, st>>>(Mp, N, e, Dinv, (T*)pl.P.p, (T*)pl.Q.p);
        err = cudaGetLastError();
        break;
      case CR_OP_L0UPD:
        cr_l0_upd_kernel<T><<<dim3(Mp, o.cnt), 128, 0, st>>>(Mp, N, e, Dinv, D, (T*)pl.U[o.aux].p);
        err = cudaGetLastError();
        break;
      case CR_OP_GTH:
        cr_gth_kernel<T><<<dim3(o.cnt, (Mp + kGthRows - 1) / kGthRows), kGthThreads, 0, st>>>(Mp, (const CrGthIdx*)pl.gidx.p + o.off, (const T*)pl.P.p,
                                                (const T*)pl.Q.p, (T*)pl.gam.p, (const T*)pl.om.p, D,
                                                (const T*)pl.U[o.aux].p, (T*)pl.gD.p);
        err = cudaGetLastError();
        break;
      case CR_OP_GTHS:
        cr_gth_s_kernel<T><<<dim3(o.cnt, (Mp - o.m + kGthRows - 1) / kGthRows), kGthThreads, 0, st>>>(Mp, o.m, (const int*)pl.ks.p + o.off, (const T*)pl.W.p, Dinv,
                                                  (const T*)pl.gD.p, (const T*)pl.om.p);
        err = cudaGetLastError();
        break;
      default:
        err = cudaErrorInvalidValue;
    }
    if (err != cudaSuccess) return err;
  }
  (void)MM;
  pl.factored = 1;
  return cudaSuccess;
}

// ---- substitution ------------------------------------------------------------------------------------
// Plan of one substitution: right-hand side buffer r, solution x ([N][Mp][Bpad]), mode.
template <typename T>
static cudaError_t cr_solve_plan(xbar_s* hd, CrPlan<T>& pl, T* r, T* x, int Bpad, bool initial, bool tensor,
                                 CrSolvePlan** out) {
  for (CrSolvePlan& sp : pl.solve_cache)
    if (sp.r == (void*)r && sp.x == (void*)x && sp.Bpad == Bpad && sp.initial == initial && sp.tensor == tensor) {
      *out = &sp;
      return cudaSuccess;
    }
  const int Mp = pl.Mp, N = pl.N;
  const size_t MM = (size_t)Mp * Mp, MB = (size_t)Mp * Bpad;
  const T* Dinv = (const T*)pl.Dinv.p;
  const T* P = (const T*)pl.P.p;
  const T* Q = (const T*)pl.Q.p;
  std::vector<GemmJob<T>> jobs;
  CrSolvePlan sp;
  sp.r = r;
  sp.x = x;
  sp.Bpad = Bpad;
  sp.initial = initial;
  sp.tensor = tensor;
  const int tcn = (tensor && sizeof(T) == 4) ? (Bpad > 128 ? 256 : 128) : 0;
  auto job = [&](T* C, const T* Cin) {
    GemmJob<T> g;
    memset(&g, 0, sizeof(g));
    g.C = C;
    g.ldc = Bpad;
    g.Cin = Cin;
    g.ldcin = Bpad;
    g.alpha = (T)1;
    jobs.push_back(g);
    return (int)jobs.size() - 1;
  };
  auto seg = [&](int jid, const T* Am, int ta, const T* Bm) {
    GemmJob<T>& g = jobs[jid];
    const int s = g.nseg++;
    g.A[s] = Am;
    g.lda[s] = Mp;
    g.ta[s] = ta;
    g.B[s] = Bm;
    g.ldb[s] = Bpad;
    g.tb[s] = 0;
    g.k[s] = Mp;
  };
  auto gemm_op = [&](int off) {
    const int cnt = (int)jobs.size() - off;
    if (cnt <= 0) return;
    CrOp o;
    o.kind = CR_OP_GEMM;
    o.off = off;
    o.cnt = cnt;
    o.m = Mp;
    o.n = Bpad;
    o.aux = tcn;
    sp.ops.push_back(o);
  };
  const int L = (int)pl.lv.size();
  if (!initial) {
    for (int l = 0; l < L; ++l) {  // forward reduction of the right-hand side
      const CrLevel& lv = pl.lv[l];
      int jo = (int)jobs.size();
      if (l == 0) {
        for (int k : lv.ek) seg(job(x + k * MB, nullptr), Dinv + k * MM, 0, r + k * MB);  // y_k
        gemm_op(jo);
        CrOp o;
        o.kind = CR_OP_L0FWD;
        o.off = 0;
        o.cnt = (int)lv.kept.size();
        o.m = Mp;
        o.n = Bpad;
        o.aux = 0;
        sp.ops.push_back(o);
      } else {
        for (const CrGthIdx& k : lv.kept) {
          if (k.kl < 0 && k.kr < 0) continue;
          const int g = job(r + k.p * MB, r + k.p * MB);
          if (k.kl >= 0) seg(g, Q + k.kl * MM, 1, r + k.kl * MB);
          if (k.kr >= 0) seg(g, P + k.kr * MM, 1, r + k.kr * MB);
        }
        gemm_op(jo);
      }
    }
  }
  {  // last block
    const int jo = (int)jobs.size();
    seg(job(x + pl.root * MB, nullptr), Dinv + pl.root * MM, 0, r + pl.root * MB);
    gemm_op(jo);
  }
  for (int l = L - 1; l >= 0; --l) {  // back substitution
    const CrLevel& lv = pl.lv[l];
    const int jo = (int)jobs.size();
    for (size_t t = 0; t < lv.ek.size(); ++t) {
      const int k = lv.ek[t], p = lv.ep[t], q = lv.eq[t];
      const bool have_y = (l == 0) && !initial;  // x_k holds y_k = D_k^-1 r_k from the forward pass
      const int g = job(x + k * MB, have_y ? x + k * MB : nullptr);
      if (l > 0 && !initial) seg(g, Dinv + k * MM, 0, r + k * MB);
      seg(g, P + k * MM, 0, x + p * MB);
      if (q >= 0) seg(g, Q + k * MM, 0, x + q * MB);
    }
    gemm_op(jo);
  }
  cudaError_t e = upload(hd->A, sp.jobs, jobs, hd->st);
  if (e != cudaSuccess) return e;
  if (pl.solve_cache.size() >= 4) {  // oldest plan out, with its job list
    if (pl.solve_cache.front().jobs.p) hd->A.release(pl.solve_cache.front().jobs.p);
    pl.solve_cache.erase(pl.solve_cache.begin());
  }
  pl.solve_cache.push_back(sp);  // the cache entry owns sp.jobs from here on
  *out = &pl.solve_cache.back();
  return cudaSuccess;
}

template <typename T>
cudaError_t cr_sweep(xbar_s* hd, CrPlan<T>& pl, const CrSweepArgs<T>& a) {
  const int M = pl.M, Mp = pl.Mp, N = pl.N, Bpad = a.Bpad;
  cudaStream_t st = hd->st;
  const bool initial = a.V != nullptr;
  CrSolvePlan* sp = nullptr;
  cudaError_t e = cr_solve_plan<T>(hd, pl, a.r, a.x, Bpad, initial, a.tensor, &sp);
  if (e != cudaSuccess) return e;
  const T* e_cpl = (const T*)a.e;
  if (initial) {
    cr_rhs_kernel<T><<<dim3((Bpad + 127) / 128, Mp), 128, 0, st>>>(M, Mp, a.B, Bpad, a.src, a.V,
                                                                   a.r + (size_t)pl.root * Mp * Bpad);
  } else if (Mp > M) {
    cr_zero_pad_kernel<T><<<dim3((Bpad + 127) / 128, Mp - M, N), 128, 0, st>>>(M, Mp, Bpad, a.r);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const GemmJob<T>* jobs = (const GemmJob<T>*)sp->jobs.p;
  for (const CrOp& o : sp->ops) {
    if (o.kind == CR_OP_GEMM) {
      e = cr_run_gemm<T>(hd, pl, jobs, o);
    } else if (o.kind == CR_OP_L0FWD) {
      cr_l0_fwd_kernel<T><<<dim3((Bpad + 127) / 128, Mp, o.cnt), 128, 0, st>>>(Mp, N, Bpad, e_cpl, a.x, a.r);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
  }
  cr_currents_kernel<T><<<dim3((a.B + 127) / 128, N), 128, 0, st>>>(M, Mp, N, a.B, Bpad, a.hs, a.x, a.I,
                                                                     a.accumulate, a.max_rel, hd->status);
  return cudaGetLastError();
}

void cr_clear_solve_cache(DevArena& A, CrPlanBase& pl) {
  for (CrSolvePlan& sp : pl.solve_cache)
    if (sp.jobs.p) A.release(sp.jobs.p);
  pl.solve_cache.clear();
}

template cudaError_t cr_prepare<float>(xbar_s*, CrPlan<float>&, bool);
template cudaError_t cr_prepare<double>(xbar_s*, CrPlan<double>&, bool);
template cudaError_t cr_factor<float>(xbar_s*, CrPlan<float>&, bool, bool);
template cudaError_t cr_factor<double>(xbar_s*, CrPlan<double>&, bool, bool);
template cudaError_t cr_sweep<float>(xbar_s*, CrPlan<float>&, const CrSweepArgs<float>&);
template cudaError_t cr_sweep<double>(xbar_s*, CrPlan<double>&, const CrSweepArgs<double>&);

}  // namespace xbar
