// factor.cu -- block Thomas factorization of the word-line system (Sec. II-C: one decomposition
// per conductance map).
//
// After the bit lines are eliminated inside each column (assemble.cu) the word-line unknowns form
// a block-tridiagonal system with dense M x M diagonal blocks C_j and couplings -g_w I between
// neighbouring columns.  Block Thomas gives
//     Z_0 = C_0,   Z_j = C_j - g_w^2 X_{j-1},   X_j = Z_j^{-1}          (sequential in j)
// and the substitutions only need the X_j.  With diagonal equilibration S_j (optional) the kernel
// factors S K S instead and stores X^_j = S_j^{-1} X_j S_j^{-1}.
//
// Subtraction-free diagonals.  Z_j is an M-matrix whose row sums are small and positive (the
// conductance to ground seen from column j); forming diag(Z_j) as C_jj - g_w^2 X_jj cancels
// almost all digits in FP32.  Instead the kernel carries the grounded row sums
//     sigma_0 = h_0 + g_s,    sigma_j = h_j + g_w X_{j-1} sigma_{j-1}
// (all terms >= 0; h_j is the bit-line current functional), and sets
//     Z_ii = sigma_i + g_w [j < N-1] + sum_{k != i} |Z_ik|,
// the same idea as the GTH variant of Gaussian elimination for M-matrices.  Row sums of Z_j are
// sigma_j + g_w [j < N-1] exactly in exact arithmetic, so nothing changes mathematically.
//
// Parallel layout.  A group of co-resident blocks (cooperative launch) owns one map; block g holds
// rows [g*R, (g+1)*R) of the current matrix in shared memory and the inversion is an in-place
// blocked Gauss-Jordan sweep with panels of PB rows (no pivoting: Z_j is symmetric positive
// definite).  Before each panel its owners publish the panel rows to global memory, a bounded
// cross-block barrier orders the exchange, and every block inverts the PB x PB pivot block itself
// and updates its own rows.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace xbar {

constexpr int kFactorThreads = 256;

template <typename T>
struct FacPB;
template <>
struct FacPB<double> { static constexpr int value = 16; };
template <>
struct FacPB<float> { static constexpr int value = 16; };

template <typename T>
int factor_panel_width() { return FacPB<T>::value; }

template <typename T>
size_t factor_smem_bytes(int Mp, int R) {
  constexpr int PB = FacPB<T>::value;
  size_t n = (size_t)R * Mp + (size_t)PB * Mp + PB * PB + (size_t)R * PB + Mp + R;
  return n * sizeof(T) + 16;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(kFactorThreads)
    factor_kernel(const FactorParams<T>* __restrict__ maps, int blocks_per_map, unsigned* status) {
  constexpr int PB = FacPB<T>::value;
  const FactorParams<T> p = maps[blockIdx.x / blocks_per_map];
  const int g = blockIdx.x % blocks_per_map;
  const int M = p.M, Mp = p.Mp, N = p.N;
  const int R = (Mp + blocks_per_map - 1) / blocks_per_map;  // rows per block
  const int r0 = g * R;
  const int nr = max(0, min(R, Mp - r0));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nwarps = kFactorThreads / 32;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* rows = reinterpret_cast<T*>(smem_raw);   // [R][Mp]
  T* pn = rows + (size_t)R * Mp;              // [PB][Mp]
  T* D = pn + (size_t)PB * Mp;                // [PB][PB]
  T* W = D + PB * PB;                         // [R][PB]
  T* sigv = W + R * PB;                       // [Mp]
  T* sgm = sigv + Mp;                         // [R] sigma_j of own rows
  __shared__ unsigned flag;
  __shared__ T rinv_s;

  const uint64_t limit = wait_limit(status);
  const T gw = (T)p.gw;
  const int npanel = Mp / PB;

  for (int j = 0; j < N; ++j) {
    const double* Cj = p.Coff + (size_t)j * Mp * Mp;
    const double* sj = p.s ? p.s + (size_t)j * Mp : nullptr;
    const double* sjm = (p.s && j > 0) ? p.s + (size_t)(j - 1) * Mp : nullptr;
    const double* ejm = j > 0 ? p.e + (size_t)(j - 1) * Mp : nullptr;
    const double* hj = p.h + (size_t)j * Mp;

    // (1) sigma_j of own rows (needs X^_{j-1} own rows, still in `rows`, and all of sigma_{j-1})
    if (j > 0) {
      const T* sp = p.sig + (size_t)((j - 1) & 1) * Mp;
      for (int k = tid; k < Mp; k += kFactorThreads)
        sigv[k] = ld_cg(sp + k) * (sjm ? (T)sjm[k] : (T)1);
      __syncthreads();
      for (int r = warp; r < nr; r += nwarps) {
        const int i = r0 + r;
        T acc = 0;
        for (int k = lane; k < Mp; k += 32) acc += rows[(size_t)r * Mp + k] * sigv[k];
        acc = warp_sum(acc);
        if (lane == 0)
          sgm[r] = (i < M) ? (T)hj[i] + gw * (sjm ? (T)sjm[i] : (T)1) * acc : (T)0;
      }
    } else {
      for (int r = tid; r < nr; r += kFactorThreads) {
        const int i = r0 + r;
        sgm[r] = (i < M) ? (T)(hj[i] + p.gsrc) : (T)0;
      }
    }
    __syncthreads();
    for (int r = tid; r < nr; r += kFactorThreads) p.sig[(size_t)(j & 1) * Mp + r0 + r] = sgm[r];

    // (2) X^_{j-1} own rows to the output
    if (j > 0) {
      T* Xo = p.X + (size_t)(j - 1) * Mp * Mp + (size_t)r0 * Mp;
      for (int t = tid; t < nr * Mp; t += kFactorThreads) Xo[t] = rows[t];
    }
    __syncthreads();

    // (3) Z^_j own rows: off-diagonal, then the subtraction-free diagonal
    for (int t = tid; t < nr * Mp; t += kFactorThreads) {
      const int r = t / Mp, k = t - r * Mp, i = r0 + r;
      T v = 0;
      if (i < M && k < M && k != i) {
        const T si = sj ? (T)sj[i] : (T)1, sk = sj ? (T)sj[k] : (T)1;
        v = si * sk * (T)Cj[(size_t)i * Mp + k];
        if (j > 0) v -= (T)ejm[i] * (T)ejm[k] * rows[t];
      }
      rows[t] = v;
    }
    __syncthreads();
    for (int r = warp; r < nr; r += nwarps) {
      const int i = r0 + r;
      T acc = 0;
      for (int k = lane; k < Mp; k += 32) {
        const T sk = sj ? (T)sj[k] : (T)1;
        if (k < M) acc += fabs(rows[(size_t)r * Mp + k]) / sk;
      }
      acc = warp_sum(acc);
      if (lane == 0) {
        T d = 1;
        if (i < M) {
          const T si = sj ? (T)sj[i] : (T)1;
          d = si * si * (sgm[r] + (j < N - 1 ? gw : (T)0)) + si * acc;
        }
        rows[(size_t)r * Mp + i] = d;
      }
    }

    // (4) blocked in-place Gauss-Jordan inversion, panels of PB rows/columns
    for (int pp = 0; pp < npanel; ++pp) {
      const int P0 = pp * PB;
      const unsigned pc = (unsigned)(j * npanel + pp);
      T* pb = p.pbuf + (size_t)(pc & 1) * PB * Mp;
      __syncthreads();
      for (int t = tid; t < nr * Mp; t += kFactorThreads) {
        const int r = t / Mp, i = r0 + r;
        if (i >= P0 && i < P0 + PB) pb[(size_t)(i - P0) * Mp + (t - r * Mp)] = rows[t];
      }
      if (!group_barrier(p.bar, blocks_per_map, status, limit, &flag)) return;
      for (int t = tid; t < PB * Mp; t += kFactorThreads) pn[t] = ld_cg(pb + t);
      __syncthreads();
      for (int t = tid; t < PB * PB; t += kFactorThreads) D[t] = pn[(size_t)(t / PB) * Mp + P0 + t % PB];
      // invert the pivot block in place (scalar sweep operator, no pivoting).  The reciprocal of
      // each pivot is formed once, by the thread that owns that diagonal entry.
      if (tid == 0) rinv_s = (T)1 / D[0];
      for (int q = 0; q < PB; ++q) {
        __syncthreads();
        constexpr int PER = (PB * PB + kFactorThreads - 1) / kFactorThreads;
        T nv[PER];
        const T ri = rinv_s;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const int t = tid + u * kFactorThreads;
          if (t < PB * PB) {
            const int a = t / PB, b = t % PB;
            const T aq = D[a * PB + q], qb = D[q * PB + b], v = D[t];
            if (a == q && b == q) nv[u] = ri;
            else if (a == q) nv[u] = qb * ri;
            else if (b == q) nv[u] = -aq * ri;
            else nv[u] = v - aq * qb * ri;
          }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const int t = tid + u * kFactorThreads;
          if (t < PB * PB) {
            D[t] = nv[u];
            if (q + 1 < PB && t == (q + 1) * (PB + 1)) rinv_s = (T)1 / nv[u];
          }
        }
      }
      __syncthreads();
      // W = A_iP D for own rows outside the panel
      for (int t = tid; t < nr * PB; t += kFactorThreads) {
        const int r = t / PB, m = t % PB, i = r0 + r;
        if (i >= P0 && i < P0 + PB) continue;
        T acc = 0;
#pragma unroll
        for (int q = 0; q < PB; ++q) acc += rows[(size_t)r * Mp + P0 + q] * D[q * PB + m];
        W[t] = acc;
      }
      __syncthreads();
      for (int t = tid; t < nr * Mp; t += kFactorThreads) {
        const int r = t / Mp, k = t - r * Mp, i = r0 + r;
        const bool kin = (k >= P0 && k < P0 + PB);
        T v;
        if (i >= P0 && i < P0 + PB) {  // panel row: D * (old panel rows)
          const int q = i - P0;
          if (kin) {
            v = D[q * PB + (k - P0)];
          } else {
            T acc = 0;
#pragma unroll
            for (int m = 0; m < PB; ++m) acc += D[q * PB + m] * pn[(size_t)m * Mp + k];
            v = acc;
          }
        } else if (kin) {
          v = -W[r * PB + (k - P0)];
        } else {
          T acc = rows[t];
#pragma unroll
          for (int m = 0; m < PB; ++m) acc -= W[r * PB + m] * pn[(size_t)m * Mp + k];
          v = acc;
        }
        rows[t] = v;  // each (r, k) is read and written by the same thread only
      }
    }
    __syncthreads();
  }
  T* Xo = p.X + (size_t)(N - 1) * Mp * Mp + (size_t)r0 * Mp;
  for (int t = tid; t < nr * Mp; t += kFactorThreads) Xo[t] = rows[t];
}

template <typename T>
cudaError_t launch_factor(const FactorParams<T>* maps_dev, int nmaps, int Mp_max, int blocks_per_map,
                          unsigned* status, cudaStream_t st) {
  const int R = (Mp_max + blocks_per_map - 1) / blocks_per_map;
  const size_t smem = factor_smem_bytes<T>(Mp_max, R);
  cudaError_t err = cudaFuncSetAttribute(factor_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nmaps * blocks_per_map);
  cfg.blockDim = dim3(kFactorThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (nmaps * blocks_per_map > 1) ? 1 : 0;  // one block needs no co-residency guarantee
  return cudaLaunchKernelEx(&cfg, factor_kernel<T>, maps_dev, blocks_per_map, status);
}

template int factor_panel_width<double>();
template int factor_panel_width<float>();
template size_t factor_smem_bytes<double>(int, int);
template size_t factor_smem_bytes<float>(int, int);
template cudaError_t launch_factor<double>(const FactorParams<double>*, int, int, int, unsigned*, cudaStream_t);
template cudaError_t launch_factor<float>(const FactorParams<float>*, int, int, int, unsigned*, cudaStream_t);

}  // namespace xbar
