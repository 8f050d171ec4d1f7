// assemble.cu -- nodal-system assembly for the column-block formulation.
//
// The nodal matrix of Sec. II-A (Eqs. 1-7) couples, inside bit line j, the
// bit-line nodes u(:,j) in a tridiagonal chain T_j (segments g_b, the open top
// of Eq. 3, the sense resistor g_o at the bottom) and each u(i,j) to its
// word-line node w(i,j) through G_ij; word-line nodes couple to the next
// column through g_w.  Eliminating u(:,j) inside the column leaves, on the
// word-line nodes of column j, the dense block
//     C_j = diag(dW_j) - diag(G_j) T_j^{-1} diag(G_j)
// and the current of bit line j becomes a linear functional of w(:,j):
//     I_j = g_o u(M,j) = h_j . w_j,   h_j = g_o G_j o (T_j^{-1} e_M).
// Everything about T_j^{-1} is obtained from two subtraction-free pivot
// recurrences (top-down and bottom-up "grounded parts" of the chain), so all
// quantities keep full relative accuracy.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace xbar {

// Gc[j][i] = G[i][j] (row-major M x N input), zero in the padding rows i >= M.  With `status`
// set, every entry is also checked (finite and >= 0) and XBAR_DEV_BADINPUT recorded otherwise.
__global__ void asm_gc_kernel(MapDev m, const double* __restrict__ G, unsigned* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= m.Mp || j >= m.N) return;
  const double g = i < m.M ? G[(size_t)i * m.N + j] : 0.0;
  if (status && !(g >= 0.0 && g <= 1.79e308)) set_status(status, XBAR_DEV_BADINPUT);
  m.Gc[(size_t)j * m.Mp + i] = g;
}

// The pivot recurrences of T_j are chains of linear-fractional maps, x -> g_b (G + x) / (G + x + g_b)
// (top-down: alpha_i from alpha_{i-1} with G = G_{i-1}; bottom-up: beta_i from beta_{i+1} with
// G = G_{i+1}).  A map is the 2 x 2 matrix [[g_b, g_b G], [1, G + g_b]] acting on (x, 1), and a chain of
// them is the matrix product: all entries are >= 0, so products keep full relative accuracy.  One warp
// takes a bit line: each lane composes the maps of its segment of rows, a warp scan composes the
// segments, and each lane then walks only its own rows from the value the scan gives at their start.
struct Mob {
  double a, b, c, d;  // x -> (a x + b) / (c x + d)
};
__device__ __forceinline__ Mob mob_id() { return {1.0, 0.0, 0.0, 1.0}; }
__device__ __forceinline__ Mob mob_step(double G, double gb) { return {gb, gb * G, 1.0, G + gb}; }
// X o Y, rescaled by a power of two (exact) so that the largest entry is in [1/2, 1)
__device__ __forceinline__ Mob mob_mul(const Mob& X, const Mob& Y) {
  const Mob r{X.a * Y.a + X.b * Y.c, X.a * Y.b + X.b * Y.d, X.c * Y.a + X.d * Y.c, X.c * Y.b + X.d * Y.d};
  int e;
  frexp(fmax(fmax(r.a, r.b), fmax(r.c, r.d)), &e);
  return {ldexp(r.a, -e), ldexp(r.b, -e), ldexp(r.c, -e), ldexp(r.d, -e)};
}
__device__ __forceinline__ double mob_apply(const Mob& X, double x) { return (X.a * x + X.b) / (X.c * x + X.d); }
__device__ __forceinline__ Mob shfl_up_mob(const Mob& X, int k) {
  return {__shfl_up_sync(0xffffffffu, X.a, k), __shfl_up_sync(0xffffffffu, X.b, k),
          __shfl_up_sync(0xffffffffu, X.c, k), __shfl_up_sync(0xffffffffu, X.d, k)};
}
__device__ __forceinline__ Mob shfl_down_mob(const Mob& X, int k) {
  return {__shfl_down_sync(0xffffffffu, X.a, k), __shfl_down_sync(0xffffffffu, X.b, k),
          __shfl_down_sync(0xffffffffu, X.c, k), __shfl_down_sync(0xffffffffu, X.d, k)};
}

// One warp per bit line j (blocks of 4 warps); lane L owns rows [L K, L K + K), K = ceil(M / 32).
__global__ void asm_columns_kernel(MapDev m) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= m.N) return;  // whole warps leave together
  const int M = m.M, N = m.N, Mp = m.Mp;
  const double gs = m.gs, gw = m.gw, gb = m.gb, go = m.go;
  const double* Gc = m.Gc + (size_t)j * Mp;
  double* dW = m.dW + (size_t)j * Mp;
  double* tha = m.tha + (size_t)j * Mp;
  double* thc = m.thc + (size_t)j * Mp;
  double* tdiag = m.tdiag + (size_t)j * Mp;
  double* rho = m.rho + (size_t)j * Mp;
  double* h = m.h + (size_t)j * Mp;
  const int K = (M + 31) / 32;
  const int i0 = min(lane * K, M), i1 = min(i0 + K, M);

  // top-down: pivots d-_i = G_i + alpha_i + (i < M-1 ? g_b : g_o),
  //           alpha_0 = 0, alpha_i = g_b t / (t + g_b), t = G_{i-1} + alpha_{i-1}
  // this lane's maps produce alpha_i for i0 < i <= i1 (i <= M - 1)
  Mob P = mob_id();
  for (int i = i0 + 1; i <= i1 && i <= M - 1; ++i) P = mob_mul(mob_step(Gc[i - 1], gb), P);
#pragma unroll
  for (int k = 1; k < 32; k <<= 1) {  // inclusive scan: P = S_L o S_{L-1} o ... o S_0
    const Mob Y = shfl_up_mob(P, k);
    if (lane >= k) P = mob_mul(P, Y);
  }
  Mob E = shfl_up_mob(P, 1);  // the maps before this lane's rows
  if (lane == 0) E = mob_id();
  double alpha = mob_apply(E, 0.0);  // alpha_{i0}
  for (int i = i0; i < i1; ++i) {
    const double g = Gc[i];
    if (i > i0) {
      const double t = Gc[i - 1] + alpha;
      alpha = gb * t / (t + gb);
    }
    const double dminus = g + alpha + (i < M - 1 ? gb : go);
    const double inv = 1.0 / dminus;
    dW[i] = g + (j == 0 ? gs : gw) + (j < N - 1 ? gw : 0.0);
    tha[i] = g * inv;
    thc[i] = gb * inv;
    tdiag[i] = alpha;  // kept until the bottom-up pass (same thread)
  }
  // bottom-up: pivots d+_i = G_i + beta_i + (i > 0 ? g_b : 0),
  //            beta_{M-1} = g_o, beta_i = g_b t / (t + g_b), t = G_{i+1} + beta_{i+1}
  // this lane's maps produce beta_i for i0 <= i < i1 (i <= M - 2)
  Mob Q = mob_id();
  for (int i = i0; i < min(i1, M - 1); ++i) Q = mob_mul(Q, mob_step(Gc[i + 1], gb));  // g_i0 o ... o g_top
#pragma unroll
  for (int k = 1; k < 32; k <<= 1) {  // inclusive suffix scan: Q = T_L o T_{L+1} o ... o T_31
    const Mob Y = shfl_down_mob(Q, k);
    if (lane + k < 32) Q = mob_mul(Q, Y);
  }
  Mob U = shfl_down_mob(Q, 1);  // the maps below this lane's rows
  if (lane == 31) U = mob_id();
  // diag(T^-1)_i = 1 / (G_i + alpha_i + beta_i);  rho_i = g_b / d+_i;  h_i = g_o G_i diag(T^-1)_i q_i,
  // q_i = prod_{k=i+1}^{M-1} rho_k
  double beta = mob_apply(U, go);  // beta_{i1} (g_o when i1 >= M - 1)
  double rp = 1.0;                 // product of rho over this lane's rows
  for (int i = i1 - 1; i >= i0; --i) {
    const double g = Gc[i];
    if (i < M - 1) {
      const double t = Gc[i + 1] + beta;
      beta = gb * t / (t + gb);
    } else {
      beta = go;
    }
    const double dplus = g + beta + (i > 0 ? gb : 0.0);
    tdiag[i] = 1.0 / (g + tdiag[i] + beta);
    rho[i] = gb / dplus;
    rp *= rho[i];
  }
  double qs = rp;  // suffix product over lanes L .. 31
#pragma unroll
  for (int k = 1; k < 32; k <<= 1) {
    const double y = __shfl_down_sync(0xffffffffu, qs, k);
    if (lane + k < 32) qs *= y;
  }
  double q = __shfl_down_sync(0xffffffffu, qs, 1);  // rows below this lane's
  if (lane == 31) q = 1.0;
  for (int i = i1 - 1; i >= i0; --i) {
    if (i < i1 - 1) q *= rho[i + 1];
    h[i] = go * Gc[i] * tdiag[i] * q;
  }
  for (int i = M + lane; i < Mp; i += 32) {
    dW[i] = 1.0;
    tha[i] = 0.0;
    thc[i] = 0.0;
    tdiag[i] = 0.0;
    rho[i] = 0.0;
    h[i] = 0.0;
  }
}

// Equilibration and coupling vectors; one thread per (j, i).
__global__ void asm_scale_kernel(MapDev m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= m.Mp || j >= m.N) return;
  const int Mp = m.Mp;
  const size_t o = (size_t)j * Mp + i;
  const bool real = i < m.M;
  const double s = real ? 1.0 / sqrt(m.dW[o]) : 1.0;
  const double snext = (real && j + 1 < m.N) ? 1.0 / sqrt(m.dW[o + Mp]) : 0.0;
  const double e_eq = (real && j + 1 < m.N) ? m.gw * s * snext : 0.0;
  const double e_pl = (real && j + 1 < m.N) ? m.gw : 0.0;
  m.s_eq[o] = s;
  m.e_eq[o] = e_eq;
  m.e_pl[o] = e_pl;
  m.hs_eq[o] = s * m.h[o];
  m.s32[o] = (float)s;
  m.e32[o] = (float)e_eq;
  m.hs32[o] = (float)(s * m.h[o]);
  auto pair = [](double x) {
    const float hi = (float)x;
    return make_float2(hi, (float)(x - (double)hi));
  };
  m.Gc2[o] = pair(m.Gc[o]);
  m.h2[o] = pair(m.h[o]);
  m.tha2[o] = pair(m.tha[o]);
  m.thc2[o] = pair(m.thc[o]);
  if (j == 0) {
    m.src_eq[i] = real ? m.gs * s : 0.0;
    m.src_pl[i] = real ? m.gs : 0.0;
    m.src32[i] = (float)(real ? m.gs * s : 0.0);
  }
}

// Off-diagonal of C_j: Coff_j[i][k] = -G_i G_k T^-1_{ik} (i != k), zero on the diagonal and in
// padding.  One thread per (j, row i) computes the row with running products along k and stores
// it as column i (the block is symmetric), which keeps the stores coalesced.
__global__ void asm_coff_kernel(MapDev m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= m.Mp || j >= m.N) return;
  const int M = m.M, Mp = m.Mp;
  double* C = m.Coff + (size_t)j * Mp * Mp;
  const double* Gc = m.Gc + (size_t)j * Mp;
  const double* tdiag = m.tdiag + (size_t)j * Mp;
  const double* rho = m.rho + (size_t)j * Mp;
  if (i >= M) {
    for (int k = 0; k < Mp; ++k) C[(size_t)k * Mp + i] = 0.0;
    return;
  }
  const double gi = Gc[i];
  C[(size_t)i * Mp + i] = 0.0;
  double p = tdiag[i];  // T^-1_{i,k} for k > i: tdiag_i * prod_{m=i+1}^{k} rho_m
  for (int k = i + 1; k < M; ++k) {
    p *= rho[k];
    C[(size_t)k * Mp + i] = -gi * Gc[k] * p;
  }
  double pr = 1.0;      // T^-1_{i,k} for k < i: tdiag_k * prod_{m=k+1}^{i} rho_m
  for (int k = i - 1; k >= 0; --k) {
    pr *= rho[k + 1];
    C[(size_t)k * Mp + i] = -gi * Gc[k] * tdiag[k] * pr;
  }
  for (int k = M; k < Mp; ++k) C[(size_t)k * Mp + i] = 0.0;
}

cudaError_t launch_store_g(const MapDev& m, const double* G_dev, unsigned* status, cudaStream_t st) {
  dim3 g((m.Mp + 127) / 128, m.N);
  asm_gc_kernel<<<g, 128, 0, st>>>(m, G_dev, status);
  return cudaGetLastError();
}

cudaError_t launch_assemble(const MapDev& m, cudaStream_t st) {
  asm_columns_kernel<<<(m.N + 3) / 4, 128, 0, st>>>(m);
  dim3 g2((m.Mp + 127) / 128, m.N);
  asm_scale_kernel<<<g2, 128, 0, st>>>(m);
  asm_coff_kernel<<<g2, 128, 0, st>>>(m);
  return cudaGetLastError();
}

__global__ void d2f_kernel(const double* a, float* b, size_t n) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    b[k] = (float)a[k];
}

cudaError_t launch_d2f(const double* a, float* b, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  d2f_kernel<<<blocks, 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

}  // namespace xbar
