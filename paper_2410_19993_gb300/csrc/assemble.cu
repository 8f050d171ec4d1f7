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

// One thread per bit line j: the chain recurrences of T_j (sequential in i), from Gc.
__global__ void asm_columns_kernel(MapDev m) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m.N) return;
  const int M = m.M, N = m.N, Mp = m.Mp;
  const double gs = m.gs, gw = m.gw, gb = m.gb, go = m.go;
  double* Gc = m.Gc + (size_t)j * Mp;
  double* dW = m.dW + (size_t)j * Mp;
  double* tha = m.tha + (size_t)j * Mp;
  double* thc = m.thc + (size_t)j * Mp;
  double* tdiag = m.tdiag + (size_t)j * Mp;
  double* rho = m.rho + (size_t)j * Mp;
  double* h = m.h + (size_t)j * Mp;

  // top-down: pivots d-_i = G_i + alpha_i + (i < M-1 ? g_b : g_o),
  //           alpha_0 = 0, alpha_i = g_b t / (t + g_b), t = G_{i-1} + alpha_{i-1}
  double alpha = 0.0, gprev = 0.0;
  for (int i = 0; i < M; ++i) {
    const double g = Gc[i];
    if (i > 0) {
      const double t = gprev + alpha;
      alpha = gb * t / (t + gb);
    }
    const double dminus = g + alpha + (i < M - 1 ? gb : go);
    const double inv = 1.0 / dminus;
    dW[i] = g + (j == 0 ? gs : gw) + (j < N - 1 ? gw : 0.0);
    tha[i] = g * inv;
    thc[i] = gb * inv;
    tdiag[i] = alpha;  // kept until the bottom-up pass
    gprev = g;
  }
  // bottom-up: pivots d+_i = G_i + beta_i + (i > 0 ? g_b : 0),
  //            beta_{M-1} = g_o, beta_i = g_b t / (t + g_b), t = G_{i+1} + beta_{i+1}
  // diag(T^-1)_i = 1 / (G_i + alpha_i + beta_i);  T^-1_{i,k} = T^-1_{i,k-1} * g_b / d+_k  (k > i)
  double beta = go, gnext = 0.0, q = 1.0;
  for (int i = M - 1; i >= 0; --i) {
    const double g = Gc[i];
    if (i < M - 1) {
      const double t = gnext + beta;
      beta = gb * t / (t + gb);
    }
    const double dplus = g + beta + (i > 0 ? gb : 0.0);
    const double td = 1.0 / (g + tdiag[i] + beta);
    tdiag[i] = td;
    if (i < M - 1) q *= rho[i + 1];  // q = prod_{k=i+1}^{M-1} rho_k
    rho[i] = gb / dplus;
    h[i] = go * g * td * q;
    gnext = g;
  }
  for (int i = M; i < Mp; ++i) {
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
  asm_columns_kernel<<<(m.N + 63) / 64, 64, 0, st>>>(m);
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
