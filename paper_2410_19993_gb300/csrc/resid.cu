// resid.cu -- FP64 steps of mixed-precision iterative refinement, and node-voltage output.
//
// The refinement state is the FP64 vector w of word-line node voltages.  Bit-line voltages are
// not stored: for any w they follow from the bit-line rows of the nodal system (Eqs. 3, 4, 7),
//     T_j u_j = G_j o w_j     (tridiagonal chain of bit line j),
// solved here in FP64 with the same subtraction-free pivots as the assembly.  The word-line rows
// (Eqs. 1, 2, 5, 6) then give the residual of the nodal system restricted to word-line nodes:
//     r(i,j) = b(i,j) + g_w (w(i,j-1) + w(i,j+1)) + G_ij u(i,j) - dW(i,j) w(i,j),
// b = g_s V_i at j = 0.  The bit-line rows hold exactly by construction of u, so r is the full
// residual of the 2MN system.  These two kernels and the update w += s o dhat are the only FP64
// arithmetic of the mixed path.
//
// One thread per (column j, input vector b); consecutive threads take consecutive b, so every
// access to the [N][Mp][Bpad] arrays is coalesced.  Loops run along the chain i.
#include <math.h>

#include "common.cuh"
#include "handle.h"
#include "kernels.h"

namespace xbar {

// w = (first ? 0 : w) + s * dhat  (FP64),  I[b][j] = h_j . w_j  (FP64)
__global__ void update_kernel(ResidParams p, int first) {
  if (p.skip && *p.skip) return;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (b >= p.Bpad || j >= p.N) return;
  const size_t base = (size_t)j * p.Mp;
  double Iacc = 0.0;
  for (int i = 0; i < p.M; ++i) {
    const size_t o = (base + i) * p.Bpad + b;
    const float d = p.s32[base + i] * p.dhat[o];
    const double wn = (first ? 0.0 : p.w[o]) + (double)d;
    p.w[o] = wn;
    Iacc = fma(p.h[base + i], wn, Iacc);
  }
  if (b < p.B) p.I[(size_t)b * p.N + j] = Iacc;
}

// forward half of the bit-line chain solve: phi_i = tha_i w_i + thc_i phi_{i-1}
__device__ __forceinline__ void chain_forward(const ResidParams& p, int j, int b) {
  const size_t base = (size_t)j * p.Mp;
  double phi = 0.0;
  for (int i = 0; i < p.M; ++i) {
    const size_t o = (base + i) * p.Bpad + b;
    phi = fma(p.thc[base + i], phi, p.tha[base + i] * p.w[o]);
    p.phi[o] = phi;
  }
}

__global__ void resid_kernel(ResidParams p) {
  if (p.skip && *p.skip) return;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (b >= p.Bpad || j >= p.N) return;
  chain_forward(p, j, b);
  const size_t base = (size_t)j * p.Mp;
  const bool has_l = j > 0, has_r = j + 1 < p.N;
  const bool src = (j == 0) && (b < p.B);
  double u = 0.0;
  float rmax = 0.0f;  // |r| tracked in FP32: only its magnitude is reported
  const size_t col = (size_t)p.Mp * p.Bpad;
  for (int i = p.M - 1; i >= 0; --i) {
    const size_t o = (base + i) * p.Bpad + b;
    u = fma(p.thc[base + i], u, p.phi[o]);  // u_i = phi_i + thc_i u_{i+1}
    const double wi = p.w[o];
    double nb = has_l ? p.w[o - col] : 0.0;
    if (has_r) nb = has_l ? nb + p.w[o + col] : p.w[o + col];
    double r = src ? p.gs * p.V[(size_t)b * p.M + i] : 0.0;
    r = fma(p.gw, nb, r);
    r = fma(p.Gc[base + i], u, r);
    r = fma(-p.dW[base + i], wi, r);
    const float rf = (float)r;
    rmax = fmaxf(rmax, fabsf(rf));
    p.rhat[o] = rf * p.s32[base + i];
  }
  if (!(rmax <= 3.0e38f)) set_status(p.status, XBAR_DEV_NONFINITE);
  // block max of |r| then one atomic (non-negative doubles order like their bit patterns)
  for (int off = 16; off > 0; off >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, off));
  if ((threadIdx.x & 31) == 0 && p.rmax)
    atomicMax(p.rmax, (unsigned long long)__double_as_longlong((double)rmax));
}

// bit-line voltages u = T^-1 (G o w), written over the scratch array `u`
__global__ void blvolt_kernel(ResidParams p, double* u_out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (b >= p.Bpad || j >= p.N) return;
  ResidParams q = p;
  q.phi = u_out;
  chain_forward(q, j, b);
  const size_t base = (size_t)j * p.Mp;
  double u = 0.0;
  for (int i = p.M - 1; i >= 0; --i) {
    const size_t o = (base + i) * p.Bpad + b;
    u = fma(p.thc[base + i], u, u_out[o]);
    u_out[o] = u;
  }
}

cudaError_t launch_update(const ResidParams& p, int first, cudaStream_t st) {
  dim3 grid((p.Bpad + 127) / 128, p.N);
  update_kernel<<<grid, 128, 0, st>>>(p, first);
  return cudaGetLastError();
}

cudaError_t launch_resid(const ResidParams& p, cudaStream_t st) {
  dim3 grid((p.Bpad + 127) / 128, p.N);
  resid_kernel<<<grid, 128, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_blvolt(const ResidParams& p, double* u, cudaStream_t st) {
  dim3 grid((p.Bpad + 127) / 128, p.N);
  blvolt_kernel<<<grid, 128, 0, st>>>(p, u);
  return cudaGetLastError();
}

__global__ void ir_init_kernel(IrState* s) {
  s->done = 0;
  s->iters = 0;
  s->last = 0.0f;
  s->prev = 0.0f;
  s->maxrel = 0.0f;
  s->rmax = 0ull;
  s->rinf = 0.0;
}

// the stopping rule of the host-driven loop: converged when this correction is within tol, or when
// the observed contraction rho = |dI_k| / |dI_{k-1}| (<= 1/2) bounds the error left after it
__global__ void ir_check_kernel(IrState* s, double tol) {
  if (s->done) return;
  const float mr = s->maxrel;
  s->prev = s->last;
  s->last = mr;
  s->iters += 1;
  s->rinf = __longlong_as_double((long long)s->rmax);
  const double rho = (s->iters >= 2 && s->prev > 0.0f) ? (double)mr / s->prev : 1.0;
  if (mr == mr && (mr <= tol || (rho <= 0.5 && (double)mr * rho / (1.0 - rho) <= tol))) s->done = 1;
  s->maxrel = 0.0f;
  s->rmax = 0ull;
}

cudaError_t launch_ir_init(IrState* state, cudaStream_t st) {
  ir_init_kernel<<<1, 1, 0, st>>>(state);
  return cudaGetLastError();
}

cudaError_t launch_ir_check(IrState* state, double tol, cudaStream_t st) {
  ir_check_kernel<<<1, 1, 0, st>>>(state, tol);
  return cudaGetLastError();
}

// out[b][i][j] = src[(j*Mp + i)*Bpad + b] for b < B, i < M: 32 x 32 tiles over (b, j) per row i
__global__ void to_user_kernel(const double* __restrict__ src, double* __restrict__ out, int M, int Mp, int N,
                               int B, int Bpad) {
  __shared__ double tile[32][33];
  const int i = blockIdx.z;
  const int bt = blockIdx.x * 32, jt = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int j = jt + r, b = bt + tx;
    tile[r][tx] = (j < N && b < Bpad) ? src[((size_t)j * Mp + i) * Bpad + b] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int b = bt + r, j = jt + tx;
    if (b < B && j < N) out[((size_t)b * M + i) * N + j] = tile[tx][r];
  }
}

cudaError_t launch_to_user_layout(const double* src, double* out, int M, int Mp, int N, int B, int Bpad,
                                  cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  dim3 grid((B + 31) / 32, (N + 31) / 32, M);
  to_user_kernel<<<grid, dim3(32, 8), 0, st>>>(src, out, M, Mp, N, B, Bpad);
  return cudaGetLastError();
}

}  // namespace xbar
