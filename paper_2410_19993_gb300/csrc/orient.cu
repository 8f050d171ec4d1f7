// orient.cu -- blocking over rows: the mirrored crossbar whose column blocks are the original rows.
//
// The block-tridiagonal word-line system (Sec. II-B column ordering, bit lines eliminated inside
// each column) has N blocks of M rows.  When N < M the other orientation is cheaper: eliminate the
// word lines inside each row instead and block over the M rows, with N x N blocks (the factor
// costs ~M N^3 instead of ~N M^3, a substitution ~4 M N^2 instead of ~4 N M^2 per vector; paper
// Sec. II-B notes that the band structure follows the orientation).
//
// Rather than a second formulation, the library builds the mirrored crossbar
//     M' = N, N' = M,  G'(i', j') = G(M-1-j', N-1-i'),
//     R_s' = R_sense, R_sense' = R_s, R_w' = R_b, R_b' = R_w,
// i.e. word line i' of the mirror is bit line N-1-i' of the original and bit line j' of the mirror
// is word line M-1-j'.  Its nodal matrix has exactly the original form (source resistor at the
// start of every word line, sense resistor at the end of every bit line), so assembly, both factor
// algorithms and both substitutions apply unchanged.  Only the right-hand side and the output move:
//  * the sources V_i now sit behind the mirror's sense resistors, at the bottom of its bit line
//    j' = M-1-i, and the mirror's source resistors lead to ground.  Eliminating bit line j' then
//    gives the word-line right-hand side  r_j' = V_(M-1-j') h'_j',  h'_j' = g_o' G'_j' o T'_j'^-1 e
//    (the same vector that maps the mirror's word-line voltages to its sense current);
//  * the original sense current of bit line j flows through the mirror's source resistor of word
//    line N-1-j into ground:  I_j = g_s' w'(N-1-j, column 0)  (the mirror's first block);
//  * node voltages: original word-line node (i, j) is the mirror's bit-line node (N-1-j, M-1-i),
//    original bit-line node (i, j) the mirror's word-line node (N-1-j, M-1-i).  The mirror's
//    bit-line voltages follow from its chain with the source term: T' u' = G' o w' + g_o' V e_last.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace xbar {

// Gc2[j'][i'] = Gc[N-1-i'][M-1-j'] (both [blocks][padded rows]), zero in the padding rows
__global__ void mirror_gc_kernel(const double* __restrict__ Gc, int M, int Mp, int N, double* __restrict__ Gc2,
                                 int Mp2) {
  const int i2 = blockIdx.x * blockDim.x + threadIdx.x;  // mirror row (< Mp2), original column N-1-i2
  const int j2 = blockIdx.y;                             // mirror column, original row M-1-j2
  if (i2 >= Mp2 || j2 >= M) return;
  Gc2[(size_t)j2 * Mp2 + i2] = i2 < N ? Gc[(size_t)(N - 1 - i2) * Mp + (M - 1 - j2)] : 0.0;
}

// rhs[j'][i'][b] = V[b][M-1-j'] h'[j'][i'] for real rows and vectors, zero elsewhere
__global__ void orient_rhs_kernel(const double* __restrict__ V, const double* __restrict__ h2, int M, int M2,
                                  int Mp2, int B, int Bpad, double* __restrict__ rhs) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int i2 = blockIdx.y, j2 = blockIdx.z;
  if (b >= Bpad) return;
  double v = 0.0;
  if (b < B && i2 < M2) v = V[(size_t)b * M + (M - 1 - j2)] * h2[(size_t)j2 * Mp2 + i2];
  rhs[((size_t)j2 * Mp2 + i2) * Bpad + b] = v;
}

// I[b][j] = g_s' w'[0][N-1-j][b]
__global__ void orient_currents_kernel(const double* __restrict__ w2, int N, int Bpad, int B, double gs2,
                                       double* __restrict__ I) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (b >= B) return;
  I[(size_t)b * N + j] = gs2 * w2[(size_t)(N - 1 - j) * Bpad + b];
}

// The mirror's bit-line voltages with the source at the bottom of each chain:
// forward phi_i = tha_i w_i + thc_i phi_(i-1) (+ g_o' V / d_last at the last row, 1/d_last = thc_last / g_b'),
// back u_i = phi_i + thc_i u_(i+1); written into u ([M'-blocks][Mp'][Bpad]).
__global__ void orient_blvolt_kernel(MapDev m2, const double* __restrict__ w2, const double* __restrict__ V,
                                     int M, int B, int Bpad, double* __restrict__ u) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int j2 = blockIdx.y;
  if (b >= Bpad || j2 >= m2.N) return;
  const int M2 = m2.M;
  const size_t base = (size_t)j2 * m2.Mp;
  const double vb = b < B ? V[(size_t)b * M + (M - 1 - j2)] : 0.0;
  const double csrc = m2.go * m2.thc[base + M2 - 1] / m2.gb;
  double phi = 0.0;
  for (int i = 0; i < M2; ++i) {
    const size_t o = (base + i) * Bpad + b;
    phi = fma(m2.thc[base + i], phi, m2.tha[base + i] * w2[o]);
    if (i == M2 - 1) phi = fma(csrc, vb, phi);
    u[o] = phi;
  }
  double uu = 0.0;
  for (int i = M2 - 1; i >= 0; --i) {
    const size_t o = (base + i) * Bpad + b;
    uu = fma(m2.thc[base + i], uu, u[o]);
    u[o] = uu;
  }
}

// out[b][i][j] = src2[(M-1-i)][(N-1-j)][b] (mirror layout [M blocks][Mp2][Bpad]): 32 x 32 tiles
// over (b, j) per original row i, read along b and written along j
__global__ void orient_to_user_kernel(const double* __restrict__ src2, double* __restrict__ out, int M, int N,
                                      int Mp2, int B, int Bpad) {
  __shared__ double tile[32][33];
  const int i = blockIdx.z;
  const int bt = blockIdx.x * 32, jt = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const size_t blk = (size_t)(M - 1 - i) * Mp2;
  for (int r = ty; r < 32; r += 8) {
    const int j = jt + r, b = bt + tx;
    tile[r][tx] = (j < N && b < Bpad) ? src2[(blk + (N - 1 - j)) * Bpad + b] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int b = bt + r, j = jt + tx;
    if (b < B && j < N) out[((size_t)b * M + i) * N + j] = tile[tx][r];
  }
}

// ---- the mirror in mixed precision (FP32 factor, float-pair refinement state) ---------------------
// equilibrated right-hand side of the FP32 substitution: rhs[j'][i'][b] = s[j'][i'] V[b][M-1-j'] h'[j'][i']
__global__ void orient_rhs32_kernel(const double* __restrict__ V, const double* __restrict__ h2,
                                    const float* __restrict__ s32, int M, int M2, int Mp2, int B, int Bpad,
                                    float* __restrict__ rhs) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int i2 = blockIdx.y, j2 = blockIdx.z;
  if (b >= Bpad) return;
  float v = 0.0f;
  if (b < B && i2 < M2) {
    const size_t c = (size_t)j2 * Mp2 + i2;
    v = s32[c] * (float)(V[(size_t)b * M + (M - 1 - j2)] * h2[c]);
  }
  rhs[((size_t)j2 * Mp2 + i2) * Bpad + b] = v;
}

// I[b][j] = g_s' w'[0][N-1-j][b] from the float-pair state (hi + lo), or from its FP32 form w1
__global__ void orient_state_currents_kernel(const float2* __restrict__ w2, const float* __restrict__ w1, int N,
                                             int Bpad, int B, double gs2, double* __restrict__ I) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (b >= B) return;
  const size_t o = (size_t)(N - 1 - j) * Bpad + b;
  const double w = w1 ? (double)w1[o] : (double)w2[o].x + (double)w2[o].y;
  I[(size_t)b * N + j] = gs2 * w;
}

// the correction's current change dI = g_s' s[0][N-1-j] dhat[0][N-1-j][b]: I += dI and the maximum of
// |dI| / |I| (atomic, non-negative floats) for the stopping rule
__global__ void orient_correction_currents_kernel(const float* __restrict__ dhat, const float* __restrict__ s32,
                                                  int N, int Bpad, int B, double gs2, double* __restrict__ I,
                                                  float* __restrict__ max_rel, unsigned* status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  float rel = 0.0f;
  if (b < B) {
    const int i2 = N - 1 - j;
    const double d = gs2 * (double)s32[i2] * (double)dhat[(size_t)i2 * Bpad + b];
    if (!isfinite(d)) set_status(status, XBAR_DEV_NONFINITE);
    double* Ip = I + (size_t)b * N + j;
    const double In = *Ip + d;
    *Ip = In;
    rel = (float)(fabs(d) / fmax(fabs(In), 1e-300));
  }
  const unsigned live = __activemask();
  rel = __uint_as_float(__reduce_max_sync(live, __float_as_uint(rel)));
  if ((threadIdx.x & 31) == __ffs(live) - 1 && max_rel && rel > 0.0f) atomic_max_nonneg(max_rel, rel);
}

cudaError_t launch_orient_rhs32(const double* V, const double* h2, const float* s32, int M, int M2, int Mp2, int B,
                                int Bpad, float* rhs, cudaStream_t st) {
  orient_rhs32_kernel<<<dim3((Bpad + 127) / 128, Mp2, M), 128, 0, st>>>(V, h2, s32, M, M2, Mp2, B, Bpad, rhs);
  return cudaGetLastError();
}

cudaError_t launch_orient_state_currents(const float2* w2, const float* w1, int N, int Bpad, int B, double gs2,
                                         double* I, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  orient_state_currents_kernel<<<dim3((B + 127) / 128, N), 128, 0, st>>>(w2, w1, N, Bpad, B, gs2, I);
  return cudaGetLastError();
}

cudaError_t launch_orient_correction_currents(const float* dhat, const float* s32, int N, int Bpad, int B,
                                              double gs2, double* I, float* max_rel, unsigned* status,
                                              cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  orient_correction_currents_kernel<<<dim3((B + 127) / 128, N), 128, 0, st>>>(dhat, s32, N, Bpad, B, gs2, I,
                                                                               max_rel, status);
  return cudaGetLastError();
}

cudaError_t launch_mirror_gc(const double* Gc, int M, int Mp, int N, double* Gc2, int Mp2, cudaStream_t st) {
  mirror_gc_kernel<<<dim3((Mp2 + 127) / 128, M), 128, 0, st>>>(Gc, M, Mp, N, Gc2, Mp2);
  return cudaGetLastError();
}

cudaError_t launch_orient_rhs(const double* V, const double* h2, int M, int M2, int Mp2, int B, int Bpad,
                              double* rhs, cudaStream_t st) {
  orient_rhs_kernel<<<dim3((Bpad + 127) / 128, Mp2, M), 128, 0, st>>>(V, h2, M, M2, Mp2, B, Bpad, rhs);
  return cudaGetLastError();
}

cudaError_t launch_orient_currents(const double* w2, int N, int Bpad, int B, double gs2, double* I,
                                   cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  orient_currents_kernel<<<dim3((B + 127) / 128, N), 128, 0, st>>>(w2, N, Bpad, B, gs2, I);
  return cudaGetLastError();
}

cudaError_t launch_orient_blvolt(const MapDev& m2, const double* w2, const double* V, int M, int B, int Bpad,
                                 double* u, cudaStream_t st) {
  orient_blvolt_kernel<<<dim3((Bpad + 127) / 128, m2.N), 128, 0, st>>>(m2, w2, V, M, B, Bpad, u);
  return cudaGetLastError();
}

cudaError_t launch_orient_to_user(const double* src2, double* out, int M, int N, int Mp2, int B, int Bpad,
                                  cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  dim3 grid((B + 31) / 32, (N + 31) / 32, M);
  orient_to_user_kernel<<<grid, dim3(32, 8), 0, st>>>(src2, out, M, N, Mp2, B, Bpad);
  return cudaGetLastError();
}

}  // namespace xbar
