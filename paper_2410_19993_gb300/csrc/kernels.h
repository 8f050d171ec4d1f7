// kernels.h -- host-side declarations of the libxbar kernel launchers.
//
// Layouts (all device memory, row-major):
//   per-column vectors   [N][Mp]        element (j, i) at j*Mp + i (Mp = M padded to 16)
//   per-column matrices  [N][Mp][Mp]    block j, row i, column k at (j*Mp + i)*Mp + k
//   batch vectors        [N][Mp][Bpad]  column j, row i, input vector b at (j*Mp + i)*Bpad + b
//   user inputs          V[B][M], I[B][N], node voltages [B][M][N]
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

namespace xbar {

// Per-crossbar assembled data (device pointers, FP64 unless noted).
struct MapDev {
  int M = 0, N = 0, Mp = 0;
  double gs = 0, gw = 0, gb = 0, go = 0;
  double* Gc = nullptr;     // [N][Mp]  G transposed: Gc[j][i] = G[i][j]
  double* dW = nullptr;     // [N][Mp]  word-line row diagonal of the nodal matrix
  double* h = nullptr;      // [N][Mp]  I_j = h_j . w_j  (w_j = word-line voltages of column j)
  double* tha = nullptr;    // [N][Mp]  bit-line chain forward sweep: phi_i = tha_i w_i + thc_i phi_{i-1}
  double* thc = nullptr;    // [N][Mp]  and back sweep u_i = phi_i + thc_i u_{i+1}
  double* tdiag = nullptr;  // [N][Mp]  diagonal of the inverse bit-line chain matrix
  double* rho = nullptr;    // [N][Mp]  ratio of consecutive inverse entries along a row
  double* Coff = nullptr;   // [N][Mp][Mp] off-diagonal of the column block after bit-line elimination
  double* s_eq = nullptr;   // [N][Mp]  diagonal equilibration scale (dW^-1/2)
  double* e_eq = nullptr;   // [N][Mp]  coupling of column j to j+1, equilibrated
  double* e_pl = nullptr;   // [N][Mp]  coupling, plain (g_w)
  double* hs_eq = nullptr;  // [N][Mp]  s_eq * h
  double* src_eq = nullptr; // [Mp]     g_s * s_eq[0]
  double* src_pl = nullptr; // [Mp]     g_s
  float* s32 = nullptr;     // FP32 copies of the equilibrated vectors
  float* e32 = nullptr;
  float* hs32 = nullptr;
  float* src32 = nullptr;
  // float pairs (hi + lo, ~48 significant bits) of the coefficients the refinement's residual and
  // update use: the FP64 arithmetic of the mixed path runs on the FP32 pipe
  float2* Gc2 = nullptr;
  float2* h2 = nullptr;
  float2* tha2 = nullptr;
  float2* thc2 = nullptr;
};

// ---- assembly ---------------------------------------------------------------------------------
// Gc <- G (transposed to [N][Mp]); the rest of the assembly reads Gc only.  status != NULL: check
// G on the device (XBAR_DEV_BADINPUT for a negative or non-finite entry)
cudaError_t launch_store_g(const MapDev& m, const double* G_dev, unsigned* status, cudaStream_t st);
cudaError_t launch_assemble(const MapDev& m, cudaStream_t st);

// ---- factor -----------------------------------------------------------------------------------
template <typename T>
struct FactorParams {
  int M, Mp, N;
  double gsrc, gw;
  const double* Coff;
  const double* h;
  const double* s;    // nullptr = no equilibration
  const double* e;
  T* X;               // [N][Mp][Mp] output
  T* sig;             // [2][Mp] scratch
  T* pbuf;            // scratch: [2][PB][Mp] (factor.cu), factor_cluster_pbuf_floats (factor_cluster.cu)
  unsigned* bar;      // 2 words, zeroed
};

// One group of `blocks_per_map` co-resident blocks factors each map; `maps` is a device array.
template <typename T>
cudaError_t launch_factor(const FactorParams<T>* maps_dev, int nmaps, int Mp_max, int blocks_per_map,
                          unsigned* status, cudaStream_t st);
template <typename T>
int factor_panel_width();
template <typename T>
size_t factor_smem_bytes(int Mp, int rows_per_block);

// FP32 factor on a thread-block cluster (factor_cluster.cu): 32 <= Mp <= 256
bool factor_cluster_supported(int Mp);
int factor_cluster_size(int Mp);
size_t factor_cluster_pbuf_floats(int Mp);  // panel-slot scratch (FactorParams::pbuf) of one map
cudaError_t launch_factor_cluster(const FactorParams<float>* maps_dev, int nmaps, int Mp, unsigned* status,
                                  cudaStream_t st);

// ---- sweeps (forward + back substitution, current extraction) ---------------------------------
template <typename T>
struct SweepParams {
  int M, Mp, N, B, Bp, Bpad;
  const T* X;          // [N][Mp][Mp]
  const T* e;          // [N][Mp]
  const T* hs;         // [N][Mp]
  const T* src;        // [Mp]   initial mode: rhs_0 = src * V_b
  const double* V;     // [B][M] initial mode, else nullptr
  const T* rhs;        // [N][Mp][Bpad] correction mode, else nullptr
  T* z;                // N * Mp * Bpad scratch, layout private to each sweep kernel
  T* w;                // [N][Mp][Bpad] solution, or nullptr
  double* I;           // [B][N]
  int accumulate;      // 0: I = dI   1: I += dI
  float* max_rel;      // atomic max of |dI| / |I| (accumulate mode), or nullptr
  unsigned* status;
  const int* skip = nullptr;  // if set and nonzero at launch, the kernel does nothing
  // tensor-core sweep only: write the refinement state s32 o w as FP32 ([N][Mp][Bpad]; its
  // float-pair low part is 0) instead of w, so that the first update pass is not needed
  float* w1out = nullptr;
  const float* s32 = nullptr;  // [N][Mp]
};

template <typename T>
cudaError_t launch_sweep(const SweepParams<T>& p, cudaStream_t st);
template <typename T>
int sweep_panel_width(int Mp, int B, int nsm);

// ---- tensor-core (tcgen05, three-term BF16) FP32 sweeps: panels of 64 vectors, Mp <= 256 -----
bool sweep_tc_supported(int Mp);
int sweep_tc_rows(int Mp);  // rows of the tiled factor (128 or 256)
constexpr int kSweepTcPanel = 64;
// X (FP32 [N][Mp][Mp]) -> Xt: three-term BF16 split in the MMA's chunked core-matrix order
size_t sweep_tc_tile_bytes(int Mp, int N);
cudaError_t launch_sweep_tc_tile(const float* X, void* Xt, int Mp, int N, cudaStream_t st);
// terms = leading BF16 terms of the split used (1..3): 3 gives FP32-level accuracy
cudaError_t launch_sweep_tc(const SweepParams<float>& p, const void* Xt, int terms, cudaStream_t st);

// ---- blocking over rows (orient.cu): the mirrored crossbar M' = N, N' = M ---------------------
// Gc2[j'][i'] = Gc[N-1-i'][M-1-j'] (Gc: [N][Mp] of the original, Gc2: [M][Mp2], Mp2 >= N)
cudaError_t launch_mirror_gc(const double* Gc, int M, int Mp, int N, double* Gc2, int Mp2, cudaStream_t st);
// rhs[j'][i'][b] = V[b][M-1-j'] h2[j'][i'] ([M][Mp2][Bpad]; zero in padding rows and vectors)
cudaError_t launch_orient_rhs(const double* V, const double* h2, int M, int M2, int Mp2, int B, int Bpad,
                              double* rhs, cudaStream_t st);
// I[b][j] = gs2 w2[0][N-1-j][b]
cudaError_t launch_orient_currents(const double* w2, int N, int Bpad, int B, double gs2, double* I,
                                   cudaStream_t st);
// the mirror's bit-line voltages u ([M][Mp2][Bpad]) from its word-line voltages w2 and the sources
cudaError_t launch_orient_blvolt(const MapDev& m2, const double* w2, const double* V, int M, int B, int Bpad,
                                 double* u, cudaStream_t st);
// mixed precision: equilibrated FP32 right-hand side s o (V h'), currents from the float-pair
// state, and the correction's current change (I += dI, max |dI| / |I| into max_rel)
cudaError_t launch_orient_rhs32(const double* V, const double* h2, const float* s32, int M, int M2, int Mp2, int B,
                                int Bpad, float* rhs, cudaStream_t st);
cudaError_t launch_orient_state_currents(const float2* w2, const float* w1, int N, int Bpad, int B, double gs2,
                                         double* I, cudaStream_t st);
cudaError_t launch_orient_correction_currents(const float* dhat, const float* s32, int N, int Bpad, int B,
                                              double gs2, double* I, float* max_rel, unsigned* status,
                                              cudaStream_t st);
// out[b][i][j] = src2[M-1-i][N-1-j][b]
cudaError_t launch_orient_to_user(const double* src2, double* out, int M, int N, int Mp2, int B, int Bpad,
                                  cudaStream_t st);

// ---- transfer-matrix mode (transfer.cu) -------------------------------------------------------
cudaError_t launch_eye(double* E, int M, cudaStream_t st);  // E = I (M x M, FP64)
// C[R x N] = A[R x K] . B[K x N], FP64, row-major
cudaError_t launch_gemm_f64(const double* A, const double* B, double* C, int R, int K, int N, cudaStream_t st);

// ---- BF16 tensor-core GEMM (gemm_bf16.cu): C[m][n] = sum_k A(m,k) B(n,k) ---------------------
enum { GEMM_EPI_STORE = 0, GEMM_EPI_BIAS_RELU = 1, GEMM_EPI_MASK = 2 };
struct GemmBf16Params {
  int M, N, K;                          // multiples of 128, 128, 64
  const struct __nv_bfloat16* A;        // A(m,k) = A[m*sAm + k*sAk]   (sAk == 1 or sAm == 1)
  long sAm, sAk;
  const struct __nv_bfloat16* B;        // B(n,k) = B[n*sBn + k*sBk]   (sBk == 1 or sBn == 1)
  long sBn, sBk;
  int mode;                             // GEMM_EPI_*
  float* C;                             // EPI_STORE: C[m*ldc + n] (= or atomically +=)
  long ldc;
  int atomic;
  const float* bias;                    // EPI_BIAS_RELU: out = relu(C + bias[n])
  const struct __nv_bfloat16* mask;     // EPI_MASK: out = mask > 0 ? C : 0
  long ldm;
  struct __nv_bfloat16* out;            // BF16 output of EPI_BIAS_RELU / EPI_MASK
  long ldo;
  unsigned* status;
};
// ksplit > 1 splits K over blocks and requires EPI_STORE with atomic = 1 (C zeroed by the caller)
cudaError_t launch_gemm_bf16(const GemmBf16Params& p, int ksplit, cudaStream_t st);

// ---- surrogate prediction: second and output layers fused with the result (surrogate_infer.cu) ---
struct SurInferParams {
  long rows;                        // B * N rows, row r = b*N + j
  int N;
  const float* P;                   // [>= N][256]  per-column part of the first layer
  const float* Q;                   // [>= B][256]  per-vector part of the first layer
  const float* b1;                  // [256]
  const struct __nv_bfloat16* W2;   // [256][256] (output unit, input unit) in the kernel's B-operand
                                    // layout (launch_surrogate_w2_tile)
  const float* b2;                  // [256]
  const float* W3;                  // [2][256]
  const float* b3;                  // [2]
  const double* Iid;                // [rows] ideal currents
  const double* Iln;                // [rows] line-model currents
  double mu, sigma, cal, bound;
  double* I;                        // [rows] prediction
  double* est;                      // [rows] relative error estimate (may be NULL)
  int* flag;                        // [B] set to 1 where an estimate exceeds bound (may be NULL)
  unsigned* status;
};
cudaError_t launch_surrogate_infer(const SurInferParams& p, int nsm, cudaStream_t st);
// W2 (BF16 [256][256], row = output unit) -> W2t (128 KB) in the layout launch_surrogate_infer reads
cudaError_t launch_surrogate_w2_tile(const struct __nv_bfloat16* W2, void* W2t, cudaStream_t st);

// ---- batched GEMM job lists (gemm_jobs.cu, gemm_jobs_tc.cu) -----------------------------------
// One job: C = Cin + alpha * sum_s op(A_s) op(B_s)   (Cin may be NULL: then C = alpha * sum; Cin
// may equal C).  op(A_s) is m x k_s: ta = 0 reads A_s[i * lda + kk], ta = 1 reads A_s[kk * lda + i];
// op(B_s) is k_s x n: tb = 0 reads B_s[kk * ldb + j], tb = 1 reads B_s[j * ldb + kk].  All jobs of
// one launch share m and n; each is cut into row x column tiles of the kernel's tile shape.
template <typename T>
struct GemmJob {
  T* C;
  const T* Cin;
  int ldc, ldcin;
  int nseg;
  T alpha;
  const T* A[3];
  const T* B[3];
  int lda[3], ldb[3], k[3];
  int ta[3], tb[3];
};
// CUDA cores (FP32 or FP64), 64 x 64 output tiles
template <typename T>
cudaError_t launch_gemm_jobs(const GemmJob<T>* jobs_dev, int njobs, int m, int n, unsigned* status, cudaStream_t st);
// tensor cores (tcgen05, FP32 operands split into three BF16 terms, six products per K step, FP32
// accumulation in tensor memory), 128 x TN output tiles with TN = 128 or 256, persistent over the
// SMs.  k_s must be multiples of 16.
cudaError_t launch_gemm_jobs_tc(const GemmJob<float>* jobs_dev, int njobs, int m, int n, int tn, int nsm,
                                unsigned* status, cudaStream_t st);

// In-place Gauss-Jordan inversion (no pivoting) of symmetric M-matrices, one block per matrix:
// dst = src^-1 (n x n, n <= 128; src may equal dst)
template <typename T>
struct GjJob {
  const T* src;
  T* dst;
  int lds, ldd;
};
template <typename T>
cudaError_t launch_gj_inverse(const GjJob<T>* jobs_dev, int njobs, int n, unsigned* status, cudaStream_t st);

// ---- block cyclic reduction over the columns (cr.cu) ------------------------------------------
bool cr_supported(int Mp, int N);

// ---- FP64 refinement kernels and node voltages ------------------------------------------------
struct ResidParams {
  int M, Mp, N, B, Bpad;
  double gs, gw;
  double gb, go;        // bit-line segment and sense conductances (bit-line sources only)
  const double* Gc;
  const double* dW;
  const double* h;
  const double* tha;
  const double* thc;
  const float* s32;
  const double* V;      // [B][M]
  double* w;            // [N][Mp][Bpad] FP64 word-line voltages (state)
  const float* dhat;    // [N][Mp][Bpad] scaled correction from the FP32 sweep
  double* phi;          // [N][Mp][Bpad] scratch
  float* rhat;          // [N][Mp][Bpad] scaled residual for the next FP32 sweep
  double* I;            // [B][N]
  unsigned long long* rmax;  // bit pattern of max |r| (non-negative double)
  unsigned* status;
  const int* skip;           // if set and nonzero at launch, the kernel does nothing
  // mixed path: the state w and the scratch phi as float pairs (in the w / phi buffers)
  float2* w2;
  float2* phi2;
  const float2* Gc2;
  const float2* h2;
  const float2* tha2;
  const float2* thc2;
  // the refinement state as FP32 (low part 0, as the initial tensor-core sweep writes it) instead
  // of w2, for the first residual and the first update (which writes w2); nullptr: w2
  const float* w1;
  // sources on the bit-line chains instead (the mirrored crossbar of orient.cu): the word-line
  // source potential is 0 (V unused) and the bottom node of bit line j is driven through g_o by
  // Vbl[b][N-1-j] ([B][N]); nullptr: the usual sources V on the word lines
  const double* Vbl;
};
// w = (first ? 0 : w) + s * dhat ; I = h . w    (float-pair state w2)
cudaError_t launch_update(const ResidParams& p, int first, cudaStream_t st);
// w2 (float pairs) -> w (double), in place: the node-voltage output reads doubles
cudaError_t launch_pair_to_double(const ResidParams& p, cudaStream_t st);
// rhat = s * (b - K w)   with K the word-line system after bit-line elimination
cudaError_t launch_resid(const ResidParams& p, cudaStream_t st);
// bit-line voltages u = T^-1 (G o w) into `u` ([N][Mp][Bpad]), in place of phi
cudaError_t launch_blvolt(const ResidParams& p, double* u, cudaStream_t st);
// out[b][i][j] = src[(j*Mp + i)*Bpad + b]
cudaError_t launch_to_user_layout(const double* src, double* out, int M, int Mp, int N, int B, int Bpad,
                                  cudaStream_t st);
// device-driven refinement control (one thread): reset the state / apply the stopping rule to the
// correction just computed (state->maxrel, state->rmax), set state->done, and re-arm the
// accumulators for the next pass
struct IrState;
cudaError_t launch_ir_init(IrState* state, cudaStream_t st);
cudaError_t launch_ir_check(IrState* state, double tol, cudaStream_t st);
// FP64 -> FP32 copy
cudaError_t launch_d2f(const double* a, float* b, size_t n, cudaStream_t st);

}  // namespace xbar
