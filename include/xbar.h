/*
 * xbar.h -- C ABI of libxbar, a GB300 (sm_103a) solver for the DC nodal
 * equations of memristive crossbars with interconnect parasitics, after
 * XbarSim (Kolinko, Amin, Zand, Bakos, arXiv 2410.19993).
 *
 * Problem (Sec. II "Methodology", Sec. II-A "Circuit Model", Eqs. 1-7): an
 * M x N crossbar has M word lines (rows i) and N bit lines (columns j), a
 * memristor of conductance G_ij at every crossing, and wire resistors between
 * neighbouring devices.  Source V_i drives word line i at its first column
 * through R_s; the far end of every word line is open (Eq. 2); the top of every
 * bit line is open (Eq. 3); the bottom of bit line j is tied to ground through
 * R_sense, and the current through that termination is output I_j.  Word-line
 * segments are R_w, bit-line segments R_b.  With R_s = R_w and R_sense = R_b
 * this is exactly the paper's circuit (its Eq. 5 uses G_WL for the source
 * segment).  Nodal analysis gives a symmetric 2MN x 2MN system G v = i.
 *
 * Method (Sec. II-C, Sec. III-A): decompose the nodal matrix once per
 * conductance map, then run forward/back substitution for every input vector
 * of a batch.  libxbar eliminates each bit line's tridiagonal chain inside its
 * column, which leaves a block-tridiagonal system over the N columns with
 * dense M x M blocks, and factors that with block Thomas; the substitutions
 * become chains of dense products streamed over panels of input vectors.
 *
 * Conventions
 *   - Pointers may be host or device memory.  The library asks the CUDA
 *     runtime which one each pointer is.  Device buffers are used in place;
 *     host buffers are staged through library-owned device memory with copies
 *     on the handle's stream, and such calls return only once the stream has
 *     drained.  With all-device buffers the work is asynchronous on the
 *     handle's stream; results are valid once the caller synchronises it.
 *   - Matrices are row-major and dense: G is M x N (G[i*N + j] is the device
 *     at word line i, bit line j); V is B x M (row b is one input vector, in
 *     volts); I is B x N (amperes); node voltages are B x M x N.
 *   - Every call returns an xbar_status; none exits or throws.  On failure
 *     xbar_last_error() returns a message for the calling thread.
 *   - Handles share no state: different handles may be used at the same time
 *     from different host threads, and their work may overlap on the GPU when
 *     they run on different streams (for example, factoring the next
 *     conductance map while another handle solves).  One handle must not be
 *     used from two threads at once.
 *   - Errors detected on the device (a bounded wait that timed out, a
 *     non-finite value) are recorded in a device status word and reported by
 *     the next call that synchronises (xbar_solve always does when it
 *     iterates; xbar_sync does on request).
 */
#ifndef XBAR_H
#define XBAR_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xbar_s* xbar_t;
typedef struct xbar_batch_s* xbar_batch_t;

typedef enum {
  XBAR_OK = 0,
  XBAR_EINVAL = 1,    /* invalid argument (size, resistance, conductance, pointer, precision) */
  XBAR_ENOMEM = 2,    /* device or host allocation failed */
  XBAR_ECUDA = 3,     /* CUDA runtime error */
  XBAR_ESTATE = 4,    /* call out of order, e.g. solve before factor */
  XBAR_ENOTCONV = 5,  /* iterative refinement did not reach tol within max_iter */
  XBAR_ETIMEOUT = 6   /* a bounded device-side wait expired; the kernel returned early */
} xbar_status;

typedef enum {
  /* Plain FP64: factor and substitutions in double precision, no refinement. */
  XBAR_FP64 = 0,
  /* Mixed: diagonal equilibration, FP32 factor and FP32 substitutions, then
   * iterative refinement whose residual r = b - A x and solution update are
   * computed in float pairs (hi + lo, ~48 significant bits) on the FP32 pipe. */
  XBAR_FP32_IR = 1
} xbar_precision;

typedef struct {
  int iters;          /* refinement corrections applied (0 for XBAR_FP64) */
  double max_rel_dI;  /* max over (b, j) of |dI| / |I| of the last correction */
  double resid_inf;   /* max |r| of the last refinement residual, in amperes (0 for XBAR_FP64) */
  double err_est;     /* estimated max relative current error of the result */
  int n_fallback;     /* xbar_surrogate_solve: vectors solved exactly (0 elsewhere) */
} xbar_solve_info;

/*
 * xbar_assemble -- build the nodal system of one crossbar (Sec. II-A,
 * Eqs. 1-7) and create a handle for it.
 *   M, N          word lines and bit lines, 1 <= M <= 1024, N >= 1.
 *   G             M x N conductances in siemens, finite and >= 0 (host or
 *                 device; copied, so the caller may free it on return).
 *   R_s, R_w, R_b, R_sense   source, word-line segment, bit-line segment and
 *                 sense resistances in ohms, finite and > 0.
 *   cuda_stream   cudaStream_t all work of this handle runs on (NULL = legacy
 *                 default stream).
 *   out           receives the handle; owns all device memory it allocates.
 * The conductances are stored at once; the per-column elimination data (bit-line
 * chain pivots, the blocks C_j of xbar_factor) are formed by the first
 * xbar_factor, so callers that only need the map (xbar_surrogate_solve) skip them.
 * Errors: XBAR_EINVAL for out-of-range sizes, non-positive or non-finite
 * resistances, negative or non-finite conductances (checked on the host after
 * copying G), or NULL pointers; XBAR_ENOMEM; XBAR_ECUDA.
 */
xbar_status xbar_assemble(int M, int N, const double* G, double R_s, double R_w, double R_b,
                          double R_sense, void* cuda_stream, xbar_t* out);

/*
 * xbar_factor -- decompose the assembled system once (Sec. II-C, LU of the
 * nodal matrix; Sec. III-A, one decomposition per batch).  Block Thomas over
 * the N columns: for each column j the M x M Schur complement
 *   Z_j = C_j - g_w^2 X_{j-1},   X_j = Z_j^{-1},
 * where C_j is the column's word-line block after its bit-line chain is
 * eliminated.  Diagonals are formed without subtraction from the grounded
 * row sums, so the factor keeps high relative accuracy in FP32.
 * The factor (N x M x M values) is stored in the handle.  Calling it again
 * re-factors (e.g. with another precision).
 * Errors: XBAR_EINVAL (bad handle or precision), XBAR_ENOMEM, XBAR_ECUDA,
 * XBAR_ETIMEOUT (a cross-block wait of the cooperative factor kernel expired).
 */
xbar_status xbar_factor(xbar_t h, xbar_precision p);

/*
 * xbar_solve -- substitute a batch of input vectors (Sec. II-C forward/back
 * substitution; Sec. III-A batch processing) and extract outputs.
 *   B          number of input vectors, >= 0 (B = 0 is a no-op).
 *   V          B x M input voltages (host or device).
 *   I          B x N bit-line termination currents (output, host or device).
 *   vWL, vBL   B x M x N word-line / bit-line node voltages (outputs, may be
 *              NULL; host or device).
 *   tol        XBAR_FP32_IR only: target max relative current error (e.g.
 *              1e-8).  Refinement stops after the correction k whose
 *              max |dI|/|I| (call it d_k) is <= tol, or, from the second
 *              correction on, when the observed contraction rho = d_k/d_{k-1}
 *              is <= 1/2 and d_k rho / (1 - rho) <= tol (the error left after
 *              applying correction k under linear convergence).  Ignored for
 *              XBAR_FP64.
 *   max_iter   XBAR_FP32_IR only: most corrections to apply (>= 1).
 *   info       optional diagnostics (may be NULL).
 * Errors: XBAR_ESTATE if not factored; XBAR_EINVAL for B < 0, NULL V or I, or
 * max_iter < 1 in mixed mode; XBAR_ENOTCONV if refinement did not reach tol
 * (outputs then hold the last iterate); XBAR_ENOMEM; XBAR_ECUDA.
 */
xbar_status xbar_solve(xbar_t h, int B, const double* V, double* I, double* vWL, double* vBL,
                       double tol, int max_iter, xbar_solve_info* info);

/* Kernel-variant options of a handle (value -1 = automatic choice). */
typedef enum {
  XBAR_OPT_SWEEP_KERNEL = 0,  /* FP32 substitutions: 0 = CUDA-core kernel, 1 = tensor-core kernel */
  XBAR_OPT_FACTOR_KERNEL = 1, /* FP32 factor: 0 = cooperative-group kernel, 1 = cluster kernel */
  XBAR_OPT_ALGORITHM = 2,     /* factor + substitution: 0 = block Thomas over the columns (N
                                 dependent block steps), 1 = block cyclic reduction over the
                                 columns (ceil(log2 N) levels of independent dense block products;
                                 M <= 256).  Takes effect at the next xbar_factor. */
  XBAR_OPT_CR_PRODUCTS = 3,   /* cyclic reduction in XBAR_FP32_IR: 0 = products on the CUDA
                                 cores, 1 = on the tensor cores (three-term BF16 split; M >= 128) */
  XBAR_OPT_WAIT_LIMIT_NS = 4, /* limit of every bounded device-side wait of this handle's
                                 kernels, in ns (value > 0); -1 or 0 restores the default of 2 s.
                                 A wait that runs out makes its kernel record a timeout and
                                 return; the next call that reads the handle's device status
                                 returns XBAR_ETIMEOUT and the results of that work are invalid.
                                 Synchronises the handle's stream. */
  XBAR_OPT_ORIENTATION = 5,   /* XBAR_FP64 factors: 0 = blocks over the N columns (M x M blocks,
                                 bit lines eliminated inside each column; Sec. II-B ordering),
                                 1 = blocks over the M rows (N x N blocks, word lines eliminated
                                 inside each row: the same system written for the mirrored
                                 crossbar M' = N, N' = M with R_s and R_sense, R_w and R_b
                                 exchanged; needs N <= 1024), -1 (default) = rows when 2N <= M.
                                 Blocked over rows with XBAR_OPT_ALGORITHM left at -1, the factor
                                 is block cyclic reduction when N <= 256 (its M small blocks are
                                 what cyclic reduction is for), else block Thomas.
                                 Results are the same up to rounding; the cost of the factor
                                 scales as N M^3 or M N^3 and of a substitution as N M^2 or M N^2.
                                 XBAR_FP32_IR factors block over rows only when this option is 1
                                 (the refinement then runs on the mirrored crossbar); the tile
                                 batch (xbar_batch_run) blocks over rows in XBAR_FP64 only.  Takes
                                 effect at the next xbar_factor. */
  XBAR_OPT_EAGER_ASSEMBLY = 6 /* 1 = xbar_set_conductances also forms the column elimination data
                                 (Sec. II-A), on the handle's stream, so that a factor queued
                                 behind it starts at once (a caller pipelining maps over two
                                 streams records an event after the call); 0 or -1 (default) =
                                 the next xbar_factor forms them, and callers that need only the
                                 map (the surrogate) never pay for them. */
} xbar_option;

/* Select a kernel variant for later xbar_factor / xbar_solve calls (value -1, 0 or 1; a
 * variant that does not support the handle's size falls back to the other), or set the wait
 * limit (XBAR_OPT_WAIT_LIMIT_NS).  Errors: XBAR_EINVAL, XBAR_ECUDA. */
xbar_status xbar_set_option(xbar_t h, xbar_option opt, int value);

/*
 * xbar_set_conductances -- load a new conductance map G into the handle (same
 * M, N and resistances; host or device pointer) without reallocating.  The
 * handle becomes unfactored; as after xbar_assemble, the column elimination data
 * are formed by the next xbar_factor, or here, asynchronously on the handle's
 * stream, when XBAR_OPT_EAGER_ASSEMBLY is 1.  A host G is validated before the
 * call returns.  A device G is read and validated on the device, asynchronously
 * on the handle's stream (the call does not wait for that stream): a negative or
 * non-finite entry is reported as XBAR_EINVAL by the next call that reads the
 * handle's device status (xbar_sync, an XBAR_FP32_IR xbar_solve, a solve with
 * host buffers), and results computed from such a map are meaningless.
 * Errors: XBAR_EINVAL (NULL handle/G, negative or non-finite host G), XBAR_ECUDA.
 */
xbar_status xbar_set_conductances(xbar_t h, const double* G);

/* Per-phase device time of one handle, from CUDA events recorded on its stream
 * around every kernel launch while profiling is enabled. */
typedef enum {
  XBAR_PHASE_ASSEMBLE = 0,  /* nodal assembly kernels */
  XBAR_PHASE_FACTOR = 1,    /* block Thomas factor kernel */
  XBAR_PHASE_SWEEP = 2,     /* forward/back substitution + current extraction */
  XBAR_PHASE_RESID = 3,     /* residual of refinement (float pairs) */
  XBAR_PHASE_UPDATE = 4,    /* solution update of refinement (float pairs) */
  XBAR_PHASE_OUTPUT = 5,    /* node-voltage extraction and layout */
  XBAR_NPHASES = 6
} xbar_phase;

typedef struct {
  int launches[XBAR_NPHASES];   /* kernel launches per phase */
  double ms[XBAR_NPHASES];      /* summed device milliseconds per phase */
} xbar_profile;

/* Enable (1) or disable (0) event timing on the handle; enabling resets it. */
xbar_status xbar_profile_enable(xbar_t h, int enable);
/* Synchronise the stream and return the accumulated per-phase times
 * (out may not be NULL); reset != 0 clears the accumulators afterwards. */
xbar_status xbar_profile_read(xbar_t h, xbar_profile* out, int reset);

/*
 * xbar_solve_noalloc -- the substitution of xbar_solve for a handle factored
 * with XBAR_FP64, for callers that must not allocate device memory while they
 * solve (for example a latency-critical loop in which cudaMalloc/cudaFree
 * could implicitly synchronise the device, or a process whose device memory is
 * owned by a framework allocator that forbids allocations outside its pool).
 * The paper has no counterpart: this is a memory-management variant only.
 *   B   number of input vectors, >= 0.
 *   V   B x M input voltages, device memory.
 *   I   B x N bit-line currents (output), device memory.
 * The kernel's scratch (N x Mp x Bpad doubles, Mp = M rounded up to 16, Bpad
 * = B rounded up to the kernel's panel width) lives in a fixed 64 MiB device
 * array inside libxbar that every GPU loading the library keeps until exit;
 * larger requests fail with XBAR_EINVAL and a message giving the sizes.
 * Nothing is allocated or freed.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.  The address is kept for the life of the process: after
 * cudaDeviceReset (or anything else that replaces the device's primary context)
 * the entry point must not be used again in that process.  All calls share the
 * array, so calls whose work overlaps on the GPU race on it.  Work is
 * asynchronous on the handle's stream.
 * Errors: XBAR_ESTATE (not factored with XBAR_FP64 by block Thomas), XBAR_EINVAL
 * (NULL or host pointers, B < 0, scratch too large), XBAR_ECUDA.
 */
xbar_status xbar_solve_noalloc(xbar_t h, int B, const double* V, double* I);

/*
 * Transfer-matrix (currents-only) mode.  The nodal system of Sec. II (Eqs. 1-7)
 * is linear in the word-line source voltages, so the bit-line currents of any
 * input vector are I = V G_eff with the M x N transfer matrix
 * G_eff[i][j] = dI_j / dV_i (the currents for a unit voltage on word line i
 * alone).  This mode answers currents only (no node voltages) and is a
 * different path from the substitutions: it is reported separately.
 *
 * xbar_transfer_matrix -- G_eff of the handle's current factorization, from M
 * unit-input solves through xbar_solve (same precision, tol and max_iter
 * meaning; for XBAR_FP32_IR each entry then carries the certified relative
 * error of a current).  It is kept in the handle until the next xbar_factor or
 * xbar_set_conductances; a call while it is valid does no solves.
 *   Geff  optional M x N row-major copy (device or host memory; NULL: none).
 *   info  optional: the unit solves' refinement summary (zeros when cached).
 * Synchronises the handle's stream.  Errors: XBAR_EINVAL (NULL handle),
 * XBAR_ESTATE (not factored), the errors of xbar_solve, XBAR_ECUDA.
 *
 * xbar_solve_transfer -- I = V G_eff for B input vectors: one FP64 matrix
 * product (2 M N flops per vector), accumulated over the word lines in order.
 * For non-negative V every term is non-negative (the inverse of the nodal
 * matrix is entrywise positive), so the relative error of each current is at
 * most that of the G_eff entries plus FP64 rounding; for signed inputs the
 * bound is relative to sum_i |V_i| G_eff[i][j].
 *   B  number of input vectors, >= 0.   V  B x M (device or host memory).
 *   I  B x N output (device or host memory).
 * Asynchronous on the handle's stream for device pointers; host pointers are
 * staged and the call synchronises.  Errors: XBAR_EINVAL (NULL handle, V or I;
 * B < 0), XBAR_ESTATE (no valid G_eff: call xbar_transfer_matrix after the
 * last xbar_factor), XBAR_ECUDA.
 */
xbar_status xbar_transfer_matrix(xbar_t h, double tol, int max_iter, double* Geff, xbar_solve_info* info);
xbar_status xbar_solve_transfer(xbar_t h, int B, const double* V, double* I);

/* ---------------------------------------------------------------------------------------------
 * Batches of tiles: many crossbars of uneven sizes, such as the tiles a network layer is mapped
 * onto or the parts of a large crossbar split as in Sec. III-C ("Partitioning"), factored and
 * solved with their input batches by one CUDA-graph launch.
 * ------------------------------------------------------------------------------------------- */
typedef struct {
  int M, N;           /* tile size (word lines, bit lines), as in xbar_assemble */
  const double* G;    /* M x N conductances (host or device; copied) */
  double R_s, R_w, R_b, R_sense;
} xbar_tile;

/* Assemble T tiles; each tile gets its own stream.  Runs start after the work already queued on
 * `cuda_stream` (NULL = legacy default stream) and return when finished.
 * Errors: as xbar_assemble, for the first failing tile. */
xbar_status xbar_batch_create(int T, const xbar_tile* tiles, void* cuda_stream, xbar_batch_t* out);

/*
 * xbar_batch_run -- factor every tile with precision p (Sec. II-C: one decomposition per map)
 * and substitute its batch (Sec. III-A), all as one CUDA-graph launch.
 *   B[t]       input vectors of tile t (>= 0)
 *   V[t]       B[t] x M_t input voltages, DEVICE memory
 *   I[t]       B[t] x N_t bit-line currents (output), DEVICE memory
 *   tol, max_iter   as xbar_solve; refinement runs exactly max_iter passes per tile, and the
 *              passes after a tile has converged (same stopping rule as xbar_solve) skip their
 *              work on the device.
 *   infos      optional, T entries.
 * The first run with a given (p, B, V, I, tol, max_iter) executes once eagerly (sizing every
 * workspace) and captures the graph; later runs with the same signature replay it.  Returns
 * after the graph has completed.  Errors: XBAR_EINVAL (NULL or host pointers, B < 0, bad
 * precision), XBAR_ENOTCONV (some tile did not converge; infos say which), XBAR_ETIMEOUT,
 * XBAR_ECUDA, XBAR_ENOMEM.
 */
xbar_status xbar_batch_run(xbar_batch_t b, xbar_precision p, const int* B, const double* const* V,
                           double* const* I, double tol, int max_iter, xbar_solve_info* infos);

/*
 * xbar_batch_autotune -- for every distinct (M, N, B[t]) time the kernel variants (tensor-core
 * vs CUDA-core FP32 substitutions, cluster vs cooperative-group FP32 factor) on one tile, keep
 * the fastest for all tiles of that shape.  cache_path (may be NULL) is a JSON file of earlier
 * choices, read first and rewritten with new ones.  Only XBAR_FP32_IR has variants.
 */
xbar_status xbar_batch_autotune(xbar_batch_t b, xbar_precision p, const int* B, const char* cache_path);

/* The handle of tile t (owned by the batch: do not destroy it). */
xbar_status xbar_batch_tile(xbar_batch_t b, int t, xbar_t* out);

/* Release the batch, its tiles, streams and graph.  NULL is accepted. */
xbar_status xbar_batch_destroy(xbar_batch_t b);

/* ---------------------------------------------------------------------------------------------
 * Learned surrogate of the column currents, with the exact solver as fallback and judge.
 *
 * The paper's closing section proposes driving whole neural-network simulations with the solver;
 * at that scale most input vectors need only a close estimate.  Two stages:
 *   line model: every word line solved alone with the bit lines at ground, then every bit line
 *     solved alone with its devices driven by those word-line voltages; each further pass
 *     solves the word lines again with their devices tied to the latest bit-line voltages, then
 *     the bit lines again (block Gauss-Seidel between the two sets of lines, which converges to
 *     the exact solution).  Linear in V: I_line = V T_line, T_line found per map from the M unit
 *     inputs in O(passes M^2 N).  One pass: T_line(i, j) = tau(i, j) G(i, j) g_o x_j(i) with tau
 *     the word-line voltage ratios and x_j bit line j's response to a unit bottom current.
 *   network: for bit line j it reads 3M features
 *     x = [ G(:,j) / g_scale,  V / v_scale,  S(:,j) / (N g_scale) ],  S(i, j) = sum_{l>=j} G(i, l)
 *     (3M -> 256 -> 256 -> 2, ReLU, BF16 weights and activations, FP32 accumulation) with outputs
 *     (n0, n1), trained on the line model's error relative to the ideal MVM, standardised:
 *       q = (I_j - I_line,j) / I_ideal,j,  I_ideal,j = sum_i V_i G_ij,  qh = (q - mu) / sigma;
 *       n0 ~ qh,   n1 ~ log |n0 - qh|  (the network's own error).
 * Prediction: I_j = I_line,j + I_ideal,j (mu + sigma n0); its deviation from the ideal MVM is
 * (I_line,j - I_ideal,j)/I_ideal,j + mu + sigma n0.  Relative error estimate
 * c sigma exp(n1) |I_ideal,j| / |I_j| with c from calibration.
 * Training loss per row: (n0 - qh)^2 + 0.1 (n1 - log(|n0 - qh| + 1e-6))^2 (the log target is
 * held constant), mean over the rows of a minibatch, Adam (beta 0.9 / 0.999, eps 1e-8) on FP32
 * master weights.  Flat parameter order: W1 [256][Fp] (Fp = 3M rounded up to 128; padding
 * columns zero), b1 [256], W2 [256][256], b2 [256], W3 [2][256], b3 [2]; W[o][i] maps input i to
 * output o.
 * ------------------------------------------------------------------------------------------- */
typedef struct xbar_surrogate_s* xbar_surrogate_t;

/* Create a surrogate for M x N maps (1 <= M <= 1024) of the circuit (R_s, R_w, R_b, R_sense, as
 * in xbar_assemble) whose line model runs line_passes passes (1..64), with He-initialised
 * weights from `seed`.  g_scale, v_scale > 0 normalise conductances and voltages.  Work is queued
 * on `cuda_stream` (NULL = legacy default stream).  Errors: XBAR_EINVAL, XBAR_ENOMEM, XBAR_ECUDA. */
xbar_status xbar_surrogate_create(int M, int N, double R_s, double R_w, double R_b, double R_sense,
                                  int line_passes, double g_scale, double v_scale, unsigned seed,
                                  void* cuda_stream, xbar_surrogate_t* out);

/* Read (get != NULL) and/or replace (set != NULL) the flat FP32 parameters (host or device);
 * *count (may be NULL) receives their number.  `set` is applied before `get`. */
xbar_status xbar_surrogate_params(xbar_surrogate_t s, float* get, const float* set, int* count);

/* Read (get != NULL) and/or replace (set != NULL; applied first) the three scalars around the
 * network: {mu, sigma, c}.  The target is standardised as (y - mu) / sigma; mu and sigma are set
 * from the targets of the first xbar_surrogate_train call unless set here first (default 0, 1);
 * c is the calibrated error-estimate scale (default 1).  Errors: XBAR_EINVAL (sigma or c <= 0). */
xbar_status xbar_surrogate_scaling(xbar_surrogate_t s, const double* set, double* get);

/* Loss and gradient of one minibatch without updating: X is R x 3M FP32 features (host or
 * device, row-major), y R raw targets q (standardised inside with mu, sigma).
 * loss[0] = mean (n0 - qh)^2, loss[1] = mean (n1 - t)^2;
 * grad (may be NULL) receives the gradient of loss[0] + 0.1 loss[1] in the flat order.  The
 * network computes in BF16 exactly as in training. */
xbar_status xbar_surrogate_grad(xbar_surrogate_t s, int R, const float* X, const float* y, double* loss,
                                float* grad);

/* Train on n_maps maps: G[m] (M x N), V[m] (B[m] x M) and the exact currents I[m] (B[m] x N)
 * (host or device).  Rows are shuffled in minibatches of batch_rows (a multiple of 128) each
 * epoch; loss_per_epoch (may be NULL, 2*epochs) receives the two mean losses of each epoch. */
xbar_status xbar_surrogate_train(xbar_surrogate_t s, int n_maps, const double* const* G, const int* B,
                                 const double* const* V, const double* const* I, int epochs, int batch_rows,
                                 double lr, unsigned seed, double* loss_per_epoch);

/* Set the error-estimate scale c so that the given quantile (0 < q <= 1) of |I_pred - I| / |I|
 * over held-out maps lies at or below c exp(out1).  *scale_out (may be NULL) receives c. */
xbar_status xbar_surrogate_calibrate(xbar_surrogate_t s, int n_maps, const double* const* G, const int* B,
                                     const double* const* V, const double* const* I, double quantile,
                                     double* scale_out);

/* Predict the B x N currents of map G for inputs V (B x M); err_est (may be NULL) receives the
 * relative error estimates.  Host or device pointers; returns when the results are written. */
xbar_status xbar_surrogate_predict(xbar_surrogate_t s, const double* G, int B, const double* V, double* I,
                                   double* err_est);

/* Predict for the map held by `exact` (an assembled handle of the same M, N and circuit) and replace every
 * input vector with an error estimate above `bound` by the exact solution (xbar_solve with
 * XBAR_FP32_IR, tol 1e-8; the handle is factored on first need).  V, I, err_est: DEVICE memory.
 * info->n_fallback counts the vectors solved exactly; the other fields describe that solve. */
xbar_status xbar_surrogate_solve(xbar_surrogate_t s, xbar_t exact, int B, const double* V, double* I,
                                 double bound, double* err_est, xbar_solve_info* info);

/* Release the surrogate.  NULL is accepted. */
xbar_status xbar_surrogate_destroy(xbar_surrogate_t s);

/* Wait for the handle's stream and report any device-recorded error. */
xbar_status xbar_sync(xbar_t h);

/* Release the handle and all memory it owns.  NULL is accepted. */
xbar_status xbar_destroy(xbar_t h);

/* Message describing the last failure on the calling thread ("" if none). */
const char* xbar_last_error(void);

/* Library version string. */
const char* xbar_version(void);

#ifdef __cplusplus
}
#endif
#endif /* XBAR_H */
