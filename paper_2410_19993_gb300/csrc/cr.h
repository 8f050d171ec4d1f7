// cr.h -- state of the block-cyclic-reduction factor and substitution of one handle (cr.cu).
// Included by handle.h after the definition of Buf.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "kernels.h"

struct xbar_s;

namespace xbar {

// kept block p of a level: eliminated neighbours kl < p < kr and the kept blocks pp < p < pn of
// the next level (-1 where absent)
struct CrGthIdx {
  int p, kl, kr, pn, pp;
};

// one level of odd-even reduction: eliminated blocks (k, with kept neighbours p < k < q, q = -1
// at the end) and kept blocks
struct CrLevel {
  std::vector<int> ek, ep, eq;
  std::vector<CrGthIdx> kept;
};

enum {
  CR_OP_INIT = 0,   // level-0 blocks, weights, leakage, diagonals
  CR_OP_GJ,         // batched Gauss-Jordan inverses (off/cnt into the inverse jobs, m = size)
  CR_OP_GEMM,       // batched products (off/cnt into the GEMM jobs, m x n; aux = tensor-core tile
                    // width, 0 = CUDA cores)
  CR_OP_L0PQ,       // level-0 couplings P, Q (diagonal scalings)
  CR_OP_L0UPD,      // level-0 Schur complements and next couplings (aux = U buffer written)
  CR_OP_GTH,        // leakage and diagonals of the kept blocks (aux = U buffer of the next level)
  CR_OP_GTHS,       // diagonal of the 2 x 2 inversion's Schur complement (m = 128)
  CR_OP_L0FWD       // substitution: level-0 right-hand-side reduction
};

struct CrOp {
  int kind, off, cnt, m, n, aux;
};

struct CrSolvePlan {
  void* r = nullptr;
  void* x = nullptr;
  int Bpad = 0;
  bool initial = false, tensor = false;
  Buf jobs;
  std::vector<CrOp> ops;
};

struct CrPlanBase {
  int built = 0, factored = 0;
  int M = 0, Mp = 0, N = 0;
  bool tensor = false;
  std::vector<CrLevel> lv;
  int root = 0;
  std::vector<CrOp> ops;  // the factor
  int njobs_factor = 0;
  std::vector<CrSolvePlan> solve_cache;
};

// device arrays of one precision ([N][Mp][Mp] blocks, [N][Mp] vectors)
template <typename T>
struct CrPlan : CrPlanBase {
  Buf D, Dinv, P, Q, U[2], W, gam, om, gD;
  Buf jobs, gj, gidx, ks;
};

// arguments of one substitution (the semantics of the block-Thomas sweeps: initial mode when V is
// set, correction mode otherwise; r is overwritten)
template <typename T>
struct CrSweepArgs {
  int B, Bpad;
  const double* V;   // [B][M] initial mode, else nullptr
  const T* src;      // [Mp] initial mode: r_0 = src o V_b
  T* r;              // [N][Mp][Bpad] right-hand side (destroyed); in initial mode only column 0 is used
  T* x;              // [N][Mp][Bpad] solution
  const T* e;        // [N][Mp] word-line coupling (as factored)
  const T* hs;       // [N][Mp] current functional
  double* I;         // [B][N]
  int accumulate;    // 0: I = dI, 1: I += dI
  float* max_rel;    // max |dI|/|I| (accumulate mode) or nullptr
  bool tensor;       // products on the tensor cores (FP32)
};

// build the level plan, its job lists and buffers if the shape or product engine changed
template <typename T>
cudaError_t cr_prepare(xbar_s* h, CrPlan<T>& pl, bool tensor);
template <typename T>
cudaError_t cr_factor(xbar_s* h, CrPlan<T>& pl, bool tensor, bool equilibrate);
template <typename T>
cudaError_t cr_sweep(xbar_s* h, CrPlan<T>& pl, const CrSweepArgs<T>& a);
// release the device buffers of the cached substitution plans
void cr_clear_solve_cache(DevArena& A, CrPlanBase& pl);

}  // namespace xbar
