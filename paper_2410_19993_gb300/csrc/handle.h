// handle.h -- internal state of a libxbar handle (shared by api.cu and batch.cu).
#pragma once
#include <cuda_runtime.h>
#include <string.h>

#include <utility>
#include <vector>

#include "kernels.h"
#include "xbar.h"

namespace xbar {
// device allocation owned by a handle; freed in reverse order on destroy
// Allocation-failure injection for tests (host side only): with XBAR_FAIL_ALLOC_AFTER=n in the
// environment, the allocations through any DevArena after the first n (counted from the moment
// the variable took its current value) fail with cudaErrorMemoryAllocation without calling
// cudaMalloc.  Unset, it costs one getenv per allocation.
bool alloc_injected_failure();

struct DevArena {
  std::vector<void*> ptrs;
  cudaError_t alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (alloc_injected_failure()) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
  void release(void* p) {
    for (size_t k = 0; k < ptrs.size(); ++k)
      if (ptrs[k] == p) {
        cudaFree(p);
        ptrs.erase(ptrs.begin() + k);
        return;
      }
  }
  void free_all() {
    for (size_t k = ptrs.size(); k-- > 0;) cudaFree(ptrs[k]);
    ptrs.clear();
  }
};

inline bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// growable device buffer
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

inline cudaError_t ensure(DevArena& A, Buf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return cudaSuccess;
  if (b.p) A.release(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = A.alloc(&b.p, bytes);
  if (e == cudaSuccess) b.bytes = bytes;
  return e;
}

inline int round_up(int a, int m) { return ((a + m - 1) / m) * m; }

}  // namespace xbar

#include "cr.h"

namespace xbar {


// per-handle refinement state on the device (graph-driven solves)
struct IrState {
  int done;        // 1 once converged (later passes skip)
  int iters;       // corrections applied
  float last, prev;  // max |dI|/|I| of the last two corrections
  float maxrel;    // written by the correction sweep
  float pad;
  unsigned long long rmax;  // bit pattern of max |r| of the last residual
  double rinf;
};

}  // namespace xbar

// kernel-variant options of a handle (-1 = automatic)
struct xbar_opts {
  int sweep = -1;   // 0 = CUDA-core FP32 sweep, 1 = tensor-core sweep
  int factor = -1;  // 0 = cooperative-group factor, 1 = cluster factor
  int algo = -1;    // 0 = block Thomas, 1 = block cyclic reduction
  int cr_tensor = -1;  // cyclic reduction, FP32 products: 0 = CUDA cores, 1 = tensor cores
  int orient = -1;  // FP64 factors: 0 = column blocks, 1 = row blocks (mirrored crossbar), -1 = rows when 2N <= M
  int eager_asm = -1;  // 1 = xbar_set_conductances also assembles; otherwise the next factor does
};

struct xbar_s {
  xbar::MapDev m;
  double R[4] = {0, 0, 0, 0};
  cudaStream_t st = nullptr;
  int dev = 0, nsm = 0;
  int assembled = 0;  // per-column elimination data formed from Gc (lazily, by the first factor)
  int factored = 0;
  xbar_precision prec = XBAR_FP64;
  xbar::DevArena A;
  unsigned* status = nullptr;      // device status block (xbar::DevStatus)
  unsigned long long wait_ns = 0;  // limit of the device waits, 0 = the default (host copy)
  xbar_opts opt;
  // factor
  xbar::Buf X, fsig, fpbuf, fbar, fparams;
  // host copy of the parameter block last uploaded to `fparams` (skip identical uploads)
  unsigned char fparams_host[sizeof(xbar::FactorParams<double>)] = {};
  size_t fparams_bytes = 0;
  const void* fparams_dev = nullptr;
  xbar::Buf Xt;    // tensor-core tiled TF32 hi/lo copy of the FP32 factor
  int tc_ready = 0;
  // solve workspace
  xbar::Buf z, dhat, rhat, w64, phi, maxrel, rmax, irstate;
  xbar::Buf w1;  // FP32 refinement state written by the initial tensor-core sweep
  // staging for host pointers
  xbar::Buf sV, sI, svWL, svBL;
  // block cyclic reduction (cr.cu): plans of both precisions; cr_active = factored by it
  xbar::CrPlan<float> cr32;
  xbar::CrPlan<double> cr64;
  int cr_active = 0;
  // blocking over rows (orient.cu): the mirrored crossbar, factored in this handle's place when
  // orient_active (FP64 factors only); it shares this handle's stream and device
  xbar_s* mirror = nullptr;
  int orient_active = 0;
  // transfer-matrix mode: G_eff of the current factorization (valid until the next factor)
  xbar::Buf geff, eye;
  int geff_valid = 0;
  // profiling: events recorded around launches, resolved in xbar_profile_read
  int prof_on = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  xbar_profile prof;
};

namespace xbar {

// RAII scope that brackets the launches of one phase with events when profiling is on
struct PhaseScope {
  xbar_s* h;
  int phase;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int nlaunch;
  PhaseScope(xbar_s* h_, int ph, int n = 1) : h(h_), phase(ph), nlaunch(n) {
    if (!h->prof_on) return;
    e0 = take();
    e1 = take();
    if (e0) cudaEventRecord(e0, h->st);
  }
  cudaEvent_t take() {
    if (!h->ev_pool.empty()) {
      cudaEvent_t e = h->ev_pool.back();
      h->ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  ~PhaseScope() {
    if (!h->prof_on || !e0 || !e1) return;
    cudaEventRecord(e1, h->st);
    h->pending.push_back({phase, {e0, e1}});
    h->prof.launches[phase] += nlaunch;
  }
};

// error reporting shared by the C entry points
xbar_status set_error(xbar_status s, const char* fmt, ...);

// kernel-variant selection (environment XBAR_SWEEP=simt|tc, XBAR_FACTOR=group|cluster override)
bool use_tc_sweep(const xbar_s* h);
bool use_cluster_factor(const xbar_s* h);
// block cyclic reduction (handle option XBAR_OPT_ALGORITHM, environment XBAR_ALGO=cr|thomas)
bool use_cr(const xbar_s* h);
// input vectors per panel of the cyclic-reduction substitution (Bpad = B rounded up to it)
constexpr int kCrPanel = 16;

// factor a handle (FP64 or equilibrated FP32); upload_params = false reuses the parameter block
// already on the device (graph capture)
xbar_status factor_handle(xbar_s* h, xbar_precision p, bool upload_params);

// currents-only solve with device pointers, refinement driven on the device: exactly
// `max_iter` refinement passes are enqueued and passes after convergence skip their work; no
// host synchronisation (capturable).  The workspace must have been sized by an earlier call.
xbar_status solve_device_driven(xbar_s* h, int B, const double* V, double* I, double tol, int max_iter,
                                bool allow_alloc);

}  // namespace xbar
