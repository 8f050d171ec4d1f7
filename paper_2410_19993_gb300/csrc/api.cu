// api.cu -- host implementation of the libxbar C ABI (include/xbar.h).
#include <math.h>
#include <stddef.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "xbar.h"
#include "common.cuh"
#include "handle.h"
#include "kernels.h"

using namespace xbar;

static thread_local std::string g_last_error;

static xbar_status fail(xbar_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

xbar_status xbar::set_error(xbar_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

#define XB_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      if (e_ == cudaErrorMemoryAllocation) {                                               \
        cudaGetLastError();                                                                \
        return fail(XBAR_ENOMEM, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      }                                                                                    \
      return fail(XBAR_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    }                                                                                      \
  } while (0)

static const char* kVersion = "libxbar 0.2 (sm_103a)";

bool xbar::alloc_injected_failure() {
  static std::mutex mu;
  static std::string armed;
  static long long count = 0;
  const char* v = getenv("XBAR_FAIL_ALLOC_AFTER");
  std::lock_guard<std::mutex> lock(mu);
  if (!v || !*v) {
    armed.clear();
    return false;
  }
  if (armed != v) {  // a new value re-arms the counter
    armed = v;
    count = 0;
  }
  return count++ >= atoll(v);
}

extern "C" const char* xbar_version(void) { return kVersion; }
extern "C" const char* xbar_last_error(void) { return g_last_error.c_str(); }

static xbar_status check_status(xbar_t h) {
  unsigned s = 0;
  XB_CUDA(cudaMemcpyAsync(&s, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->st));
  XB_CUDA(cudaStreamSynchronize(h->st));
  if (s) {
    XB_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->st));
    if (s & XBAR_DEV_TIMEOUT) return fail(XBAR_ETIMEOUT, "a bounded device wait expired (status 0x%x)", s);
    if (s & XBAR_DEV_BADINPUT)
      return fail(XBAR_EINVAL, "a conductance passed in device memory was negative or non-finite (status 0x%x)", s);
    if (s & XBAR_DEV_BADLAUNCH) return fail(XBAR_ECUDA, "kernel launch shape inconsistent (status 0x%x)", s);
    if (s & XBAR_DEV_NONFINITE) return fail(XBAR_ECUDA, "non-finite value produced (status 0x%x)", s);
  }
  return XBAR_OK;
}

// A handle with every per-map array and its status block allocated; the map itself is stored by
// the caller.  On failure nothing is left allocated.
static xbar_status new_handle(int M, int N, const double R[4], cudaStream_t st, xbar_s** out) {
  *out = nullptr;
  xbar_s* h = new xbar_s();
  h->st = st;
  for (int k = 0; k < 4; ++k) h->R[k] = R[k];
  cudaGetDevice(&h->dev);
  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->dev);
  MapDev& m = h->m;
  m.M = M;
  m.N = N;
  m.Mp = round_up(M, 16);
  m.gs = 1.0 / R[0];
  m.gw = 1.0 / R[1];
  m.gb = 1.0 / R[2];
  m.go = 1.0 / R[3];
  const size_t nv = (size_t)N * m.Mp;
  auto cleanup = [&](xbar_status s) {
    h->A.free_all();
    delete h;
    return s;
  };
#define XB_ALLOC(ptr, bytes)                                                          \
  do {                                                                                \
    cudaError_t e_ = h->A.alloc((void**)&(ptr), (bytes));                             \
    if (e_ != cudaSuccess) {                                                          \
      cudaGetLastError();                                                             \
      return cleanup(fail(XBAR_ENOMEM, "cudaMalloc(%zu): %s", (size_t)(bytes), cudaGetErrorString(e_))); \
    }                                                                                 \
  } while (0)
  XB_ALLOC(m.Gc, nv * 8);
  XB_ALLOC(m.dW, nv * 8);
  XB_ALLOC(m.h, nv * 8);
  XB_ALLOC(m.tha, nv * 8);
  XB_ALLOC(m.thc, nv * 8);
  XB_ALLOC(m.tdiag, nv * 8);
  XB_ALLOC(m.rho, nv * 8);
  XB_ALLOC(m.s_eq, nv * 8);
  XB_ALLOC(m.e_eq, nv * 8);
  XB_ALLOC(m.e_pl, nv * 8);
  XB_ALLOC(m.hs_eq, nv * 8);
  XB_ALLOC(m.src_eq, (size_t)m.Mp * 8);
  XB_ALLOC(m.src_pl, (size_t)m.Mp * 8);
  XB_ALLOC(m.s32, nv * 4);
  XB_ALLOC(m.e32, nv * 4);
  XB_ALLOC(m.hs32, nv * 4);
  XB_ALLOC(m.src32, (size_t)m.Mp * 4);
  XB_ALLOC(m.Coff, nv * m.Mp * 8);
  XB_ALLOC(m.Gc2, nv * 8);
  XB_ALLOC(m.h2, nv * 8);
  XB_ALLOC(m.tha2, nv * 8);
  XB_ALLOC(m.thc2, nv * 8);
  XB_ALLOC(h->status, sizeof(DevStatus));
  cudaError_t e0 = cudaMemsetAsync(h->status, 0, sizeof(DevStatus), h->st);  // no bits, default wait limit
  if (e0 != cudaSuccess) return cleanup(fail(XBAR_ECUDA, "status block: %s", cudaGetErrorString(e0)));
#undef XB_ALLOC
  *out = h;
  return XBAR_OK;
}

extern "C" xbar_status xbar_assemble(int M, int N, const double* G, double R_s, double R_w, double R_b,
                                     double R_sense, void* cuda_stream, xbar_t* out) {
  if (!out) return fail(XBAR_EINVAL, "out is NULL");
  *out = nullptr;
  if (M < 1 || M > 1024) return fail(XBAR_EINVAL, "M=%d outside [1, 1024]", M);
  if (N < 1 || N > (1 << 20)) return fail(XBAR_EINVAL, "N=%d outside [1, 2^20]", N);
  if (!G) return fail(XBAR_EINVAL, "G is NULL");
  const double R[4] = {R_s, R_w, R_b, R_sense};
  const char* names[4] = {"R_s", "R_w", "R_b", "R_sense"};
  for (int k = 0; k < 4; ++k)
    if (!(R[k] > 0.0) || !isfinite(R[k])) return fail(XBAR_EINVAL, "%s=%g must be finite and > 0", names[k], R[k]);

  // validate G on the host
  std::vector<double> Gh((size_t)M * N);
  const bool gdev = is_device_ptr(G);
  if (gdev) {
    cudaError_t e = cudaMemcpy(Gh.data(), G, Gh.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(XBAR_ECUDA, "copy of G: %s", cudaGetErrorString(e));
  } else {
    memcpy(Gh.data(), G, Gh.size() * sizeof(double));
  }
  for (size_t k = 0; k < Gh.size(); ++k)
    if (!(Gh[k] >= 0.0) || !isfinite(Gh[k]))
      return fail(XBAR_EINVAL, "G[%zu]=%g must be finite and >= 0", k, Gh[k]);

  xbar_s* h = nullptr;
  xbar_status hs = new_handle(M, N, R, (cudaStream_t)cuda_stream, &h);
  if (hs != XBAR_OK) return hs;
  MapDev& m = h->m;
  auto cleanup = [&](xbar_status s) {
    h->A.free_all();
    delete h;
    return s;
  };
#define XB_ALLOC(ptr, bytes)                                                          \
  do {                                                                                \
    cudaError_t e_ = h->A.alloc((void**)&(ptr), (bytes));                             \
    if (e_ != cudaSuccess) {                                                          \
      cudaGetLastError();                                                             \
      return cleanup(fail(XBAR_ENOMEM, "cudaMalloc(%zu): %s", (size_t)(bytes), cudaGetErrorString(e_))); \
    }                                                                                 \
  } while (0)
  double* Gd = nullptr;
  XB_ALLOC(Gd, (size_t)M * N * 8);
#undef XB_ALLOC
  cudaError_t e = cudaMemcpyAsync(Gd, Gh.data(), (size_t)M * N * 8, cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess) {
    PhaseScope ps(h, XBAR_PHASE_ASSEMBLE, 1);
    e = launch_store_g(m, Gd, nullptr, h->st);  // validated on the host above
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return cleanup(fail(XBAR_ECUDA, "assembly: %s", cudaGetErrorString(e)));
  h->A.release(Gd);
  *out = h;
  return XBAR_OK;
}

// kernel launches of one cyclic-reduction substitution (for the per-phase launch counts)
static int cr_sweep_launches(const xbar_s* h, int B, bool initial) {
  (void)B;
  const int L = (int)(h->prec == XBAR_FP64 ? h->cr64.lv.size() : h->cr32.lv.size());
  // right-hand side (or pad clear), last block, back levels, currents; forward levels in
  // correction mode (level 0: two launches)
  return 3 + L + (initial ? 0 : L + 1);
}

// BF16 terms of the tensor-core sweep for refinement correction `it` (0-based).  A correction
// only needs accuracy relative to its own size, so the first two are solved with two terms
// (~2^-17 per product); one term (2^-9 per product, accumulated over the 2N - 1 dependent steps)
// proved too coarse to certify convergence.  Any later correction (slow convergence) uses all
// three (FP32-level accuracy).
static int correction_terms(int it) { return it < 2 ? 2 : 3; }
// The initial solve's error is set by the FP32 factor (~1e-4..1e-3 relative at 256 x 256), far
// above what the two leading BF16 terms of the factor blocks add (~2^-17 per product): the third
// term would only lengthen the sweep's operand stream.
constexpr int kInitialTerms = 2;

// Kernel variants.  FP32 substitutions run on the tensor cores (sweep_tc.cu) when the block fits
// (Mp <= 256) and FP32 factors on a thread-block cluster (factor_cluster.cu) when 32 <= Mp <= 256,
// unless the handle's options (xbar_set_option, set by the batch autotuner) or the environment
// (XBAR_SWEEP=simt|tc, XBAR_FACTOR=group|cluster) choose otherwise.
bool xbar::use_tc_sweep(const xbar_s* h) {
  if (!sweep_tc_supported(h->m.Mp)) return false;
  const char* e = getenv("XBAR_SWEEP");
  if (e && strcmp(e, "simt") == 0) return false;
  if (e && strcmp(e, "tc") == 0) return true;
  return h->opt.sweep != 0;
}

bool xbar::use_cluster_factor(const xbar_s* h) {
  if (!factor_cluster_supported(h->m.Mp)) return false;
  const char* e = getenv("XBAR_FACTOR");
  if (e && strcmp(e, "group") == 0) return false;
  if (e && strcmp(e, "cluster") == 0) return true;
  return h->opt.factor != 0;
}

// Block cyclic reduction when the handle's option (or XBAR_ALGO=cr|thomas) asks for it and the
// block fits (Mp <= 256); block Thomas otherwise.
bool xbar::use_cr(const xbar_s* h) {
  if (!cr_supported(h->m.Mp, h->m.N)) return false;
  const char* e = getenv("XBAR_ALGO");
  if (e && strcmp(e, "thomas") == 0) return false;
  if (e && strcmp(e, "cr") == 0) return true;
  return h->opt.algo == 1;
}

// FP32 cyclic-reduction products on the tensor cores when the blocks are at least 128 rows
static bool use_cr_tensor(const xbar_s* h) {
  if (h->m.Mp < 128) return false;
  const char* e = getenv("XBAR_CR_PRODUCTS");
  if (e && strcmp(e, "simt") == 0) return false;
  if (e && strcmp(e, "tc") == 0) return true;
  return h->opt.cr_tensor != 0;
}

// Blocking over rows (orient.cu): the handle's option 1 (rows) or 0 (columns), or
// XBAR_ORIENT=rows|columns; automatic (-1): rows for FP64 factors when 2N <= M, where the N x N
// blocks make the factor ~(M/N)^2 and each substitution ~M/N times cheaper (mixed precision keeps
// columns unless asked).  The mirror has N rows per block, so N must be within the handle limit.
static bool use_rows(const xbar_s* h, xbar_precision p) {
  if (h->m.N > 1024) return false;
  const char* e = getenv("XBAR_ORIENT");
  if (e && strcmp(e, "columns") == 0) return false;
  if (e && strcmp(e, "rows") == 0) return true;
  if (h->opt.orient >= 0) return h->opt.orient == 1;
  return p == XBAR_FP64 && 2 * h->m.N <= h->m.M;
}

// Build (once) and refresh the mirrored crossbar from this handle's map, then factor it in
// precision p.  The mirror shares the handle's stream, device and status block.
static xbar_status factor_mirror(xbar_s* h, xbar_precision p) {
  const MapDev& m = h->m;
  if (!h->mirror) {
    // R_s' = R_sense, R_w' = R_b, R_b' = R_w, R_sense' = R_s
    const double R2[4] = {h->R[3], h->R[2], h->R[1], h->R[0]};
    xbar_s* g = nullptr;
    xbar_status s = new_handle(m.N, m.M, R2, h->st, &g);
    if (s != XBAR_OK) return s;
    g->A.release(g->status);
    g->status = h->status;
    h->mirror = g;
  }
  xbar_s* g = h->mirror;
  g->opt = h->opt;
  g->opt.orient = 0;
  // automatic algorithm: the mirror's many small blocks (M blocks of N rows) are what cyclic
  // reduction is for, against M dependent block steps of block Thomas
  if (h->opt.algo < 0 && cr_supported(g->m.Mp, g->m.N)) g->opt.algo = 1;
  g->prof_on = 0;  // the caller's phase scopes count the mirror's launches
  XB_CUDA(launch_mirror_gc(m.Gc, m.M, m.Mp, m.N, g->m.Gc, g->m.Mp, h->st));
  g->assembled = 0;
  return factor_handle(g, p, true);
}

// FP64 solve of a row-blocked factorization: the mirror's right-hand side, its substitution (block
// Thomas or cyclic reduction, as it was factored), the currents from its first block and, if asked,
// the node voltages mapped back.  Workspace in the mirror (grown only with allow_alloc).
static xbar_status solve_rows(xbar_s* h, int B, const double* dV, double* dI, double* dvWL, double* dvBL,
                              bool allow_alloc) {
  xbar_s* g = h->mirror;
  const MapDev& m2 = g->m;
  const int M = h->m.M, N = h->m.N, M2 = m2.M, Mp2 = m2.Mp, N2 = m2.N;
  cudaStream_t st = h->st;
  const bool cr = g->cr_active != 0;
  const int Bp = cr ? kCrPanel : sweep_panel_width<double>(Mp2, B, g->nsm);
  const int Bpad = ((B + Bp - 1) / Bp) * Bp;
  const size_t nst = (size_t)N2 * Mp2 * Bpad;
  auto need = [&](Buf& b, size_t bytes) -> bool {
    if (b.p && b.bytes >= bytes) return true;
    return allow_alloc && ensure(g->A, b, bytes) == cudaSuccess;
  };
  if (!need(g->z, nst * 8) || !need(g->w64, nst * 8) || !need(g->phi, nst * 8) ||
      !need(g->sI, (size_t)Bpad * N2 * 8))
    return fail(XBAR_ENOMEM, "workspace of the row-blocked solve");
  double* rhs = (double*)g->phi.p;  // consumed by the substitution; then the mirror's bit-line voltages
  double* w2 = (double*)g->w64.p;
  {
    PhaseScope ps(h, XBAR_PHASE_SWEEP, 2 + (cr ? cr_sweep_launches(g, B, false) : 1));
    XB_CUDA(launch_orient_rhs(dV, m2.h, M, M2, Mp2, B, Bpad, rhs, st));
    if (cr) {
      CrSweepArgs<double> ca;
      memset(&ca, 0, sizeof(ca));
      ca.B = B;
      ca.Bpad = Bpad;
      ca.V = nullptr;
      ca.src = m2.src_pl;
      ca.r = rhs;
      ca.x = w2;
      ca.e = m2.e_pl;
      ca.hs = m2.h;
      ca.I = (double*)g->sI.p;
      XB_CUDA(cr_sweep<double>(g, g->cr64, ca));
    } else {
      SweepParams<double> sp;
      sp.M = M2;
      sp.Mp = Mp2;
      sp.N = N2;
      sp.B = B;
      sp.Bp = Bp;
      sp.Bpad = Bpad;
      sp.X = (const double*)g->X.p;
      sp.e = m2.e_pl;
      sp.hs = m2.h;
      sp.src = m2.src_pl;
      sp.V = nullptr;
      sp.rhs = rhs;
      sp.z = (double*)g->z.p;
      sp.w = w2;
      sp.I = (double*)g->sI.p;
      sp.accumulate = 0;
      sp.max_rel = nullptr;
      sp.status = g->status;
      XB_CUDA(launch_sweep<double>(sp, st));
    }
    XB_CUDA(launch_orient_currents(w2, N, Bpad, B, m2.gs, dI, st));
  }
  if (dvWL || dvBL) {
    PhaseScope ps(h, XBAR_PHASE_OUTPUT, 1 + (dvWL ? 1 : 0) + (dvBL ? 1 : 0));
    XB_CUDA(launch_orient_blvolt(m2, w2, dV, M, B, Bpad, rhs, st));
    if (dvWL) XB_CUDA(launch_orient_to_user(rhs, dvWL, M, N, Mp2, B, Bpad, st));  // original WL = mirror BL
    if (dvBL) XB_CUDA(launch_orient_to_user(w2, dvBL, M, N, Mp2, B, Bpad, st));   // original BL = mirror WL
  }
  return XBAR_OK;
}

// XBAR_FP32_IR solve of a row-blocked factorization: the refinement of xbar_solve run on the
// mirror, with its sources on the bit-line chains (the residual's Vbl term) and the currents read
// from its first block: after the initial solve and every update from the float-pair state, after
// every correction from the correction itself (which also gives the stopping rule's |dI| / |I|).
struct RowsIr {
  int iters = 0;
  double last = 0.0, prev = 0.0, rinf = 0.0;
  bool converged = false;
};
static xbar_status solve_rows_mixed(xbar_s* h, int B, const double* dV, double* dI, double* dvWL, double* dvBL,
                                    double tol, int max_iter, RowsIr* out) {
  xbar_s* g = h->mirror;
  const MapDev& m2 = g->m;
  const int N = h->m.N, M2 = m2.M, Mp2 = m2.Mp, N2 = m2.N;
  cudaStream_t st = h->st;
  const bool cr = g->cr_active != 0;
  const bool tc = g->tc_ready && !cr;
  const int Bp = cr ? kCrPanel : tc ? kSweepTcPanel : sweep_panel_width<float>(Mp2, B, g->nsm);
  const int Bpad = ((B + Bp - 1) / Bp) * Bp;
  const size_t nst = (size_t)N2 * Mp2 * Bpad;
  XB_CUDA(ensure(g->A, g->z, nst * 4));
  XB_CUDA(ensure(g->A, g->dhat, nst * 4));
  XB_CUDA(ensure(g->A, g->rhat, nst * 4));
  XB_CUDA(ensure(g->A, g->w64, nst * 8));
  XB_CUDA(ensure(g->A, g->phi, nst * 8));
  XB_CUDA(ensure(g->A, g->maxrel, 16));
  XB_CUDA(ensure(g->A, g->rmax, 16));
  XB_CUDA(ensure(g->A, g->sI, (size_t)Bpad * N2 * 8));
  if (tc) XB_CUDA(ensure(g->A, g->w1, nst * 4));
  ResidParams rp;
  memset(&rp, 0, sizeof(rp));
  rp.M = M2;
  rp.Mp = Mp2;
  rp.N = N2;
  rp.B = B;
  rp.Bpad = Bpad;
  rp.gs = m2.gs;
  rp.gw = m2.gw;
  rp.gb = m2.gb;
  rp.go = m2.go;
  rp.Gc = m2.Gc;
  rp.dW = m2.dW;
  rp.h = m2.h;
  rp.tha = m2.tha;
  rp.thc = m2.thc;
  rp.s32 = m2.s32;
  rp.V = nullptr;
  rp.Vbl = dV;
  rp.I = (double*)g->sI.p;  // the mirror's own current functional: scratch
  rp.status = g->status;
  rp.w = (double*)g->w64.p;
  rp.w2 = (float2*)g->w64.p;
  rp.dhat = (const float*)g->dhat.p;
  rp.phi = (double*)g->phi.p;
  rp.phi2 = (float2*)g->phi.p;
  rp.Gc2 = m2.Gc2;
  rp.h2 = m2.h2;
  rp.tha2 = m2.tha2;
  rp.thc2 = m2.thc2;
  rp.rhat = (float*)g->rhat.p;
  rp.rmax = (unsigned long long*)g->rmax.p;
  SweepParams<float> sp;
  sp.M = M2;
  sp.Mp = Mp2;
  sp.N = N2;
  sp.B = B;
  sp.Bp = Bp;
  sp.Bpad = Bpad;
  sp.X = (const float*)g->X.p;
  sp.e = m2.e32;
  sp.hs = m2.hs32;
  sp.src = m2.src32;
  sp.V = nullptr;
  sp.rhs = (const float*)g->rhat.p;
  sp.z = (float*)g->z.p;
  sp.w = (float*)g->dhat.p;
  sp.I = (double*)g->sI.p;
  sp.accumulate = 0;
  sp.max_rel = nullptr;
  sp.status = g->status;
  auto sweep32 = [&](int terms) -> cudaError_t {  // dhat = solve32(rhat) (rhat is overwritten by cyclic reduction)
    if (tc) return launch_sweep_tc(sp, g->Xt.p, terms, st);
    if (!cr) return launch_sweep<float>(sp, st);
    CrSweepArgs<float> ca;
    memset(&ca, 0, sizeof(ca));
    ca.B = B;
    ca.Bpad = Bpad;
    ca.V = nullptr;
    ca.src = m2.src32;
    ca.r = (float*)g->rhat.p;
    ca.x = (float*)g->dhat.p;
    ca.e = m2.e32;
    ca.hs = m2.hs32;
    ca.I = (double*)g->sI.p;
    ca.tensor = use_cr_tensor(g) && Bpad >= 128;
    return cr_sweep<float>(g, g->cr32, ca);
  };
  const int nsw = cr ? cr_sweep_launches(g, B, false) : 1;
  {  // x0 = solve32(s o (V h')), the state w = s o x0, I from the state
    PhaseScope ps(h, XBAR_PHASE_SWEEP, 1 + nsw + 1 + (tc ? 0 : 1));
    XB_CUDA(launch_orient_rhs32(dV, m2.h, m2.s32, h->m.M, M2, Mp2, B, Bpad, (float*)g->rhat.p, st));
    if (tc) {  // the sweep writes the state (FP32) itself; the first update turns it into pairs
      sp.w = nullptr;
      sp.w1out = (float*)g->w1.p;
      sp.s32 = m2.s32;
      XB_CUDA(sweep32(kInitialTerms));
      sp.w = (float*)g->dhat.p;
      sp.w1out = nullptr;
      rp.w1 = (const float*)g->w1.p;
    } else {
      XB_CUDA(sweep32(kInitialTerms));
      XB_CUDA(launch_update(rp, 1, st));
    }
    XB_CUDA(launch_orient_state_currents(rp.w2, rp.w1, N, Bpad, B, m2.gs, dI, st));
  }
  bool w_current = true;
  float mr = 0.0f;
  for (int it = 0; it < max_iter; ++it) {
    XB_CUDA(cudaMemsetAsync(g->rmax.p, 0, 8, st));
    {
      PhaseScope ps(h, XBAR_PHASE_RESID);
      XB_CUDA(launch_resid(rp, st));  // rhat = s o (b - A w), sources on the bit-line chains
    }
    XB_CUDA(cudaMemsetAsync(g->maxrel.p, 0, 4, st));
    {
      PhaseScope ps(h, XBAR_PHASE_SWEEP, nsw + 1);
      XB_CUDA(sweep32(correction_terms(it)));
      XB_CUDA(launch_orient_correction_currents((const float*)g->dhat.p, m2.s32, N, Bpad, B, m2.gs, dI,
                                                (float*)g->maxrel.p, g->status, st));
    }
    w_current = false;
    ++out->iters;
    unsigned long long rbits = 0;
    XB_CUDA(cudaMemcpyAsync(&mr, g->maxrel.p, 4, cudaMemcpyDeviceToHost, st));
    XB_CUDA(cudaMemcpyAsync(&rbits, g->rmax.p, 8, cudaMemcpyDeviceToHost, st));
    XB_CUDA(cudaStreamSynchronize(st));
    memcpy(&out->rinf, &rbits, 8);
    out->prev = out->last;
    out->last = mr;
    if (!(mr == mr)) break;
    const double rho = (it >= 1 && out->prev > 0.0) ? (double)mr / out->prev : 1.0;
    if (mr <= tol || (rho <= 0.5 && (double)mr * rho / (1.0 - rho) <= tol)) {
      out->converged = true;
      break;
    }
    {
      PhaseScope ps(h, XBAR_PHASE_UPDATE, 2);
      XB_CUDA(launch_update(rp, 0, st));  // w += s o dhat (into the pairs)
      rp.w1 = nullptr;
      XB_CUDA(launch_orient_state_currents(rp.w2, nullptr, N, Bpad, B, m2.gs, dI, st));
    }
    w_current = true;
  }
  if (dvWL || dvBL) {
    PhaseScope ps(h, XBAR_PHASE_OUTPUT, 2 + (w_current ? 0 : 1) + (dvWL ? 1 : 0) + (dvBL ? 1 : 0));
    if (!w_current) XB_CUDA(launch_update(rp, 0, st));
    XB_CUDA(launch_pair_to_double(rp, st));  // the state as doubles, in place
    XB_CUDA(launch_orient_blvolt(m2, rp.w, dV, h->m.M, B, Bpad, rp.phi, st));
    if (dvWL) XB_CUDA(launch_orient_to_user(rp.phi, dvWL, h->m.M, N, Mp2, B, Bpad, st));
    if (dvBL) XB_CUDA(launch_orient_to_user(rp.w, dvBL, h->m.M, N, Mp2, B, Bpad, st));
  }
  return XBAR_OK;
}

template <typename T>
static xbar_status do_factor_cr(xbar_t h, bool equilibrate) {
  xbar::CrPlan<T>& pl = *reinterpret_cast<xbar::CrPlan<T>*>(sizeof(T) == 4 ? (void*)&h->cr32 : (void*)&h->cr64);
  const bool tensor = sizeof(T) == 4 && use_cr_tensor(h);
  XB_CUDA(xbar::cr_prepare<T>(h, pl, tensor));  // level plan and buffers (once per shape)
  PhaseScope ps(h, XBAR_PHASE_FACTOR, (int)pl.ops.size());
  XB_CUDA(xbar::cr_factor<T>(h, pl, tensor, equilibrate));
  return XBAR_OK;
}

template <typename T>
static xbar_status do_factor(xbar_t h, bool equilibrate, bool upload) {
  MapDev& m = h->m;
  const int Mp = m.Mp, N = m.N;
  const int PB = factor_panel_width<T>();
  int bpm;
  // FP64 needs many SMs (the FP64 pipe is 1/64 of FP32); FP32 is latency-bound, so fewer blocks
  // (cheaper cross-block barriers) with 16 rows each
  if (Mp <= 32) bpm = 1;
  else bpm = std::min(h->nsm, Mp / (sizeof(T) == 8 ? 2 : 16));
  if (bpm < 1) bpm = 1;
  XB_CUDA(ensure(h->A, h->X, (size_t)N * Mp * Mp * sizeof(T)));
  XB_CUDA(ensure(h->A, h->fsig, 2 * (size_t)Mp * sizeof(T)));
  size_t pbuf_n = 2 * (size_t)PB * Mp;
  if (sizeof(T) == 4 && factor_cluster_supported(Mp)) pbuf_n = std::max(pbuf_n, factor_cluster_pbuf_floats(Mp));
  XB_CUDA(ensure(h->A, h->fpbuf, pbuf_n * sizeof(T)));
  XB_CUDA(ensure(h->A, h->fbar, 2 * sizeof(unsigned)));
  XB_CUDA(ensure(h->A, h->fparams, sizeof(FactorParams<T>)));
  FactorParams<T> fp;
  memset(&fp, 0, sizeof(fp));  // padding too: the block is compared byte for byte below
  fp.M = m.M;
  fp.Mp = Mp;
  fp.N = N;
  fp.gsrc = m.gs;
  fp.gw = m.gw;
  fp.Coff = m.Coff;
  fp.h = m.h;
  fp.s = equilibrate ? m.s_eq : nullptr;
  fp.e = equilibrate ? m.e_eq : m.e_pl;
  fp.X = (T*)h->X.p;
  fp.sig = (T*)h->fsig.p;
  fp.pbuf = (T*)h->fpbuf.p;
  fp.bar = (unsigned*)h->fbar.p;
  XB_CUDA(cudaMemsetAsync(h->fbar.p, 0, 2 * sizeof(unsigned), h->st));
  if (upload) {
    // The block changes only when a buffer is (re)allocated.  Upload it, and wait for the copy out
    // of this stack variable, only when it differs from what the device holds: a repeated factor
    // then returns without waiting for its stream (with two maps in flight, the next map's factor
    // is issued without stalling the host in front of the current map's solve).
    static_assert(sizeof(fp) <= sizeof(h->fparams_host), "parameter cache too small");
    if (h->fparams_dev != h->fparams.p || h->fparams_bytes != sizeof(fp) ||
        memcmp(h->fparams_host, &fp, sizeof(fp)) != 0) {
      XB_CUDA(cudaMemcpyAsync(h->fparams.p, &fp, sizeof(fp), cudaMemcpyHostToDevice, h->st));
      XB_CUDA(cudaStreamSynchronize(h->st));  // fp is a stack variable
      memcpy(h->fparams_host, &fp, sizeof(fp));
      h->fparams_bytes = sizeof(fp);
      h->fparams_dev = h->fparams.p;
    }
  }
  PhaseScope ps(h, XBAR_PHASE_FACTOR, sizeof(T) == 4 && use_tc_sweep(h) ? 2 : 1);
  if (sizeof(T) == 4 && use_cluster_factor(h))
    XB_CUDA(launch_factor_cluster((const FactorParams<float>*)h->fparams.p, 1, Mp, h->status, h->st));
  else
    XB_CUDA(launch_factor<T>((const FactorParams<T>*)h->fparams.p, 1, Mp, bpm, h->status, h->st));
  h->tc_ready = 0;
  if (sizeof(T) == 4 && use_tc_sweep(h)) {
    XB_CUDA(ensure(h->A, h->Xt, sweep_tc_tile_bytes(Mp, N)));
    XB_CUDA(launch_sweep_tc_tile((const float*)h->X.p, h->Xt.p, Mp, N, h->st));
    h->tc_ready = 1;
  }
  return XBAR_OK;
}

xbar_status xbar::factor_handle(xbar_s* h, xbar_precision p, bool upload_params) {
  h->factored = 0;
  h->geff_valid = 0;
  h->orient_active = 0;
  if (use_rows(h, p)) {  // the mirrored crossbar (blocks over rows), factored in this handle's place
    PhaseScope ps(h, XBAR_PHASE_FACTOR, 1);
    xbar_status s = factor_mirror(h, p);
    if (s != XBAR_OK) return s;
    // map remap + assembly (3) + the factor (one launch, or the cyclic reduction's operations)
    const xbar_s* g = h->mirror;
    ps.nlaunch = 4 + (g->cr_active ? (int)(p == XBAR_FP64 ? g->cr64.ops.size() : g->cr32.ops.size())
                                   : 1 + g->tc_ready);
    h->orient_active = 1;
    h->cr_active = 0;
    h->tc_ready = 0;
    h->prec = p;
    h->factored = 1;
    return XBAR_OK;
  }
  if (!h->assembled) {  // the elimination data of the current conductances
    PhaseScope ps(h, XBAR_PHASE_ASSEMBLE, 3);
    XB_CUDA(launch_assemble(h->m, h->st));
    h->assembled = 1;
  }
  const bool cr = use_cr(h);
  h->tc_ready = 0;
  xbar_status s;
  if (cr) s = (p == XBAR_FP64) ? do_factor_cr<double>(h, false) : do_factor_cr<float>(h, true);
  else s = (p == XBAR_FP64) ? do_factor<double>(h, false, upload_params) : do_factor<float>(h, true, upload_params);
  if (s != XBAR_OK) return s;
  h->cr_active = cr ? 1 : 0;
  h->prec = p;
  h->factored = 1;
  return XBAR_OK;
}

extern "C" xbar_status xbar_factor(xbar_t h, xbar_precision p) {
  if (!h) return fail(XBAR_EINVAL, "handle is NULL");
  if (p != XBAR_FP64 && p != XBAR_FP32_IR) return fail(XBAR_EINVAL, "unknown precision %d", (int)p);
  XB_CUDA(cudaSetDevice(h->dev));
  return factor_handle(h, p, true);
}

extern "C" xbar_status xbar_set_option(xbar_t h, xbar_option opt, int value) {
  if (!h) return fail(XBAR_EINVAL, "handle is NULL");
  if (opt == XBAR_OPT_WAIT_LIMIT_NS) {
    if (value < -1) return fail(XBAR_EINVAL, "wait limit %d ns < -1", value);
    XB_CUDA(cudaSetDevice(h->dev));
    h->wait_ns = value > 0 ? (unsigned long long)value : 0ull;  // 0: the default
    // pageable source: the copy is staged before the call returns, and later kernels of the
    // stream see the new limit
    XB_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(h->status) + offsetof(DevStatus, wait_ns), &h->wait_ns,
                            sizeof(h->wait_ns), cudaMemcpyHostToDevice, h->st));
    XB_CUDA(cudaStreamSynchronize(h->st));
    return XBAR_OK;
  }
  if (value < -1 || value > 1) return fail(XBAR_EINVAL, "option value %d outside [-1, 1]", value);
  switch (opt) {
    case XBAR_OPT_SWEEP_KERNEL: h->opt.sweep = value; break;
    case XBAR_OPT_FACTOR_KERNEL: h->opt.factor = value; break;
    case XBAR_OPT_ALGORITHM: h->opt.algo = value; break;
    case XBAR_OPT_CR_PRODUCTS: h->opt.cr_tensor = value; break;
    case XBAR_OPT_ORIENTATION: h->opt.orient = value; break;
    case XBAR_OPT_EAGER_ASSEMBLY: h->opt.eager_asm = value; break;
    default: return fail(XBAR_EINVAL, "unknown option %d", (int)opt);
  }
  return XBAR_OK;
}

extern "C" xbar_status xbar_sync(xbar_t h) {
  if (!h) return fail(XBAR_EINVAL, "handle is NULL");
  XB_CUDA(cudaSetDevice(h->dev));
  XB_CUDA(cudaStreamSynchronize(h->st));
  return check_status(h);
}

extern "C" xbar_status xbar_solve(xbar_t h, int B, const double* V, double* I, double* vWL, double* vBL,
                                  double tol, int max_iter, xbar_solve_info* info) {
  if (!h) return fail(XBAR_EINVAL, "handle is NULL");
  if (info) memset(info, 0, sizeof(*info));
  if (!h->factored) return fail(XBAR_ESTATE, "xbar_solve called before xbar_factor");
  if (B < 0) return fail(XBAR_EINVAL, "B=%d < 0", B);
  if (B == 0) return XBAR_OK;
  if (!V || !I) return fail(XBAR_EINVAL, "V and I must not be NULL");
  const bool mixed = h->prec == XBAR_FP32_IR;
  if (mixed && max_iter < 1) return fail(XBAR_EINVAL, "max_iter=%d < 1", max_iter);
  if (mixed && !(tol >= 0.0)) return fail(XBAR_EINVAL, "tol=%g must be >= 0", tol);
  XB_CUDA(cudaSetDevice(h->dev));
  MapDev& m = h->m;
  const int M = m.M, Mp = m.Mp, N = m.N;
  cudaStream_t st = h->st;

  // stage host pointers
  const bool vdev = is_device_ptr(V), idev = is_device_ptr(I);
  const bool want_v = vWL || vBL;
  const bool wdev = !vWL || is_device_ptr(vWL), bdev = !vBL || is_device_ptr(vBL);
  const double* dV = V;
  double* dI = I;
  double *dvWL = vWL, *dvBL = vBL;
  const size_t nVB = (size_t)B * M, nIB = (size_t)B * N, nvolt = (size_t)B * M * N;
  if (!vdev) {
    XB_CUDA(ensure(h->A, h->sV, nVB * 8));
    XB_CUDA(cudaMemcpyAsync(h->sV.p, V, nVB * 8, cudaMemcpyHostToDevice, st));
    dV = (const double*)h->sV.p;
  }
  if (!idev) {
    XB_CUDA(ensure(h->A, h->sI, nIB * 8));
    dI = (double*)h->sI.p;
  }
  if (vWL && !wdev) {
    XB_CUDA(ensure(h->A, h->svWL, nvolt * 8));
    dvWL = (double*)h->svWL.p;
  }
  if (vBL && !bdev) {
    XB_CUDA(ensure(h->A, h->svBL, nvolt * 8));
    dvBL = (double*)h->svBL.p;
  }

  if (h->orient_active) {  // blocked over rows: the mirrored crossbar's solve
    RowsIr ir;
    xbar_status s = mixed ? solve_rows_mixed(h, B, dV, dI, dvWL, dvBL, tol, max_iter, &ir)
                          : solve_rows(h, B, dV, dI, dvWL, dvBL, true);
    if (s != XBAR_OK) return s;
    if (!idev) XB_CUDA(cudaMemcpyAsync(I, dI, nIB * 8, cudaMemcpyDeviceToHost, st));
    if (vWL && !wdev) XB_CUDA(cudaMemcpyAsync(vWL, dvWL, nvolt * 8, cudaMemcpyDeviceToHost, st));
    if (vBL && !bdev) XB_CUDA(cudaMemcpyAsync(vBL, dvBL, nvolt * 8, cudaMemcpyDeviceToHost, st));
    if (mixed || !idev || (vWL && !wdev) || (vBL && !bdev) || !vdev) {
      xbar_status cs = check_status(h);
      if (cs != XBAR_OK) return cs;
    }
    if (info && mixed) {
      info->iters = ir.iters;
      info->max_rel_dI = ir.last;
      info->resid_inf = ir.rinf;
      double est = ir.last;
      if (ir.iters >= 2 && ir.prev > 0.0) {
        const double rate = ir.last / ir.prev;
        if (rate < 1.0) est = ir.last * rate / (1.0 - rate);
      }
      info->err_est = est;
    }
    if (mixed && !ir.converged)
      return fail(XBAR_ENOTCONV, "refinement stopped after %d corrections with max |dI|/|I| = %g > tol = %g",
                  ir.iters, ir.last, tol);
    return XBAR_OK;
  }

  const bool cr = h->cr_active != 0;
  const bool tc = mixed && h->tc_ready && !cr;
  const int Bp = cr ? kCrPanel
                    : tc ? kSweepTcPanel
                         : (mixed ? sweep_panel_width<float>(Mp, B, h->nsm) : sweep_panel_width<double>(Mp, B, h->nsm));
  const int nblk = (B + Bp - 1) / Bp;
  const int Bpad = nblk * Bp;
  const size_t nst = (size_t)N * Mp * Bpad;

  ResidParams rp;
  memset(&rp, 0, sizeof(rp));
  rp.M = M;
  rp.Mp = Mp;
  rp.N = N;
  rp.B = B;
  rp.Bpad = Bpad;
  rp.gs = m.gs;
  rp.gw = m.gw;
  rp.Gc = m.Gc;
  rp.dW = m.dW;
  rp.h = m.h;
  rp.tha = m.tha;
  rp.thc = m.thc;
  rp.s32 = m.s32;
  rp.V = dV;
  rp.I = dI;
  rp.status = h->status;

  int iters = 0;
  double last = 0.0, prev = 0.0, rinf = 0.0;
  bool converged = true;
  if (!mixed) {
    XB_CUDA(ensure(h->A, h->z, nst * 8));
    if (want_v || cr) XB_CUDA(ensure(h->A, h->w64, nst * 8));
    if (want_v) XB_CUDA(ensure(h->A, h->phi, nst * 8));
    SweepParams<double> sp;
    sp.M = M;
    sp.Mp = Mp;
    sp.N = N;
    sp.B = B;
    sp.Bp = Bp;
    sp.Bpad = Bpad;
    sp.X = (const double*)h->X.p;
    sp.e = m.e_pl;
    sp.hs = m.h;
    sp.src = m.src_pl;
    sp.V = dV;
    sp.rhs = nullptr;
    sp.z = (double*)h->z.p;
    sp.w = want_v ? (double*)h->w64.p : nullptr;
    sp.I = dI;
    sp.accumulate = 0;
    sp.max_rel = nullptr;
    sp.status = h->status;
    if (cr) {
      PhaseScope ps(h, XBAR_PHASE_SWEEP, cr_sweep_launches(h, B, true));
      CrSweepArgs<double> ca;
      memset(&ca, 0, sizeof(ca));
      ca.B = B;
      ca.Bpad = Bpad;
      ca.V = dV;
      ca.src = m.src_pl;
      ca.r = (double*)h->z.p;
      ca.x = (double*)h->w64.p;
      ca.e = m.e_pl;
      ca.hs = m.h;
      ca.I = dI;
      XB_CUDA(cr_sweep<double>(h, h->cr64, ca));
    } else {
      PhaseScope ps(h, XBAR_PHASE_SWEEP);
      XB_CUDA(launch_sweep<double>(sp, st));
    }
    rp.w = (double*)h->w64.p;
    rp.phi = (double*)h->phi.p;
  } else {
    XB_CUDA(ensure(h->A, h->z, nst * 4));
    XB_CUDA(ensure(h->A, h->dhat, nst * 4));
    XB_CUDA(ensure(h->A, h->rhat, nst * 4));
    XB_CUDA(ensure(h->A, h->w64, nst * 8));
    XB_CUDA(ensure(h->A, h->phi, nst * 8));
    XB_CUDA(ensure(h->A, h->maxrel, 16));
    XB_CUDA(ensure(h->A, h->rmax, 16));
    rp.w = (double*)h->w64.p;
    rp.w2 = (float2*)h->w64.p;
    rp.dhat = (const float*)h->dhat.p;
    rp.phi = (double*)h->phi.p;
    rp.phi2 = (float2*)h->phi.p;
    rp.Gc2 = m.Gc2;
    rp.h2 = m.h2;
    rp.tha2 = m.tha2;
    rp.thc2 = m.thc2;
    rp.rhat = (float*)h->rhat.p;
    rp.rmax = (unsigned long long*)h->rmax.p;
    SweepParams<float> sp;
    sp.M = M;
    sp.Mp = Mp;
    sp.N = N;
    sp.B = B;
    sp.Bp = Bp;
    sp.Bpad = Bpad;
    sp.X = (const float*)h->X.p;
    sp.e = m.e32;
    sp.hs = m.hs32;
    sp.src = m.src32;
    sp.V = dV;
    sp.rhs = nullptr;
    sp.z = (float*)h->z.p;
    sp.w = (float*)h->dhat.p;
    sp.I = dI;
    sp.accumulate = 0;
    sp.max_rel = nullptr;
    sp.status = h->status;
    // FP32 substitution of the factor's algorithm (CUDA-core block-Thomas sweep, or cyclic
    // reduction with the right-hand side in z (initial) or rhat (corrections), both overwritten)
    auto sweep32 = [&](const SweepParams<float>& q) -> cudaError_t {
      if (!cr) return launch_sweep<float>(q, st);
      CrSweepArgs<float> ca;
      memset(&ca, 0, sizeof(ca));
      ca.B = B;
      ca.Bpad = Bpad;
      ca.V = q.V;
      ca.src = m.src32;
      ca.r = q.V ? (float*)h->z.p : (float*)h->rhat.p;
      ca.x = q.w;
      ca.e = m.e32;
      ca.hs = m.hs32;
      ca.I = q.I;
      ca.accumulate = q.accumulate;
      ca.max_rel = q.max_rel;
      ca.tensor = use_cr_tensor(h) && Bpad >= 128;  // wide batches: products on the tensor cores
      return cr_sweep<float>(h, h->cr32, ca);
    };
    if (tc) {  // x0 = solve32(b); the sweep writes the state w = s o x0 (FP32) itself
      PhaseScope ps(h, XBAR_PHASE_SWEEP);
      XB_CUDA(ensure(h->A, h->w1, nst * 4));
      sp.w = nullptr;
      sp.w1out = (float*)h->w1.p;
      sp.s32 = m.s32;
      XB_CUDA(launch_sweep_tc(sp, h->Xt.p, kInitialTerms, st));
      sp.w = (float*)h->dhat.p;
      sp.w1out = nullptr;
      rp.w1 = (const float*)h->w1.p;  // read as (w, 0) until the first update writes the pairs
    } else {
      {
        PhaseScope ps(h, XBAR_PHASE_SWEEP, cr ? cr_sweep_launches(h, B, true) : 1);
        XB_CUDA(sweep32(sp));                   // x0 = solve32(b)
      }
      PhaseScope ps(h, XBAR_PHASE_UPDATE);
      XB_CUDA(launch_update(rp, 1, st));        // w = s o dhat, I = h . w
    }
    converged = false;
    bool w_current = true;                      // w includes every correction so far
    float mr = 0.0f;
    for (int it = 0; it < max_iter; ++it) {
      XB_CUDA(cudaMemsetAsync(h->rmax.p, 0, 8, st));
      {
        PhaseScope ps(h, XBAR_PHASE_RESID);
        XB_CUDA(launch_resid(rp, st));          // rhat = s o (b - A w)   [float pairs]
      }
      XB_CUDA(cudaMemsetAsync(h->maxrel.p, 0, 4, st));
      sp.V = nullptr;
      sp.rhs = (const float*)h->rhat.p;
      sp.accumulate = 1;
      sp.max_rel = (float*)h->maxrel.p;
      {
        PhaseScope ps(h, XBAR_PHASE_SWEEP, cr ? cr_sweep_launches(h, B, false) : 1);  // dhat = solve32(rhat), I += dI
        if (tc) XB_CUDA(launch_sweep_tc(sp, h->Xt.p, correction_terms(it), st));
        else XB_CUDA(sweep32(sp));
      }
      w_current = false;
      ++iters;
      unsigned long long rbits = 0;
      XB_CUDA(cudaMemcpyAsync(&mr, h->maxrel.p, 4, cudaMemcpyDeviceToHost, st));
      XB_CUDA(cudaMemcpyAsync(&rbits, h->rmax.p, 8, cudaMemcpyDeviceToHost, st));
      XB_CUDA(cudaStreamSynchronize(st));
      memcpy(&rinf, &rbits, 8);
      prev = last;
      last = mr;
      if (!(mr == mr)) break;                   // NaN: give up, reported below
      // converged when this correction is within tol, or when the observed linear contraction
      // rate rho = |dI_k| / |dI_{k-1}| bounds what remains after applying it:
      // |dI_k| rho / (1 - rho) <= tol (rho <= 1/2, at least two corrections)
      const double rho = (it >= 1 && prev > 0.0) ? (double)mr / prev : 1.0;
      if (mr <= tol || (rho <= 0.5 && (double)mr * rho / (1.0 - rho) <= tol)) {
        converged = true;
        break;
      }
      {
        PhaseScope ps(h, XBAR_PHASE_UPDATE);
        XB_CUDA(launch_update(rp, 0, st));      // w += s o dhat, I = h . w   [float pairs]
      }
      rp.w1 = nullptr;
      w_current = true;
    }
    if (want_v && !w_current) {
      PhaseScope ps(h, XBAR_PHASE_UPDATE);
      XB_CUDA(launch_update(rp, 0, st));
    }
    if (want_v) {  // the node-voltage output reads the state as doubles
      PhaseScope ps(h, XBAR_PHASE_OUTPUT);
      XB_CUDA(launch_pair_to_double(rp, st));
    }
  }
  if (want_v) {
    PhaseScope ps(h, XBAR_PHASE_OUTPUT, 1 + (dvWL ? 1 : 0) + (dvBL ? 1 : 0));
    XB_CUDA(launch_blvolt(rp, (double*)h->phi.p, st));
    if (dvWL) XB_CUDA(launch_to_user_layout((const double*)h->w64.p, dvWL, M, Mp, N, B, Bpad, st));
    if (dvBL) XB_CUDA(launch_to_user_layout((const double*)h->phi.p, dvBL, M, Mp, N, B, Bpad, st));
  }
  const bool any_host = !idev || (vWL && !wdev) || (vBL && !bdev) || !vdev;
  if (!idev) XB_CUDA(cudaMemcpyAsync(I, dI, nIB * 8, cudaMemcpyDeviceToHost, st));
  if (vWL && !wdev) XB_CUDA(cudaMemcpyAsync(vWL, dvWL, nvolt * 8, cudaMemcpyDeviceToHost, st));
  if (vBL && !bdev) XB_CUDA(cudaMemcpyAsync(vBL, dvBL, nvolt * 8, cudaMemcpyDeviceToHost, st));
  if (mixed || any_host) {
    xbar_status s = check_status(h);
    if (s != XBAR_OK) return s;
  }
  if (info) {
    info->iters = iters;
    info->max_rel_dI = last;
    info->resid_inf = rinf;
    double est = last;
    if (iters >= 2 && prev > 0.0) {
      const double rate = last / prev;
      if (rate < 1.0) est = last * rate / (1.0 - rate);
    }
    info->err_est = mixed ? est : 0.0;
    info->n_fallback = 0;
  }
  if (mixed && !converged)
    return fail(XBAR_ENOTCONV, "refinement stopped after %d corrections with max |dI|/|I| = %g > tol = %g",
                iters, last, tol);
  return XBAR_OK;
}

xbar_status xbar::solve_device_driven(xbar_s* h, int B, const double* dV, double* dI, double tol, int max_iter,
                                      bool allow_alloc) {
  MapDev& m = h->m;
  const int M = m.M, Mp = m.Mp, N = m.N;
  cudaStream_t st = h->st;
  if (h->orient_active && h->prec != XBAR_FP64)
    return fail(XBAR_ESTATE, "device-driven solves (tile batches) block over rows in XBAR_FP64 only");
  if (h->orient_active) {  // FP64, blocked over rows (stream-ordered launches only)
    if (!(h->irstate.p && h->irstate.bytes >= sizeof(IrState)) &&
        !(allow_alloc && ensure(h->A, h->irstate, sizeof(IrState)) == cudaSuccess))
      return fail(XBAR_ENOMEM, "refinement state");
    XB_CUDA(launch_ir_init((IrState*)h->irstate.p, st));
    return solve_rows(h, B, dV, dI, nullptr, nullptr, allow_alloc);
  }
  if (h->cr_active)
    return fail(XBAR_ESTATE, "device-driven solves (tile batches) need a block-Thomas factorization");
  const bool mixed = h->prec == XBAR_FP32_IR;
  const bool tc = mixed && h->tc_ready;
  const int Bp = tc ? kSweepTcPanel
                    : (mixed ? sweep_panel_width<float>(Mp, B, h->nsm) : sweep_panel_width<double>(Mp, B, h->nsm));
  const int Bpad = ((B + Bp - 1) / Bp) * Bp;
  const size_t nst = (size_t)N * Mp * Bpad;
  auto need = [&](Buf& b, size_t bytes) -> bool {
    if (b.p && b.bytes >= bytes) return true;
    return allow_alloc && ensure(h->A, b, bytes) == cudaSuccess;
  };
  if (!need(h->irstate, sizeof(IrState))) return fail(XBAR_ENOMEM, "refinement state");
  IrState* state = (IrState*)h->irstate.p;
  if (!mixed) {
    if (!need(h->z, nst * 8)) return fail(XBAR_ENOMEM, "workspace not prepared for this batch size");
    SweepParams<double> sp;
    sp.M = M; sp.Mp = Mp; sp.N = N; sp.B = B; sp.Bp = Bp; sp.Bpad = Bpad;
    sp.X = (const double*)h->X.p; sp.e = m.e_pl; sp.hs = m.h; sp.src = m.src_pl;
    sp.V = dV; sp.rhs = nullptr; sp.z = (double*)h->z.p; sp.w = nullptr; sp.I = dI;
    sp.accumulate = 0; sp.max_rel = nullptr; sp.status = h->status;
    XB_CUDA(launch_ir_init(state, st));
    XB_CUDA(launch_sweep<double>(sp, st));
    return XBAR_OK;
  }
  if (!need(h->z, nst * 4) || !need(h->dhat, nst * 4) || !need(h->rhat, nst * 4) || !need(h->w64, nst * 8) ||
      !need(h->phi, nst * 8))
    return fail(XBAR_ENOMEM, "workspace not prepared for this batch size");
  ResidParams rp;
  memset(&rp, 0, sizeof(rp));
  rp.M = M; rp.Mp = Mp; rp.N = N; rp.B = B; rp.Bpad = Bpad;
  rp.gs = m.gs; rp.gw = m.gw; rp.Gc = m.Gc; rp.dW = m.dW; rp.h = m.h; rp.tha = m.tha; rp.thc = m.thc;
  rp.s32 = m.s32; rp.V = dV; rp.I = dI; rp.status = h->status;
  rp.w = (double*)h->w64.p; rp.dhat = (const float*)h->dhat.p; rp.phi = (double*)h->phi.p;
  rp.w2 = (float2*)h->w64.p; rp.phi2 = (float2*)h->phi.p;
  rp.Gc2 = m.Gc2; rp.h2 = m.h2; rp.tha2 = m.tha2; rp.thc2 = m.thc2;
  rp.rhat = (float*)h->rhat.p; rp.rmax = &state->rmax;
  SweepParams<float> sp;
  sp.M = M; sp.Mp = Mp; sp.N = N; sp.B = B; sp.Bp = Bp; sp.Bpad = Bpad;
  sp.X = (const float*)h->X.p; sp.e = m.e32; sp.hs = m.hs32; sp.src = m.src32;
  sp.V = dV; sp.rhs = nullptr; sp.z = (float*)h->z.p; sp.w = (float*)h->dhat.p; sp.I = dI;
  sp.accumulate = 0; sp.max_rel = nullptr; sp.status = h->status;
  auto sweep = [&](int terms) -> cudaError_t {
    return tc ? launch_sweep_tc(sp, h->Xt.p, terms, st) : launch_sweep<float>(sp, st);
  };
  XB_CUDA(launch_ir_init(state, st));
  if (tc) {  // x0 = solve32(b); the sweep writes the state w = s o x0 (FP32) itself
    if (!need(h->w1, nst * 4)) return fail(XBAR_ENOMEM, "workspace not prepared for this batch size");
    sp.w = nullptr;
    sp.w1out = (float*)h->w1.p;
    sp.s32 = m.s32;
    XB_CUDA(sweep(kInitialTerms));
    sp.w = (float*)h->dhat.p;
    sp.w1out = nullptr;
    rp.w1 = (const float*)h->w1.p;  // read as (w, 0) until the first update writes the pairs
  } else {
    XB_CUDA(sweep(kInitialTerms));       // x0 = solve32(b)
    XB_CUDA(launch_update(rp, 1, st));   // w = s o dhat, I = h . w
  }
  sp.V = nullptr;
  sp.rhs = (const float*)h->rhat.p;
  sp.accumulate = 1;
  sp.max_rel = &state->maxrel;
  sp.skip = &state->done;
  rp.skip = &state->done;
  for (int it = 0; it < max_iter; ++it) {
    XB_CUDA(launch_resid(rp, st));       // rhat = s o (b - A w)   [float pairs]  (skipped once converged)
    XB_CUDA(sweep(correction_terms(it)));  // dhat = solve32(rhat), I += dI
    XB_CUDA(launch_ir_check(state, tol, st));
    XB_CUDA(launch_update(rp, 0, st));   // w += s o dhat, I = h . w   (skipped once converged)
    rp.w1 = nullptr;                     // later passes read the pairs the update wrote
  }
  return XBAR_OK;
}

extern "C" xbar_status xbar_destroy(xbar_t h) {
  if (!h) return XBAR_OK;
  cudaSetDevice(h->dev);
  cudaStreamSynchronize(h->st);
  if (h->mirror) {  // its status block is this handle's: not in its arena
    xbar_destroy(h->mirror);
    h->mirror = nullptr;
  }
  for (auto& pe : h->pending) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  h->A.free_all();
  delete h;
  return XBAR_OK;
}

extern "C" xbar_status xbar_profile_enable(xbar_t h, int enable) {
  if (!h) return fail(XBAR_EINVAL, "handle is NULL");
  XB_CUDA(cudaSetDevice(h->dev));
  XB_CUDA(cudaStreamSynchronize(h->st));
  for (auto& pe : h->pending) {
    h->ev_pool.push_back(pe.second.first);
    h->ev_pool.push_back(pe.second.second);
  }
  h->pending.clear();
  memset(&h->prof, 0, sizeof(h->prof));
  h->prof_on = enable ? 1 : 0;
  return XBAR_OK;
}

extern "C" xbar_status xbar_profile_read(xbar_t h, xbar_profile* out, int reset) {
  if (!h || !out) return fail(XBAR_EINVAL, "handle or out is NULL");
  XB_CUDA(cudaSetDevice(h->dev));
  XB_CUDA(cudaStreamSynchronize(h->st));
  for (auto& pe : h->pending) {
    float ms = 0.0f;
    XB_CUDA(cudaEventElapsedTime(&ms, pe.second.first, pe.second.second));
    h->prof.ms[pe.first] += ms;
    h->ev_pool.push_back(pe.second.first);
    h->ev_pool.push_back(pe.second.second);
  }
  h->pending.clear();
  *out = h->prof;
  if (reset) memset(&h->prof, 0, sizeof(h->prof));
  return XBAR_OK;
}

extern "C" xbar_status xbar_set_conductances(xbar_t h, const double* G) {
  if (!h || !G) return fail(XBAR_EINVAL, "handle or G is NULL");
  XB_CUDA(cudaSetDevice(h->dev));
  MapDev& m = h->m;
  const size_t n = (size_t)m.M * m.N;
  const bool gdev = is_device_ptr(G);
  const double* Gd = G;
  if (!gdev) {  // host map: validated here, then staged
    for (size_t k = 0; k < n; ++k)
      if (!(G[k] >= 0.0) || !isfinite(G[k])) return fail(XBAR_EINVAL, "G[%zu]=%g must be finite and >= 0", k, G[k]);
    XB_CUDA(ensure(h->A, h->sV, std::max(h->sV.bytes, n * 8)));
    XB_CUDA(cudaMemcpyAsync(h->sV.p, G, n * 8, cudaMemcpyHostToDevice, h->st));
    // G is read before the call returns; the kernels below stay asynchronous (a later xbar_solve
    // refills the staging buffer on the same stream, after they have read it)
    XB_CUDA(cudaStreamSynchronize(h->st));
    Gd = (const double*)h->sV.p;
  }
  h->factored = 0;
  h->geff_valid = 0;
  h->assembled = 0;
  {
    // a device map is validated by the transposing kernel itself (status word, reported by the
    // next call that reads it), so the host does not wait for the stream here
    const bool eager = h->opt.eager_asm == 1;
    PhaseScope ps(h, XBAR_PHASE_ASSEMBLE, eager ? 4 : 1);
    XB_CUDA(launch_store_g(m, Gd, gdev ? h->status : nullptr, h->st));
    if (eager) {  // the elimination data at once, so that a factor queued behind this call starts
      XB_CUDA(launch_assemble(m, h->st));
      h->assembled = 1;
    }
  }
  return XBAR_OK;
}

// ---------------------------------------------------------------------------------------------
// xbar_solve_noalloc: the FP64 substitution with its scratch in a fixed device array
// ---------------------------------------------------------------------------------------------
// Some callers must not allocate device memory while they solve: a latency-critical loop in which
// cudaMalloc/cudaFree could implicitly synchronise the device and stall it, or a process whose
// device memory is owned by a framework allocator that forbids allocations outside its pool.
// For them this entry point runs the same forward/back substitution kernel as xbar_solve on an
// XBAR_FP64-factored handle, but takes the kernel's scratch (the forward-sweep results, N x Mp x
// Bpad doubles) from the file-scope array below instead of the handle's growable workspace.  It
// calls no cudaMalloc, cudaFree or allocating library routine.
//
// The array is a fixed XBAR_NOALLOC_SCRATCH_BYTES (64 MiB) on every GPU that loads the library and
// stays reserved until the process exits.  Host code cannot use the array's name as an address (it
// names a host-side stand-in), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call that uses the device; make
// that first call before any stream capture.  All calls share the one array: calls whose work
// overlaps on the GPU race on it.  Its contents are whatever the last call left; the kernel writes
// every scratch element it later reads, so nothing needs clearing.
#define XBAR_NOALLOC_SCRATCH_BYTES (64ull << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[XBAR_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoallocMaxDevices] = {nullptr};

// device address of g_noalloc_scratch on the current device `dev` (looked up once per device)
cudaError_t noalloc_scratch(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (dev < 0 || dev >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}
}  // namespace

// ---- transfer-matrix mode (currents only) ------------------------------------------------------
extern "C" xbar_status xbar_transfer_matrix(xbar_t h, double tol, int max_iter, double* Geff, xbar_solve_info* info) {
  if (!h) return fail(XBAR_EINVAL, "handle is NULL");
  if (info) memset(info, 0, sizeof(*info));
  if (!h->factored) return fail(XBAR_ESTATE, "xbar_transfer_matrix called before xbar_factor");
  XB_CUDA(cudaSetDevice(h->dev));
  const int M = h->m.M, N = h->m.N;
  const size_t n = (size_t)M * N;
  if (!h->geff_valid) {  // M unit-input solves of the current factorization: row i of I is G_eff[i][:]
    XB_CUDA(ensure(h->A, h->geff, n * 8));
    XB_CUDA(ensure(h->A, h->eye, (size_t)M * M * 8));
    XB_CUDA(launch_eye((double*)h->eye.p, M, h->st));
    xbar_solve_info si;
    const xbar_status s = xbar_solve(h, M, (const double*)h->eye.p, (double*)h->geff.p, nullptr, nullptr, tol,
                                     max_iter, &si);
    if (info) *info = si;
    if (s != XBAR_OK) return s;  // message set by xbar_solve
    h->geff_valid = 1;
  }
  if (Geff) {
    XB_CUDA(cudaMemcpyAsync(Geff, h->geff.p, n * 8, cudaMemcpyDefault, h->st));
    if (!is_device_ptr(Geff)) XB_CUDA(cudaStreamSynchronize(h->st));
  }
  return check_status(h);
}

extern "C" xbar_status xbar_solve_transfer(xbar_t h, int B, const double* V, double* I) {
  if (!h) return fail(XBAR_EINVAL, "handle is NULL");
  if (!h->factored || !h->geff_valid)
    return fail(XBAR_ESTATE, "xbar_solve_transfer needs xbar_transfer_matrix after the last xbar_factor");
  if (B < 0) return fail(XBAR_EINVAL, "B=%d < 0", B);
  if (B == 0) return XBAR_OK;
  if (!V || !I) return fail(XBAR_EINVAL, "V and I must not be NULL");
  XB_CUDA(cudaSetDevice(h->dev));
  const int M = h->m.M, N = h->m.N;
  cudaStream_t st = h->st;
  const bool vdev = is_device_ptr(V), idev = is_device_ptr(I);
  const size_t nVB = (size_t)B * M, nIB = (size_t)B * N;
  const double* dV = V;
  double* dI = I;
  if (!vdev) {
    XB_CUDA(ensure(h->A, h->sV, nVB * 8));
    XB_CUDA(cudaMemcpyAsync(h->sV.p, V, nVB * 8, cudaMemcpyHostToDevice, st));
    dV = (const double*)h->sV.p;
  }
  if (!idev) {
    XB_CUDA(ensure(h->A, h->sI, nIB * 8));
    dI = (double*)h->sI.p;
  }
  {
    PhaseScope ps(h, XBAR_PHASE_SWEEP);  // the product replaces the substitutions
    XB_CUDA(launch_gemm_f64(dV, (const double*)h->geff.p, dI, B, M, N, st));
  }
  if (!idev) {  // host output: synchronise (and report device status), as xbar_solve does
    XB_CUDA(cudaMemcpyAsync(I, dI, nIB * 8, cudaMemcpyDeviceToHost, st));
    return check_status(h);
  }
  return XBAR_OK;  // asynchronous on the handle's stream
}

extern "C" xbar_status xbar_solve_noalloc(xbar_t h, int B, const double* V, double* I) {
  if (!h) return fail(XBAR_EINVAL, "handle is NULL");
  if (!h->factored || h->prec != XBAR_FP64 || h->cr_active || h->orient_active)
    return fail(XBAR_ESTATE,
                "xbar_solve_noalloc needs a handle factored with XBAR_FP64 by block Thomas over columns");
  if (B < 0) return fail(XBAR_EINVAL, "B=%d < 0", B);
  if (B == 0) return XBAR_OK;
  if (!V || !I) return fail(XBAR_EINVAL, "V and I must not be NULL");
  if (!is_device_ptr(V) || !is_device_ptr(I))
    return fail(XBAR_EINVAL, "xbar_solve_noalloc takes device pointers only (host buffers would need staging)");
  XB_CUDA(cudaSetDevice(h->dev));
  const MapDev& m = h->m;
  const int Bp = sweep_panel_width<double>(m.Mp, B, h->nsm);
  const int Bpad = ((B + Bp - 1) / Bp) * Bp;
  const size_t need = (size_t)m.N * m.Mp * Bpad * sizeof(double);
  if (need > XBAR_NOALLOC_SCRATCH_BYTES)
    return fail(XBAR_EINVAL,
                "xbar_solve_noalloc: N*Mp*Bpad*8 = %zu bytes of scratch exceeds the fixed %llu bytes "
                "(N=%d, Mp=%d, Bpad=%d); use xbar_solve or a smaller batch",
                need, (unsigned long long)XBAR_NOALLOC_SCRATCH_BYTES, m.N, m.Mp, Bpad);
  void* scratch = nullptr;
  {
    cudaError_t e = noalloc_scratch(h->dev, &scratch);
    if (e != cudaSuccess) return fail(XBAR_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
  }
  SweepParams<double> sp;
  sp.M = m.M;
  sp.Mp = m.Mp;
  sp.N = m.N;
  sp.B = B;
  sp.Bp = Bp;
  sp.Bpad = Bpad;
  sp.X = (const double*)h->X.p;
  sp.e = m.e_pl;
  sp.hs = m.h;
  sp.src = m.src_pl;
  sp.V = V;
  sp.rhs = nullptr;
  sp.z = (double*)scratch;
  sp.w = nullptr;
  sp.I = I;
  sp.accumulate = 0;
  sp.max_rel = nullptr;
  sp.status = h->status;
  XB_CUDA(launch_sweep<double>(sp, h->st));
  return XBAR_OK;
}
