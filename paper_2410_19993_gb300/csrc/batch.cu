// batch.cu -- many crossbar tiles of uneven sizes (e.g. the tiles a network layer is mapped onto,
// the partitioning of a large crossbar into smaller ones of Sec. III-C), factored and solved with
// their input batches by ONE CUDA-graph launch.
//
// Each tile is an ordinary handle on its own stream.  The first run with a given set of sizes and
// buffers is executed once eagerly (which sizes every workspace), then captured: the factor and
// the device-driven solve of every tile become parallel branches of one graph (fork/join events
// on an origin stream), refinement runs a fixed number of passes whose kernels skip their work
// once a device-side flag says the tile has converged, and no host synchronisation happens inside.
// Later runs with the same signature replay the instantiated graph with a single cudaGraphLaunch.
//
// The autotuner times the kernel variants (tensor-core vs CUDA-core FP32 substitutions, cluster
// vs cooperative-group FP32 factor; for FP64, blocks over columns vs over rows -- the mirrored
// crossbar of orient.cu) on one tile of every distinct (M, N, B), keeps the fastest, and can
// persist its choices in a small JSON file keyed by shape.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <string>
#include <vector>

#include "common.cuh"
#include "handle.h"
#include "kernels.h"

using namespace xbar;

#define XB_CUDA(call)                                                                               \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      if (e_ == cudaErrorMemoryAllocation) {                                                        \
        cudaGetLastError();                                                                         \
        return set_error(XBAR_ENOMEM, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      }                                                                                             \
      return set_error(XBAR_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    }                                                                                               \
  } while (0)

struct xbar_batch_s {
  int T = 0;
  int dev = 0;
  cudaStream_t user = nullptr;    // caller's stream: the batch starts after its prior work
  cudaStream_t origin = nullptr;  // batch-owned capture origin (the legacy stream cannot be captured)
  cudaEvent_t after_user = nullptr;
  std::vector<xbar_t> tiles;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  // cached graph and the signature it was captured for
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  std::vector<int> sigB;
  std::vector<const void*> sigV, sigI;
  int sig_prec = -1, sig_iter = -1;
  double sig_tol = -1.0;
};

static xbar_status destroy_graph(xbar_batch_t b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  return XBAR_OK;
}

extern "C" xbar_status xbar_batch_destroy(xbar_batch_t b) {
  if (!b) return XBAR_OK;
  cudaSetDevice(b->dev);
  for (cudaStream_t s : b->streams) cudaStreamSynchronize(s);
  destroy_graph(b);
  for (xbar_t h : b->tiles) xbar_destroy(h);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  if (b->after_user) cudaEventDestroy(b->after_user);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
  return XBAR_OK;
}

extern "C" xbar_status xbar_batch_create(int T, const xbar_tile* desc, void* cuda_stream, xbar_batch_t* out) {
  if (!out) return set_error(XBAR_EINVAL, "out is NULL");
  *out = nullptr;
  if (T < 1 || !desc) return set_error(XBAR_EINVAL, "need T >= 1 tile descriptions");
  xbar_batch_s* b = new xbar_batch_s();
  b->T = T;
  b->user = (cudaStream_t)cuda_stream;
  cudaGetDevice(&b->dev);
  auto bail = [&](xbar_status s) {
    xbar_batch_destroy(b);
    return s;
  };
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->after_user, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess)
    return bail(set_error(XBAR_ECUDA, "stream/event creation"));
  for (int t = 0; t < T; ++t) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return bail(set_error(XBAR_ECUDA, "stream/event creation for tile %d", t));
    b->streams.push_back(s);
    b->joins.push_back(e);
    xbar_t h = nullptr;
    const xbar_tile& d = desc[t];
    xbar_status st = xbar_assemble(d.M, d.N, d.G, d.R_s, d.R_w, d.R_b, d.R_sense, s, &h);
    if (st != XBAR_OK) return bail(st);
    b->tiles.push_back(h);
  }
  *out = b;
  return XBAR_OK;
}

extern "C" xbar_status xbar_batch_tile(xbar_batch_t b, int t, xbar_t* out) {
  if (!b || !out || t < 0 || t >= b->T) return set_error(XBAR_EINVAL, "bad batch handle or tile index");
  *out = b->tiles[t];
  return XBAR_OK;
}

// enqueue factor + device-driven solve of every tile, each on its own stream forked from `origin`
static xbar_status enqueue_all(xbar_batch_t b, xbar_precision p, const int* B, const double* const* V,
                               double* const* I, double tol, int max_iter, bool eager) {
  XB_CUDA(cudaEventRecord(b->fork, b->origin));
  for (int t = 0; t < b->T; ++t) {
    xbar_t h = b->tiles[t];
    XB_CUDA(cudaStreamWaitEvent(b->streams[t], b->fork, 0));
    xbar_status s = factor_handle(h, p, eager);
    if (s != XBAR_OK) return s;
    if (B[t] > 0) {
      s = solve_device_driven(h, B[t], V[t], I[t], tol, max_iter, eager);
      if (s != XBAR_OK) return s;
    }
    XB_CUDA(cudaEventRecord(b->joins[t], b->streams[t]));
    XB_CUDA(cudaStreamWaitEvent(b->origin, b->joins[t], 0));
  }
  return XBAR_OK;
}

extern "C" xbar_status xbar_batch_run(xbar_batch_t b, xbar_precision p, const int* B, const double* const* V,
                                      double* const* I, double tol, int max_iter, xbar_solve_info* infos) {
  if (!b || !B || !V || !I) return set_error(XBAR_EINVAL, "NULL argument");
  if (p != XBAR_FP64 && p != XBAR_FP32_IR) return set_error(XBAR_EINVAL, "unknown precision %d", (int)p);
  if (p == XBAR_FP32_IR && (max_iter < 1 || !(tol >= 0.0)))
    return set_error(XBAR_EINVAL, "mixed precision needs max_iter >= 1 and tol >= 0");
  XB_CUDA(cudaSetDevice(b->dev));
  const int T = b->T;
  for (int t = 0; t < T; ++t) {
    if (B[t] < 0) return set_error(XBAR_EINVAL, "B[%d]=%d < 0", t, B[t]);
    if (B[t] > 0 && (!is_device_ptr(V[t]) || !is_device_ptr(I[t])))
      return set_error(XBAR_EINVAL, "tile %d: V and I must be device pointers", t);
  }
  const int iters = (p == XBAR_FP32_IR) ? max_iter : 0;
  XB_CUDA(cudaEventRecord(b->after_user, b->user));  // start after the caller's queued work
  XB_CUDA(cudaStreamWaitEvent(b->origin, b->after_user, 0));
  bool same = b->exec && b->sig_prec == (int)p && b->sig_iter == iters && b->sig_tol == tol;
  for (int t = 0; same && t < T; ++t)
    same = b->sigB[t] == B[t] && b->sigV[t] == (const void*)V[t] && b->sigI[t] == (const void*)I[t] &&
           b->tiles[t]->assembled;  // new conductances: the eager run assembles them outside the graph
  if (!same) {
    destroy_graph(b);
    // eager run: sizes every workspace and uploads the factor parameters
    xbar_status s = enqueue_all(b, p, B, V, I, tol, iters, true);
    if (s != XBAR_OK) return s;
    XB_CUDA(cudaStreamSynchronize(b->origin));
    // capture
    XB_CUDA(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed));
    s = enqueue_all(b, p, B, V, I, tol, iters, false);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(b->origin, &g);
    if (s != XBAR_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (ce != cudaSuccess) return set_error(XBAR_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
    b->graph = g;
    XB_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
    b->sigB.assign(B, B + T);
    b->sigV.assign((const void* const*)V, (const void* const*)V + T);
    b->sigI.assign((const void* const*)I, (const void* const*)I + T);
    b->sig_prec = (int)p;
    b->sig_iter = iters;
    b->sig_tol = tol;
  }
  XB_CUDA(cudaGraphLaunch(b->exec, b->origin));
  XB_CUDA(cudaStreamSynchronize(b->origin));
  // per-tile results
  bool all_conv = true;
  int first_bad = -1;
  for (int t = 0; t < T; ++t) {
    xbar_t h = b->tiles[t];
    IrState st;
    memset(&st, 0, sizeof(st));
    if (B[t] > 0 && h->irstate.p) XB_CUDA(cudaMemcpy(&st, h->irstate.p, sizeof(st), cudaMemcpyDeviceToHost));
    unsigned dst = 0;
    XB_CUDA(cudaMemcpy(&dst, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (dst) {
      XB_CUDA(cudaMemset(h->status, 0, sizeof(unsigned)));
      return set_error((dst & XBAR_DEV_TIMEOUT) ? XBAR_ETIMEOUT : XBAR_ECUDA,
                       "tile %d: device status 0x%x", t, dst);
    }
    const bool conv = (p == XBAR_FP64) || B[t] == 0 || st.done;
    if (!conv && all_conv) first_bad = t;
    all_conv = all_conv && conv;
    if (infos) {
      xbar_solve_info& in = infos[t];
      in.iters = st.iters;
      in.max_rel_dI = st.last;
      in.resid_inf = st.rinf;
      double est = st.last;
      if (st.iters >= 2 && st.prev > 0.0f && st.last < st.prev) {
        const double rate = (double)st.last / st.prev;
        est = st.last * rate / (1.0 - rate);
      }
      in.err_est = (p == XBAR_FP32_IR) ? est : 0.0;
      in.n_fallback = 0;
    }
  }
  if (!all_conv)
    return set_error(XBAR_ENOTCONV, "tile %d did not reach tol = %g within %d refinement passes", first_bad, tol,
                     max_iter);
  return XBAR_OK;
}

// ---- autotuner ---------------------------------------------------------------------------------
struct TuneKey {
  int M, N, B, p;
  bool operator<(const TuneKey& o) const {
    if (M != o.M) return M < o.M;
    if (N != o.N) return N < o.N;
    if (B != o.B) return B < o.B;
    return p < o.p;
  }
};
struct TuneVal {
  int sweep = -1, factor = -1, orient = -1;
  float sweep_ms[2] = {-1, -1}, factor_ms[2] = {-1, -1};
  float orient_ms[2] = {-1, -1};  // FP64: factor + solve, blocks over columns / rows
};

static std::string key_str(const TuneKey& k) {
  char buf[96];
  snprintf(buf, sizeof(buf), "M=%d,N=%d,B=%d,prec=%d", k.M, k.N, k.B, k.p);
  return buf;
}

static std::map<TuneKey, TuneVal> load_cache(const char* path) {
  std::map<TuneKey, TuneVal> c;
  if (!path) return c;
  FILE* f = fopen(path, "r");
  if (!f) return c;
  char line[512];
  while (fgets(line, sizeof(line), f)) {
    TuneKey k;
    TuneVal v;
    const int n = sscanf(line, " \"M=%d,N=%d,B=%d,prec=%d\": {\"sweep\": %d, \"factor\": %d, \"orient\": %d", &k.M,
                         &k.N, &k.B, &k.p, &v.sweep, &v.factor, &v.orient);
    if (n >= 6) c[k] = v;  // files written before the orientation field: automatic orientation
  }
  fclose(f);
  return c;
}

static void save_cache(const char* path, const std::map<TuneKey, TuneVal>& c) {
  if (!path) return;
  FILE* f = fopen(path, "w");
  if (!f) return;
  fprintf(f, "{\n");
  size_t n = 0;
  for (const auto& kv : c) {
    const TuneVal& v = kv.second;
    fprintf(f,
            "  \"%s\": {\"sweep\": %d, \"factor\": %d, \"orient\": %d, \"sweep_ms\": [%.4f, %.4f], "
            "\"factor_ms\": [%.4f, %.4f], \"orient_ms\": [%.4f, %.4f]}%s\n",
            key_str(kv.first).c_str(), v.sweep, v.factor, v.orient, v.sweep_ms[0], v.sweep_ms[1], v.factor_ms[0],
            v.factor_ms[1], v.orient_ms[0], v.orient_ms[1], ++n < c.size() ? "," : "");
  }
  fprintf(f, "}\n");
  fclose(f);
}

// time `fn` (enqueued on stream s) once after a warm-up, in milliseconds
template <typename F>
static float time_ms(cudaStream_t s, F fn) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = -1.0f;
  if (fn() == XBAR_OK && cudaStreamSynchronize(s) == cudaSuccess) {
    cudaEventRecord(e0, s);
    if (fn() == XBAR_OK) {
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

extern "C" xbar_status xbar_batch_autotune(xbar_batch_t b, xbar_precision p, const int* B, const char* cache_path) {
  if (!b || !B) return set_error(XBAR_EINVAL, "NULL argument");
  XB_CUDA(cudaSetDevice(b->dev));
  std::map<TuneKey, TuneVal> cache = load_cache(cache_path);
  bool changed = false;
  std::map<TuneKey, int> rep;  // representative tile of every shape
  for (int t = 0; t < b->T; ++t) {
    xbar_t h = b->tiles[t];
    TuneKey k{h->m.M, h->m.N, B[t], (int)p};
    if (!rep.count(k)) rep[k] = t;
  }
  for (const auto& kv : rep) {
    const TuneKey& k = kv.first;
    xbar_t h = b->tiles[kv.second];
    TuneVal v;
    auto it = cache.find(k);
    if (it != cache.end()) {
      v = it->second;
    } else if (p == XBAR_FP32_IR && k.B > 0) {
      // scratch inputs for timing: V = 0.25 V everywhere (values do not affect the kernels' speed)
      double *dV = nullptr, *dI = nullptr;
      XB_CUDA(cudaMalloc(&dV, (size_t)k.B * k.M * 8));
      XB_CUDA(cudaMalloc(&dI, (size_t)k.B * k.N * 8));
      std::vector<double> hv((size_t)k.B * k.M, 0.25);
      cudaMemcpy(dV, hv.data(), hv.size() * 8, cudaMemcpyHostToDevice);
      const int save_f = h->opt.factor, save_s = h->opt.sweep;
      for (int f = 0; f < 2; ++f) {
        h->opt.factor = f;
        if (f == 1 && !use_cluster_factor(h)) continue;
        v.factor_ms[f] = time_ms(h->st, [&]() { return factor_handle(h, p, true); });
      }
      v.factor = (v.factor_ms[1] >= 0 && (v.factor_ms[0] < 0 || v.factor_ms[1] <= v.factor_ms[0])) ? 1 : 0;
      h->opt.factor = v.factor;
      for (int sw = 0; sw < 2; ++sw) {
        h->opt.sweep = sw;
        if (sw == 1 && !use_tc_sweep(h)) continue;
        if (factor_handle(h, p, true) != XBAR_OK) continue;
        v.sweep_ms[sw] = time_ms(h->st, [&]() { return solve_device_driven(h, k.B, dV, dI, 1e-8, 2, true); });
      }
      v.sweep = (v.sweep_ms[1] >= 0 && (v.sweep_ms[0] < 0 || v.sweep_ms[1] <= v.sweep_ms[0])) ? 1 : 0;
      h->opt.factor = save_f;
      h->opt.sweep = save_s;
      cudaFree(dV);
      cudaFree(dI);
      cache[k] = v;
      changed = true;
    } else if (p == XBAR_FP64 && k.B > 0) {
      // FP64: blocks over columns vs over rows, each timed as factor + device-driven solve
      double *dV = nullptr, *dI = nullptr;
      XB_CUDA(cudaMalloc(&dV, (size_t)k.B * k.M * 8));
      XB_CUDA(cudaMalloc(&dI, (size_t)k.B * k.N * 8));
      std::vector<double> hv((size_t)k.B * k.M, 0.25);
      cudaMemcpy(dV, hv.data(), hv.size() * 8, cudaMemcpyHostToDevice);
      const int save_o = h->opt.orient;
      for (int o = 0; o < 2; ++o) {
        if (o == 1 && k.N > 1024) continue;
        h->opt.orient = o;
        v.orient_ms[o] = time_ms(h->st, [&]() {
          xbar_status s = factor_handle(h, p, true);
          return s != XBAR_OK ? s : solve_device_driven(h, k.B, dV, dI, 1e-8, 0, true);
        });
      }
      v.orient = (v.orient_ms[1] >= 0 && (v.orient_ms[0] < 0 || v.orient_ms[1] < v.orient_ms[0])) ? 1 : 0;
      h->opt.orient = save_o;
      cudaFree(dV);
      cudaFree(dI);
      cache[k] = v;
      changed = true;
    }
    // apply to every tile of this shape
    for (int t = 0; t < b->T; ++t) {
      xbar_t ht = b->tiles[t];
      if (ht->m.M == k.M && ht->m.N == k.N && B[t] == k.B) {
        ht->opt.sweep = v.sweep;
        ht->opt.factor = v.factor;
        if (p == XBAR_FP64) ht->opt.orient = v.orient;
      }
    }
  }
  destroy_graph(b);  // choices changed: recapture on the next run
  if (changed) save_cache(cache_path, cache);
  return XBAR_OK;
}
