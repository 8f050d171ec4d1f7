// resid.cu -- extended-precision steps of mixed-precision iterative refinement, and node-voltage
// output.
//
// The refinement state is the vector w of word-line node voltages, held as float pairs
// (hi + lo, ~48 significant bits).  Bit-line voltages are not stored: for any w they follow from
// the bit-line rows of the nodal system (Eqs. 3, 4, 7),
//     T_j u_j = G_j o w_j     (tridiagonal chain of bit line j),
// solved with the same subtraction-free pivots as the assembly.  The word-line rows (Eqs. 1, 2,
// 5, 6) then give the residual of the nodal system restricted to word-line nodes,
//     r(i,j) = b(i,j) + g_w (w(i,j-1) + w(i,j+1)) + G_ij u(i,j) - dW(i,j) w(i,j),
// b = g_s V_i at j = 0, evaluated as a sum of branch currents.  The bit-line rows hold exactly by
// construction of u, so r is the full residual of the 2MN system.  The residual and the update
// w += s o dhat are the only extended-precision arithmetic of the mixed path; they run in float
// pairs on the FP32 pipe (FP64 is 1/64 of its rate on this part).  Their error, ~2^-48 of each
// branch current, bounds what refinement can reach: about 1e-10 relative current error at
// 256 x 256, against the 1e-8 target.
//
// One thread per (column j, input vector b); consecutive threads take consecutive b, so every
// access to the [N][Mp][Bpad] arrays is coalesced.  Loops run along the chain i (the residual in
// segments of rows, see resid_kernel).
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "handle.h"
#include "kernels.h"

namespace xbar {

// ---- float-pair arithmetic ----------------------------------------------------------------------
// A value is hi + lo with |lo| <= ulp(hi) / 2 (~48 significant bits).  Sums use the error-free
// two-sum transformation of the leading parts plus the sum of the trailing parts; products use
// the FMA residual of the leading product (Dekker / Knuth transformations, as in double-double
// arithmetic).  Only the FP32 pipe is used: on this part it runs 64 times the FP64 rate.
struct fp2 {
  float hi, lo;
};
__device__ __forceinline__ fp2 quick_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ fp2 two_sum(float a, float b) {
  const float s = a + b, v = s - a;
  return {s, (a - (s - v)) + (b - v)};
}
__device__ __forceinline__ fp2 padd(fp2 x, fp2 y) {
  const fp2 t = two_sum(x.hi, y.hi);
  return quick_two_sum(t.hi, t.lo + (x.lo + y.lo));
}
__device__ __forceinline__ fp2 psub(fp2 x, fp2 y) { return padd(x, fp2{-y.hi, -y.lo}); }
__device__ __forceinline__ fp2 pmul(fp2 x, fp2 y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return quick_two_sum(p, e);
}
// The same transformations without the final renormalisation, for sums and products of terms of
// one sign (no cancellation): hi + lo keeps the accuracy of the pair arithmetic above, while |lo|
// may grow to a few ulp(hi).  Three FP32 operations fewer each; the residual is bound by issue
// slots.  Differences that cancel (neighbouring node voltages) keep the normalised forms.
__device__ __forceinline__ fp2 padd_u(fp2 x, fp2 y) {
  const float s = x.hi + y.hi, v = s - x.hi;
  return {s, ((x.hi - (s - v)) + (y.hi - v)) + (x.lo + y.lo)};
}
__device__ __forceinline__ fp2 pmul_u(fp2 x, fp2 y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return {p, e};
}
// x - y for a difference that goes into a product: the exact two-sum of the leading parts plus the
// difference of the trailing ones, not renormalised (pmul_u accepts a trailing part of a few ulp)
__device__ __forceinline__ fp2 psub_u(fp2 x, fp2 y) {
  const fp2 t = two_sum(x.hi, -y.hi);
  return {t.hi, t.lo + (x.lo - y.lo)};
}
// (l - w) + (r - w), not renormalised: three exact two-sums of the leading parts, the trailing
// parts and the rounding errors summed once
__device__ __forceinline__ fp2 pdiff2_u(fp2 l, fp2 r, fp2 w) {
  const fp2 a = two_sum(l.hi, -w.hi), c = two_sum(r.hi, -w.hi), s = two_sum(a.hi, c.hi);
  return {s.hi, s.lo + ((a.lo + c.lo) + fmaf(-2.0f, w.lo, l.lo + r.lo))};
}
// the FP32 rounding of x + y: the exact two-sum of the leading parts, then everything else
__device__ __forceinline__ float psum_f(fp2 x, fp2 y) {
  const fp2 t = two_sum(x.hi, y.hi);
  return t.hi + (t.lo + (x.lo + y.lo));
}
__device__ __forceinline__ fp2 ld2(const float2* a, size_t o) {
  const float2 v = a[o];
  return {v.x, v.y};
}
__device__ __forceinline__ void st2(float2* a, size_t o, fp2 v) { a[o] = make_float2(v.hi, v.lo); }
// the refinement state at o: float pairs, or (kW1) the FP32 state the initial tensor-core sweep
// writes; for the update, whichever the parameters hold
template <bool kW1>
__device__ __forceinline__ fp2 ldw(const ResidParams& p, size_t o) {
  if constexpr (kW1) return fp2{p.w1[o], 0.0f};
  else return ld2(p.w2, o);
}
__device__ __forceinline__ fp2 ldw_any(const ResidParams& p, size_t o) {
  return p.w1 ? ldw<true>(p, o) : ldw<false>(p, o);
}
__device__ __forceinline__ fp2 split(double x) {
  const float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}

// w = (first ? 0 : w) + s * dhat,  I[b][j] = h_j . w_j   (float pairs; I written as a double).
// Rows are taken kUpd at a time with all their loads issued before the first store, so a thread
// waits for memory once per batch rather than once per row.
constexpr int kUpd = 8;
__global__ void __launch_bounds__(128, 8) update_kernel(ResidParams p, int first) {
  if (p.skip && *p.skip) return;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (b >= p.Bpad || j >= p.N) return;
  const size_t base = (size_t)j * p.Mp, rs = p.Bpad, o0 = base * rs + b;
  const float* dh = p.dhat + o0;
  float2* w2 = p.w2 + o0;
  const float* w1 = p.w1 ? p.w1 + o0 : nullptr;
  fp2 Iacc{0.0f, 0.0f};
  for (int i0 = 0; i0 < p.M; i0 += kUpd) {
    const int n = min(kUpd, p.M - i0);
    float d[kUpd];
    fp2 w[kUpd];
#pragma unroll
    for (int q = 0; q < kUpd; ++q) {
      if (q < n) {
        const long o = (long)(i0 + q) * (long)rs;
        d[q] = dh[o];
        if (!first) {
          if (w1) {
            w[q] = fp2{w1[o], 0.0f};
          } else {
            const float2 v = w2[o];
            w[q] = fp2{v.x, v.y};
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kUpd; ++q) {
      if (q < n) {
        const int i = i0 + q;
        const float dd = p.s32[base + i] * d[q];
        const fp2 wn = first ? fp2{dd, 0.0f} : padd(w[q], fp2{dd, 0.0f});
        w2[(long)i * (long)rs] = make_float2(wn.hi, wn.lo);
        Iacc = padd(Iacc, pmul(ld2(p.h2, base + i), wn));
      }
    }
  }
  if (b < p.B) p.I[(size_t)b * p.N + j] = (double)Iacc.hi + (double)Iacc.lo;
}

// Residual of the word-line rows (Eqs. 1, 2, 5, 6) as the sum of the branch currents into node
// (i, j), each formed from a voltage difference (neighbouring voltages differ by millivolts, so
// the differences keep full relative accuracy in pairs):
//   r = g_w ([j > 0] (w_{j-1} - w) + [j < N-1] (w_{j+1} - w)) + [j = 0] g_s (V_i - w) + G (u - w),
// identical to b + g_w (w_{j-1} + w_{j+1}) + G u - dW w.  u = T^-1 (G o w) by the bit-line chain
// (forward phi_i = tha_i w_i + thc_i phi_{i-1}, back u_i = phi_i + thc_i u_{i+1}; all terms >= 0).
//
// The chain is walked in segments of kSeg rows so that phi never makes a round trip through
// memory per node: a first forward walk keeps only the value entering each segment (one pair per
// kSeg nodes, in the phi scratch), then the back walk takes the segments last to first.  For each
// it loads the segment's state and its two neighbour columns at once (one memory latency per
// segment, not per row), recomputes phi from the stored entry value (the same operations, so the
// same bits), forms the word-line branch terms, and walks the segment backwards.  Per node and
// vector the state is read twice and the residual written once (20 bytes, against 36 with phi
// stored per node); the neighbour columns are read by the blocks of columns j +- 1 at about the
// same time and come from L2.
constexpr int kSeg = 4;  // rows per segment of the back walk
constexpr int kFwd = 4;  // segments per batch of loads in the forward walk

__device__ __forceinline__ fp2 phi_step(float2 thc, float2 tha, fp2 phi, fp2 w) {
  // all terms >= 0 along the chain: unnormalised pairs
  return padd_u(pmul_u(fp2{thc.x, thc.y}, phi), pmul_u(fp2{tha.x, tha.y}, w));
}

// one (column, vector) chain of the state: row i at w[i rs + d], d selecting a neighbour column
template <bool kW1>
struct StateCol {
  const float* w1;
  const float2* w2;
  size_t rs;
  __device__ __forceinline__ fp2 at(int i, long d = 0) const {
    const long o = (long)i * (long)rs + d;
    if constexpr (kW1) {
      return fp2{w1[o], 0.0f};
    } else {
      const float2 v = w2[o];
      return {v.x, v.y};
    }
  }
};

// the column's coefficients, staged in shared memory by each block
struct ColCoef {
  const float2 *thc, *tha, *Gc;
  const float* s;
};

// Back walk of one segment (rows i0 .. i0+n-1, kTail: the last, possibly short one).  kNb: which
// word-line neighbours exist (1 left, 2 right, 3 both).
template <bool kW1, int kNb, bool kTail>
__device__ __forceinline__ void back_segment(const ResidParams& p, const ColCoef& c, const StateCol<kW1>& W,
                                             long col, float* rh, fp2 f, int i0, int n, int j, int b, bool src,
                                             fp2 gw, fp2 gs, fp2& u, float& rmax) {
  fp2 wv[kSeg], e[kSeg], ph[kSeg];
  fp2 wl[kSeg], wr[kSeg];
#pragma unroll
  for (int q = 0; q < kSeg; ++q) {
    if (!kTail || q < n) {
      wv[q] = W.at(i0 + q);
      if (kNb & 1) wl[q] = W.at(i0 + q, -col);
      if (kNb & 2) wr[q] = W.at(i0 + q, col);
    }
  }
#pragma unroll
  for (int q = 0; q < kSeg; ++q) {
    if (!kTail || q < n) {
      const int i = i0 + q;
      f = phi_step(c.thc[i], c.tha[i], f, wv[q]);
      if (kTail && p.Vbl && i == p.M - 1 && b < p.B)  // g_o V / d_last, 1/d_last = thc_last / g_b
        f = padd(f, pmul(split(p.go * ((double)c.thc[i].x + (double)c.thc[i].y) / p.gb), split(p.Vbl[(size_t)b * p.N + (p.N - 1 - j)])));
      ph[q] = f;
      // the word-line branches g_w ((w_l - w) + (w_r - w)) and the source branch: terms whose
      // differences cancel, summed in pairs
      if constexpr (kNb == 3) e[q] = pmul_u(gw, pdiff2_u(wl[q], wr[q], wv[q]));
      else if constexpr (kNb == 1) e[q] = pmul_u(gw, psub_u(wl[q], wv[q]));
      else if constexpr (kNb == 2) e[q] = pmul_u(gw, psub_u(wr[q], wv[q]));
      else e[q] = fp2{0.0f, 0.0f};
      if (kNb != 1 && kNb != 3 && src)
        e[q] = padd(e[q], pmul(gs, psub(p.Vbl ? fp2{0.0f, 0.0f} : split(p.V[(size_t)b * p.M + i]), wv[q])));
    }
  }
#pragma unroll
  for (int q = kSeg - 1; q >= 0; --q) {
    if (!kTail || q < n) {
      const int i = i0 + q;
      const float2 t = c.thc[i], g = c.Gc[i];
      u = padd_u(ph[q], pmul_u(fp2{t.x, t.y}, u));
      const float rf = psum_f(pmul_u(fp2{g.x, g.y}, psub_u(u, wv[q])), e[q]);
      rmax = fmaxf(rmax, fabsf(rf));
      rh[(long)i * (long)W.rs] = rf * c.s[i];
    }
  }
}

template <bool kW1, int kNb>
__device__ __forceinline__ void back_walk(const ResidParams& p, const ColCoef& c, const StateCol<kW1>& W, long col,
                                          float* rh, const float2* ph2, int S, int j, int b, fp2& u, float& rmax) {
  const bool src = (kNb == 0 || kNb == 2) && j == 0 && b < p.B;
  const fp2 gw = split(p.gw), gs = split(p.gs);
  const int last = (S - 1) * kSeg;
  auto entry = [&](int s) {
    if (s == 0) return fp2{0.0f, 0.0f};
    const float2 v = ph2[(long)s * (long)W.rs];
    return fp2{v.x, v.y};
  };
  back_segment<kW1, kNb, true>(p, c, W, col, rh, entry(S - 1), last, p.M - last, j, b, src, gw, gs, u, rmax);
  for (int s = S - 2; s >= 0; --s)
    back_segment<kW1, kNb, false>(p, c, W, col, rh, entry(s), s * kSeg, kSeg, j, b, src, gw, gs, u, rmax);
}

template <bool kW1>
__global__ void __launch_bounds__(128, 8) resid_kernel(ResidParams p) {
  if (p.skip && *p.skip) return;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  const size_t base = (size_t)j * p.Mp;
  const int M = p.M, S = (M + kSeg - 1) / kSeg;  // segments; only the last may be short
  // the column's coefficients: thc, tha, Gc pairs and s, 28 bytes per row
  extern __shared__ float2 csm[];
  const ColCoef c{csm, csm + M, csm + 2 * M, reinterpret_cast<const float*>(csm + 3 * M)};
  for (int t = threadIdx.x; t < M; t += blockDim.x) {
    csm[t] = p.thc2[base + t];
    csm[M + t] = p.tha2[base + t];
    csm[2 * M + t] = p.Gc2[base + t];
    reinterpret_cast<float*>(csm + 3 * M)[t] = p.s32[base + t];
  }
  __syncthreads();
  if (b >= p.Bpad) return;
  const size_t rs = p.Bpad, o0 = base * rs + b;
  const StateCol<kW1> W{kW1 ? p.w1 + o0 : nullptr, kW1 ? nullptr : p.w2 + o0, rs};
  float2* ph2 = p.phi2 + o0;  // phi entering segment s (s >= 1) at ph2[s rs]
  // forward walk: segments 0 .. S-2 are full; keep the value entering each segment
  {
    fp2 phi{0.0f, 0.0f};
    for (int s = 0; s + 1 < S; s += kFwd) {
      const int nr = min(kFwd, S - 1 - s) * kSeg, i0 = s * kSeg;
      fp2 wv[kFwd * kSeg];
#pragma unroll
      for (int q = 0; q < kFwd * kSeg; ++q)
        if (q < nr) wv[q] = W.at(i0 + q);
#pragma unroll
      for (int q = 0; q < kFwd * kSeg; ++q) {
        if (q < nr) {
          phi = phi_step(c.thc[i0 + q], c.tha[i0 + q], phi, wv[q]);
          if (q % kSeg == kSeg - 1) ph2[(long)(s + q / kSeg + 1) * (long)rs] = make_float2(phi.hi, phi.lo);
        }
      }
    }
  }
  const bool has_l = j > 0, has_r = j + 1 < p.N;
  const long col = (long)p.Mp * (long)rs;
  float* rh = p.rhat + o0;
  fp2 u{0.0f, 0.0f};
  float rmax = 0.0f;  // |r| tracked in FP32: only its magnitude is reported
  if (has_l && has_r) back_walk<kW1, 3>(p, c, W, col, rh, ph2, S, j, b, u, rmax);
  else if (has_l) back_walk<kW1, 1>(p, c, W, col, rh, ph2, S, j, b, u, rmax);
  else if (has_r) back_walk<kW1, 2>(p, c, W, col, rh, ph2, S, j, b, u, rmax);
  else back_walk<kW1, 0>(p, c, W, col, rh, ph2, S, j, b, u, rmax);
  if (!(rmax <= 3.0e38f)) set_status(p.status, XBAR_DEV_NONFINITE);
  // warp max of |r| over the lanes still running (those past Bpad have left), then one atomic per
  // warp: non-negative floats and doubles order like their bit patterns
  const unsigned live = __activemask();
  rmax = __uint_as_float(__reduce_max_sync(live, __float_as_uint(rmax)));
  if ((threadIdx.x & 31) == __ffs(live) - 1 && p.rmax)
    atomicMax(p.rmax, (unsigned long long)__double_as_longlong((double)rmax));
}

// forward half of the bit-line chain solve in FP64 (node-voltage output):
// phi_i = tha_i w_i + thc_i phi_{i-1}
__device__ __forceinline__ void chain_forward(const ResidParams& p, int j, int b) {
  const size_t base = (size_t)j * p.Mp;
  double phi = 0.0;
  for (int i = 0; i < p.M; ++i) {
    const size_t o = (base + i) * p.Bpad + b;
    phi = fma(p.thc[base + i], phi, p.tha[base + i] * p.w[o]);
    p.phi[o] = phi;
  }
}

// w2 -> w in place (same 8 bytes per entry): each thread converts the entries it reads
__global__ void pair_to_double_kernel(ResidParams p, size_t n) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const float2 v = p.w2[k];
    p.w[k] = (double)v.x + (double)v.y;
  }
}

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

cudaError_t launch_pair_to_double(const ResidParams& p, cudaStream_t st) {
  const size_t n = (size_t)p.N * p.Mp * p.Bpad;
  const int blocks = (int)std::min<size_t>(4096, (n + 255) / 256);
  pair_to_double_kernel<<<blocks, 256, 0, st>>>(p, n);
  return cudaGetLastError();
}

cudaError_t launch_resid(const ResidParams& p, cudaStream_t st) {
  dim3 grid((p.Bpad + 127) / 128, p.N);
  const size_t smem = (size_t)p.M * 28;  // M <= 1024: within the default 48 KB
  if (p.w1) resid_kernel<true><<<grid, 128, smem, st>>>(p);
  else resid_kernel<false><<<grid, 128, smem, st>>>(p);
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
