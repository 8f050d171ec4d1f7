// sweep.cu -- forward and back substitution over a batch of input vectors (Sec. II-C: L y = I,
// U V = y for every right-hand side; Sec. III-A: one decomposition serves the whole batch),
// followed by extraction of the bit-line currents.
//
// With the block Thomas factor X_j of the word-line system (factor.cu), the substitutions are
//     forward   z_0 = X_0 r_0,      z_j = X_j (r_j + e_{j-1} o z_{j-1})     j = 1 .. N-1
//     back      w_{N-1} = z_{N-1},  w_j = z_j + X_j (e_j o w_{j+1})          j = N-2 .. 0
//     currents  I_j = hs_j . w_j
// where e_j is the (equilibrated) coupling between columns j and j+1 and r the right-hand side
// (for an input vector V only r_0 = src o V is nonzero; refinement passes give a full r).  Every
// step is a dense (Mp x Mp) x (Mp x Bp) product over a panel of Bp input vectors, so one block
// owns one panel and walks all 2N-1 steps; z_j goes to global memory between the two sweeps.
//
// Data movement: X_j is streamed through shared memory in chunks of KC rows by the bulk-copy
// (TMA) engine, double-buffered and completed on mbarriers with bounded waits; the running
// vector of the panel stays in shared memory; each thread accumulates a TR x TC register tile.
//
// Two tilings.  Wide panels use 8 x 4 (FP64) or 8 x 8 (FP32) register tiles.  A panel of a small
// batch would then be one or two warps, each warp's FMAs issued on a single SM sub-partition (for
// FP64, a quarter of the SM's DFMA rate), with most of a TC-wide tile spent on padding columns.
// So when the wide tiling gives fewer than four warps the kernel runs with 2 x 1 tiles instead and
// the panel is exactly ceil(B / SMs) vectors wide: a batch of one is Mp/2 threads.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace xbar {

template <typename T>
struct SweepCfg;
template <>
struct SweepCfg<float> { static constexpr int TR = 8, TC = 8, KC = 32; };
template <>
struct SweepCfg<double> { static constexpr int TR = 8, TC = 4, KC = 16; };

// the narrow tiling (all precisions)
constexpr int kNarrowTR = 2, kNarrowTC = 1;
constexpr int kMinWarps = 4;
// threads per block: at most 512 for the wide tilings (128 registers each), 1024 for the narrow one
template <int TR, int TC>
constexpr int sweep_max_threads() { return TR * TC >= 8 ? 512 : 1024; }

template <typename T>
static bool sweep_is_narrow(int Mp, int Bp) {
  constexpr int TR = SweepCfg<T>::TR, TC = SweepCfg<T>::TC;
  return Bp % TC != 0 || (Mp / TR) * (Bp / TC) < 32 * kMinWarps;
}

template <typename T>
static size_t sweep_smem_bytes(int Mp, int Bp, int KC, int TR) {
  const int nrg = Mp / TR;
  size_t n = (size_t)Mp * Bp + 2 * (size_t)KC * Mp + (size_t)nrg * Bp;
  return n * sizeof(T) + 64;
}

// rows of X_j per bulk copy: the largest of {KC, 16, 8} that divides Mp (8 for very tall blocks)
template <typename T>
static int sweep_kc(int Mp) {
  if (Mp >= 512) return 8;
  int kc = SweepCfg<T>::KC;
  while (kc > 8 && Mp % kc) kc /= 2;
  return kc;
}

template <typename T>
int sweep_panel_width(int Mp, int B, int nsm) {
  constexpr int TR = SweepCfg<T>::TR, TC = SweepCfg<T>::TC;
  const int nrg = Mp / TR;
  const int kc = sweep_kc<T>(Mp);
  const int per_sm = std::max(1, (B + nsm - 1) / nsm);
  int bp = ((per_sm + TC - 1) / TC) * TC;
  constexpr int wide_max = sweep_max_threads<TR, TC>(), narrow_max = sweep_max_threads<kNarrowTR, kNarrowTC>();
  // threads within the launch bound and shared memory <= 200 KB
  while (bp > TC && (nrg * (bp / TC) > wide_max || sweep_smem_bytes<T>(Mp, bp, kc, TR) > 200 * 1024)) bp -= TC;
  if (!sweep_is_narrow<T>(Mp, bp)) return bp;
  // fewer than four warps: narrow tiles, no padding columns.  Every width up to bp is narrow too
  // ((Mp/TR)*(Bp/TC) only grows with Bp), so launch_sweep picks the same tiling from (Mp, Bp).
  int nb = std::min(per_sm, bp);
  while (nb > 1 && ((Mp / kNarrowTR) * nb > narrow_max || sweep_smem_bytes<T>(Mp, nb, kc, kNarrowTR) > 200 * 1024))
    --nb;
  return nb;
}

// n consecutive elements from shared memory: 16-byte loads when the run is a multiple of 16 bytes
// (and then 16-byte aligned), element loads otherwise
template <typename T, int n>
__device__ __forceinline__ void load_vec(T (&r)[n], const T* p) {
  if constexpr ((n * sizeof(T)) % 16 == 0) {
    constexpr int per = 16 / sizeof(T);
#pragma unroll
    for (int q = 0; q < n / per; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(p + q * per);
      memcpy(&r[q * per], &v, 16);
    }
  } else {
#pragma unroll
    for (int q = 0; q < n; ++q) r[q] = p[q];
  }
}

template <typename T, int TR, int TC>
__global__ void __launch_bounds__(sweep_max_threads<TR, TC>()) sweep_kernel(SweepParams<T> p, int KC) {
  const int Mp = p.Mp, N = p.N, Bp = p.Bp, Bpad = p.Bpad;
  const int nrg = Mp / TR, ncg = Bp / TC;
  const int tid = threadIdx.x;
  const uint64_t wlim = wait_limit(p.status);  // read once: the waits below sit on critical paths
  const int rg = tid / ncg, cg = tid - rg * ncg;
  const int i0 = rg * TR, c0 = cg * TC;
  const int b0 = blockIdx.x * Bp;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw);                  // 2 mbarriers
  T* xs = reinterpret_cast<T*>(smem_raw + 64);                             // [2][KC][Mp]
  T* vin = xs + 2 * (size_t)KC * Mp;                                       // [Mp][Bp]
  T* red = vin + (size_t)Mp * Bp;                                          // [nrg][Bp]

  if (p.skip && *p.skip) return;
  if (nrg * ncg != (int)blockDim.x || b0 + Bp > Bpad) {
    if (tid == 0) set_status(p.status, XBAR_DEV_BADLAUNCH);
    return;
  }

  const int chunks_per_step = Mp / KC;
  const int nsteps = 2 * N - 1;
  const long long nchunks = (long long)nsteps * chunks_per_step;
  const unsigned chunk_bytes = (unsigned)(KC * Mp * sizeof(T));
  auto chunk_src = [&](long long c) -> const T* {
    const int s = (int)(c / chunks_per_step);
    const int k0 = (int)(c - (long long)s * chunks_per_step) * KC;
    const int j = s < N ? s : 2 * N - 2 - s;
    return p.X + ((size_t)j * Mp + k0) * Mp;
  };

  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(&mbar[0], chunk_bytes);
    bulk_g2s(xs, chunk_src(0), chunk_bytes, &mbar[0]);
  }

  // input of step 0
  const T* r0 = p.rhs;
#pragma unroll
  for (int a = 0; a < TR; ++a) {
    const int i = i0 + a;
#pragma unroll
    for (int c = 0; c < TC; ++c) {
      const int b = b0 + c0 + c;
      T v;
      if (p.V) v = (i < p.M && b < p.B) ? p.src[i] * (T)p.V[(size_t)b * p.M + i] : (T)0;
      else v = r0[(size_t)i * Bpad + b];
      vin[(size_t)i * Bp + c0 + c] = v;
    }
  }
  __syncthreads();

  T acc[TR][TC];
  long long c = 0;
  float local_max = 0.0f;
  for (int s = 0; s < nsteps; ++s) {
    const bool fwd = s < N;
    const int j = fwd ? s : 2 * N - 2 - s;
#pragma unroll
    for (int a = 0; a < TR; ++a)
#pragma unroll
      for (int b = 0; b < TC; ++b) acc[a][b] = (T)0;

    for (int kc = 0; kc < chunks_per_step; ++kc, ++c) {
      if (tid == 0 && c + 1 < nchunks) {
        const int nb = (int)((c + 1) & 1);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&mbar[nb], chunk_bytes);
        bulk_g2s(xs + (size_t)nb * KC * Mp, chunk_src(c + 1), chunk_bytes, &mbar[nb]);
      }
      const bool ok = mbar_wait_bounded(&mbar[c & 1], (unsigned)((c >> 1) & 1), p.status,
                                        wlim);
      if (__syncthreads_or(!ok)) return;
      const T* xb = xs + (size_t)(c & 1) * KC * Mp;
      const T* vb = vin + (size_t)kc * KC * Bp;
#pragma unroll 4
      for (int k = 0; k < KC; ++k) {
        T xr[TR], vr[TC];
        load_vec<T, TR>(xr, xb + (size_t)k * Mp + i0);
        load_vec<T, TC>(vr, vb + (size_t)k * Bp + c0);
#pragma unroll
        for (int a = 0; a < TR; ++a)
#pragma unroll
          for (int b = 0; b < TC; ++b) acc[a][b] = fma(xr[a], vr[b], acc[a][b]);
      }
      __syncthreads();  // xs[c & 1] and (last chunk) vin are free again
    }

    // ---- epilogue of step s ------------------------------------------------------------------
    const size_t rowbase = (size_t)j * Mp;
    if (fwd) {
#pragma unroll
      for (int a = 0; a < TR; ++a)
#pragma unroll
        for (int b = 0; b < TC; ++b) p.z[(rowbase + i0 + a) * Bpad + b0 + c0 + b] = acc[a][b];
    } else {
#pragma unroll
      for (int a = 0; a < TR; ++a)
#pragma unroll
        for (int b = 0; b < TC; ++b) acc[a][b] += p.z[(rowbase + i0 + a) * Bpad + b0 + c0 + b];
    }
    const bool have_w = !fwd || s == N - 1;  // w_{N-1} = z_{N-1}
    if (have_w) {
      if (p.w) {
#pragma unroll
        for (int a = 0; a < TR; ++a)
#pragma unroll
          for (int b = 0; b < TC; ++b) p.w[(rowbase + i0 + a) * Bpad + b0 + c0 + b] = acc[a][b];
      }
      // currents: I_j[b] = sum_i hs_j[i] w_j[i][b]
      T part[TC];
#pragma unroll
      for (int b = 0; b < TC; ++b) part[b] = (T)0;
#pragma unroll
      for (int a = 0; a < TR; ++a) {
        const T hv = p.hs[rowbase + i0 + a];
#pragma unroll
        for (int b = 0; b < TC; ++b) part[b] = fma(hv, acc[a][b], part[b]);
      }
      // when whole warps hold whole column groups (ncg divides 32) the lanes of one column group
      // are summed by shuffles first and one partial per warp goes through shared memory
      const bool wred = (blockDim.x & 31) == 0 && (32 % ncg) == 0;
      int nq = nrg;
      if (wred) {
        const int lane = tid & 31;
#pragma unroll
        for (int b = 0; b < TC; ++b)
          for (int o = 16; o >= ncg; o >>= 1) part[b] += __shfl_xor_sync(0xffffffffu, part[b], o);
        if (lane < ncg) {
#pragma unroll
          for (int b = 0; b < TC; ++b) red[(size_t)(tid >> 5) * Bp + c0 + b] = part[b];
        }
        nq = blockDim.x >> 5;
      } else {
#pragma unroll
        for (int b = 0; b < TC; ++b) red[(size_t)rg * Bp + c0 + b] = part[b];
      }
      __syncthreads();
      for (int t = tid; t < Bp; t += blockDim.x) {
        T sum = 0;
        for (int q = 0; q < nq; ++q) sum += red[(size_t)q * Bp + t];
        const int b = b0 + t;
        if (b < p.B) {
          double* Ip = p.I + (size_t)b * N + j;
          const double dI = (double)sum;
          if (!isfinite(dI)) set_status(p.status, XBAR_DEV_NONFINITE);
          if (p.accumulate) {
            const double In = *Ip + dI;
            *Ip = In;
            const double rel = fabs(dI) / fmax(fabs(In), 1e-300);
            local_max = fmaxf(local_max, (float)rel);
          } else {
            *Ip = dI;
          }
        }
      }
    }
    // input of step s+1
    if (s + 1 < nsteps) {
      const bool nfwd = s + 1 < N;
      const int jn = nfwd ? s + 1 : 2 * N - 3 - s;  // column of the next step
      const int jc = nfwd ? j : jn;                 // coupling index: e_{j} (fwd) or e_{jn} (bwd)
      const T* ev = p.e + (size_t)jc * Mp;
      const T* rn = (nfwd && p.rhs) ? p.rhs + (size_t)jn * Mp * Bpad : nullptr;
#pragma unroll
      for (int a = 0; a < TR; ++a) {
        const int i = i0 + a;
        const T ei = ev[i];
#pragma unroll
        for (int b = 0; b < TC; ++b) {
          T v = ei * acc[a][b];
          if (rn) v += rn[(size_t)i * Bpad + b0 + c0 + b];
          vin[(size_t)i * Bp + c0 + b] = v;
        }
      }
    }
    __syncthreads();
  }
  if (p.max_rel) {
    for (int o = 16; o > 0; o >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    if ((tid & 31) == 0 && local_max > 0.0f) atomic_max_nonneg(p.max_rel, local_max);
  }
}

template <typename T, int TR, int TC>
static cudaError_t launch_tiled(const SweepParams<T>& p, int KC, cudaStream_t st) {
  if (p.Mp % TR || p.Bp % TC || p.Mp % KC) return cudaErrorInvalidValue;
  const int threads = (p.Mp / TR) * (p.Bp / TC);
  if (threads > sweep_max_threads<TR, TC>()) return cudaErrorInvalidConfiguration;
  const int blocks = (p.B + p.Bp - 1) / p.Bp;
  if (blocks == 0) return cudaSuccess;
  if ((long long)blocks * p.Bp > p.Bpad) return cudaErrorInvalidValue;
  const size_t smem = sweep_smem_bytes<T>(p.Mp, p.Bp, KC, TR);
  cudaError_t err = cudaFuncSetAttribute(sweep_kernel<T, TR, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  sweep_kernel<T, TR, TC><<<blocks, threads, smem, st>>>(p, KC);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sweep(const SweepParams<T>& p, cudaStream_t st) {
  if (p.Mp <= 0 || p.Bp <= 0) return cudaErrorInvalidValue;
  const int KC = sweep_kc<T>(p.Mp);
  if (sweep_is_narrow<T>(p.Mp, p.Bp)) return launch_tiled<T, kNarrowTR, kNarrowTC>(p, KC, st);
  return launch_tiled<T, SweepCfg<T>::TR, SweepCfg<T>::TC>(p, KC, st);
}

template int sweep_panel_width<float>(int, int, int);
template int sweep_panel_width<double>(int, int, int);
template cudaError_t launch_sweep<float>(const SweepParams<float>&, cudaStream_t);
template cudaError_t launch_sweep<double>(const SweepParams<double>&, cudaStream_t);

}  // namespace xbar
