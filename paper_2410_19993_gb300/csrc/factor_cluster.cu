// factor_cluster.cu -- the block Thomas factorization of factor.cu on a thread-block cluster.
//
// Same mathematics as factor.cu (Z_0 = C_0, Z_j = C_j - g_w^2 X_{j-1}, X_j = Z_j^{-1}, diagonals
// from the grounded row sums sigma_j), for FP32 factors with 32 <= Mp <= 256.  A cluster of C blocks owns
// one map; block g holds rows [g R, (g+1) R) of the current matrix in shared memory (R = 16, C = Mp / R).
// The in-place blocked Gauss-Jordan inversion uses panels of R rows, so panel p is exactly block p's
// rows.  With R_p the owner's rows when panel p starts and D_p^-1 the inverse of their pivot block,
// Gauss-Jordan replaces the owner's rows by D_p^-1 R_p (D_p^-1 in the pivot columns) and every other
// block's rows by  row - W' R_p  (-W' in the pivot columns), W' = row[P] D_p^-1.  So the other blocks
// need only R_p and D_p^-1, not the owner's formed rows: the owner publishes both to its own slot of
// a global (L2-resident) buffer as soon as they exist and signals each peer's mbarrier (arrive with
// release at cluster scope; the peer waits with acquire).  The next owner computes its updated pivot
// block first and inverts it in one warp while its other warps apply the panel (look-ahead), so the
// chain from panel to panel is signal, L2 read, W', max(update, inversion).  (Pulling panels from the
// owner's shared memory instead makes all peers drain one SM's shared-memory port at once and is
// several times slower.)  Every wait is bounded; a block whose wait expires records
// XBAR_DEV_TIMEOUT and stops waiting but keeps the cluster barrier sequence (one per column step).
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace xbar {

namespace {

constexpr int kWork = 256;             // threads of the row work: one per pivot-block element / column
constexpr int kInvWarp = kWork / 32;   // one more warp inverts pivot blocks meanwhile
constexpr int kThreads = kWork + 32;
constexpr int kRows = 16;
static_assert(kWork == kRows * kRows, "one thread per element of a pivot block");

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// mapa: the shared::cluster address of `local` in block `rank` of this cluster
__device__ __forceinline__ uint32_t peer_addr(const void* local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr(local)), "r"(rank));
  return r;
}
// arrive on a peer block's mbarrier; release at cluster scope orders this block's earlier writes
__device__ __forceinline__ void arrive_peer(uint32_t bar_cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster_addr) : "memory");
}
// bounded wait for phase `parity` of a local mbarrier, acquire at cluster scope
__device__ __forceinline__ bool wait_cluster_bounded(uint64_t* bar, unsigned parity, unsigned* status) {
  auto done = [&]() {
    uint32_t d;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(d)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return d != 0;
  };
  if (done()) return true;
  const uint64_t t0 = globaltimer_ns();
  unsigned k = 0;
  while (!done()) {
    if ((++k & 255u) == 0 && globaltimer_ns() - t0 > wait_limit(status)) {
      set_status(status, XBAR_DEV_TIMEOUT);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace

// dynamic shared memory: mbarriers [16 panels + 2 staging], rows [R][Mp], pn [R][Mp], D [R][R],
// Dr [R][R], W [R][R], Bp [R][R], sigv [Mp], sv [Mp], ev [Mp], sg [2][R], then two staging buffers
// (FP64) of a column step's inputs: C_j own rows [R][Mp], s_j [Mp], s_{j-1} [Mp], e_{j-1} [Mp], h_j own rows [R]
size_t factor_cluster_smem_bytes(int Mp, int R) {
  return 18 * sizeof(uint64_t) + ((size_t)2 * R * Mp + 4 * (size_t)R * R + 3 * (size_t)Mp + 2 * R) * sizeof(float) +
         2 * ((size_t)R * Mp + 3 * (size_t)Mp + R) * sizeof(double);
}

// global panel slots, one per block of the cluster: R_p [R][Mp] then D_p^-1 [R][R]
size_t factor_cluster_pbuf_floats(int Mp) {
  const size_t C = (size_t)Mp / kRows;
  return C * ((size_t)kRows * Mp + (size_t)kRows * kRows);
}

// acc[r] (r < 16) += sign * sum_m coef[r*16 + m] * col[m], coefficients read as 16-byte broadcasts
__device__ __forceinline__ void rank16_update(float (&acc)[16], const float* __restrict__ coef,
                                              const float (&col)[16], float sign) {
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const float4* c4 = reinterpret_cast<const float4*>(coef + r * 16);
    float a = acc[r];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 c = c4[q];
      a = fmaf(sign * c.x, col[4 * q], a);
      a = fmaf(sign * c.y, col[4 * q + 1], a);
      a = fmaf(sign * c.z, col[4 * q + 2], a);
      a = fmaf(sign * c.w, col[4 * q + 3], a);
    }
    acc[r] = a;
  }
}

__global__ void __launch_bounds__(kThreads, 1)
    factor_cluster_kernel(const FactorParams<float>* __restrict__ maps, int C, unsigned* status) {
  constexpr int R = kRows;  // rows per block = panel width
  const FactorParams<float> p = maps[blockIdx.x / C];
  const uint32_t g = cluster_rank();
  const int M = p.M, Mp = p.Mp, N = p.N;
  const int r0 = (int)g * R;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t wlim = wait_limit(status);
  constexpr int nwarps = kThreads / 32;

  extern __shared__ __align__(16) unsigned char smraw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smraw);  // [16]: panel p of this column step is ready
  uint64_t* pbar = bars + 16;                            // [2]: staging buffer b has landed
  float* sm = reinterpret_cast<float*>(smraw + 18 * sizeof(uint64_t));
  float* rows = sm;                         // [R][Mp]
  float* pn = rows + (size_t)R * Mp;        // [R][Mp] the current panel's R_p
  float* Dm = pn + (size_t)R * Mp;          // [R][R] inverse of this block's pivot block
  float* Dr = Dm + R * R;                   // [R][R] the current panel's D_p^-1
  float* W = Dr + R * R;                    // [R][R] W' = own rows[P] D_p^-1
  float* Bp = W + R * R;                    // [R][R] next pivot block (look-ahead)
  float* sigv = Bp + R * R;                 // [Mp]
  float* sv = sigv + Mp;                    // [Mp] equilibration scale of column j
  float* ev = sv + Mp;                      // [Mp] coupling to column j-1
  float* sg = ev + Mp;                      // [2][R] sigma of own rows, by step parity
  double* stg = reinterpret_cast<double*>(sg + 2 * R);  // [2] staging buffers (16-byte aligned)
  const size_t stg_n = (size_t)R * Mp + 3 * (size_t)Mp + R;

  if (Mp != C * R || C > 16 || (int)blockDim.x != kThreads) {
    if (tid == 0) set_status(status, XBAR_DEV_BADLAUNCH);
    return;  // uniform across the cluster: every block sees the same arguments
  }
  const float gw = (float)p.gw;
  if (tid < C) mbar_init(&bars[tid], 1);
  if (tid == 0) {
    mbar_init(&pbar[0], 1);
    mbar_init(&pbar[1], 1);
  }
  fence_mbar_init();
  cluster_sync();  // every block's mbarriers are initialised before any peer arrives on them
  // column step jj's inputs (own rows of C_jj, s_jj, s_jj-1, e_jj-1, own h_jj) -> staging buffer jj & 1
  // by bulk copies, one step ahead (thread 0)
  auto stage_inputs = [&](int jj) {
    double* buf = stg + (size_t)(jj & 1) * stg_n;
    uint64_t* bar = &pbar[jj & 1];
    const unsigned cb = (unsigned)(R * Mp * sizeof(double)), vb = (unsigned)(Mp * sizeof(double));
    const unsigned hb = (unsigned)(R * sizeof(double));
    unsigned bytes = cb + hb;
    if (p.s) bytes += vb;
    if (p.s && jj > 0) bytes += vb;
    if (jj > 0) bytes += vb;
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(buf, p.Coff + ((size_t)jj * Mp + r0) * Mp, cb, bar);
    bulk_g2s(buf + (size_t)R * Mp + 3 * Mp, p.h + (size_t)jj * Mp + r0, hb, bar);
    if (p.s) bulk_g2s(buf + (size_t)R * Mp, p.s + (size_t)jj * Mp, vb, bar);
    if (p.s && jj > 0) bulk_g2s(buf + (size_t)R * Mp + Mp, p.s + (size_t)(jj - 1) * Mp, vb, bar);
    if (jj > 0) bulk_g2s(buf + (size_t)R * Mp + 2 * Mp, p.e + (size_t)(jj - 1) * Mp, vb, bar);
  };
  if (tid == 0) stage_inputs(0);
  const size_t slot = (size_t)R * Mp + R * R;  // floats per panel slot
  __shared__ unsigned failed;                  // a wait of this block expired: stop waiting
  if (tid == 0) failed = 0;
  __syncthreads();

  for (int j = 0; j < N; ++j) {
    // this step's inputs from the staging buffer (the next step's copies overlap this step)
    const double* stj = stg + (size_t)(j & 1) * stg_n;
    const double* Cj = stj;                                      // own rows of C_j
    const double* sj = p.s ? stj + (size_t)R * Mp : nullptr;
    const double* sjm = (p.s && j > 0) ? stj + (size_t)R * Mp + Mp : nullptr;
    const double* ejm = j > 0 ? stj + (size_t)R * Mp + 2 * Mp : nullptr;
    const double* hj = stj + (size_t)R * Mp + 3 * Mp;          // own rows: hj[r] is h_j of row r0 + r
    if (tid == 0) {
      if (j + 1 < N) stage_inputs(j + 1);
      if (!failed && !mbar_wait_bounded(&pbar[j & 1], (unsigned)((j >> 1) & 1), status, wlim))
        failed = 1;
    }
    __syncthreads();

    for (int k = tid; k < Mp; k += kThreads) {
      sv[k] = sj ? (float)sj[k] : 1.0f;
      ev[k] = ejm ? (float)ejm[k] : 0.0f;
    }
    // (1) sigma_j of own rows: h_j + g_w S X^_{j-1} S sigma_{j-1}  (X^_{j-1} own rows are in `rows`)
    if (j > 0) {
      const float* sp = p.sig + (size_t)((j - 1) & 1) * Mp;
      for (int k = tid; k < Mp; k += kThreads) sigv[k] = __ldcg(sp + k) * (sjm ? (float)sjm[k] : 1.0f);
      __syncthreads();
      for (int r = warp; r < R; r += nwarps) {
        const int i = r0 + r;
        float acc = 0.0f;
        for (int k = lane; k < Mp; k += 32) acc = fmaf(rows[(size_t)r * Mp + k], sigv[k], acc);
        acc = warp_sum_f(acc);
        if (lane == 0)
          sg[(j & 1) * R + r] = (i < M) ? (float)hj[r] + gw * (sjm ? (float)sjm[i] : 1.0f) * acc : 0.0f;
      }
    } else {
      for (int r = tid; r < R; r += kThreads) {
        const int i = r0 + r;
        sg[r] = (i < M) ? (float)(hj[r] + p.gsrc) : 0.0f;
      }
    }
    __syncthreads();
    for (int r = tid; r < R; r += kThreads) p.sig[(size_t)(j & 1) * Mp + r0 + r] = sg[(j & 1) * R + r];

    // (2) + (3) Z^_j own rows (off-diagonal, then the subtraction-free diagonal) in place of
    // X^_{j-1}, whose own rows go to the output on the way: each element of `rows` is read, stored
    // to X and overwritten by the same thread, so no thread can overwrite an element of X^_{j-1}
    // before it has been stored
    float* Xo = j > 0 ? p.X + (size_t)(j - 1) * Mp * Mp + (size_t)r0 * Mp : nullptr;
    for (int t = tid * 2; t < R * Mp; t += kThreads * 2) {
      const int r = t / Mp, k = t - r * Mp, i = r0 + r;
      const double2 c2 = *reinterpret_cast<const double2*>(Cj + t);
      const float si = sv[i], ei = ev[i];
      const float x0 = j > 0 ? rows[t] : 0.0f, x1 = j > 0 ? rows[t + 1] : 0.0f;  // X^_{j-1}
      if (j > 0) *reinterpret_cast<float2*>(Xo + t) = make_float2(x0, x1);
      float v0 = 0.0f, v1 = 0.0f;
      if (i < M) {
        if (k < M && k != i) v0 = si * sv[k] * (float)c2.x - ei * ev[k] * x0;
        if (k + 1 < M && k + 1 != i) v1 = si * sv[k + 1] * (float)c2.y - ei * ev[k + 1] * x1;
      }
      rows[t] = v0;
      rows[t + 1] = v1;
    }
    __syncthreads();
    for (int r = warp; r < R; r += nwarps) {
      const int i = r0 + r;
      float acc = 0.0f;
      for (int k = lane; k < M; k += 32) acc += fabsf(rows[(size_t)r * Mp + k]) / sv[k];
      acc = warp_sum_f(acc);
      if (lane == 0) {
        float d = 1.0f;
        if (i < M) {
          const float si = sv[i];
          d = si * si * (sg[(j & 1) * R + r] + (j < N - 1 ? gw : 0.0f)) + si * acc;
        }
        rows[(size_t)r * Mp + i] = d;
      }
    }
    __syncthreads();

    // (4) blocked Gauss-Jordan inversion; panel p = rows of block p.
    // Pivot blocks are inverted in one warp's registers (Gauss-Jordan, no pivoting: the block is
    // symmetric positive definite).  Lane l holds column l % 16 of rows 8 (l / 16) .. + 7; each
    // pivot's row, column and diagonal arrive by shuffles.
    static_assert(R == 16, "register layout assumes 16 x 16 pivot blocks");
    const int pb = lane & 15, pa0 = (lane >> 4) * 8;
    float* myslot = p.pbuf + (size_t)g * slot;  // R_g then D_g^-1
    auto invert_publish = [&](float (&d)[8]) {  // warp kInvWarp: D^-1 to Dm and to this block's slot
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int qe = q & 7, qlane = (q >> 3) << 4;
        const float piv = __shfl_sync(0xffffffffu, d[qe], qlane | q);   // D[q][q]
        const float rowq = __shfl_sync(0xffffffffu, d[qe], qlane | pb);  // D[q][b]
        float colq[8];                                                   // D[a0 + e][q]
#pragma unroll
        for (int e = 0; e < 8; ++e) colq[e] = __shfl_sync(0xffffffffu, d[e], (lane & 16) | q);
        const float ri = __fdividef(1.0f, piv);
        // column q: -D[a][q] / piv; elsewhere D[a][b] - D[a][q] D[q][b] / piv; row q: D[q][b] / piv
        const bool incol = pb == q;
        const float f = incol ? ri : rowq * ri;
#pragma unroll
        for (int e = 0; e < 8; ++e) d[e] = fmaf(-colq[e], f, incol ? 0.0f : d[e]);
        if ((lane & 16) == qlane) d[qe] = f;  // the half-warp holding row q
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        Dm[(pa0 + e) * R + pb] = d[e];
        myslot[(size_t)R * Mp + (pa0 + e) * R + pb] = d[e];
      }
    };
    auto signal_peers = [&]() {  // after a __syncthreads that follows every write of the slot
      if (tid < C && tid != (int)g) arrive_peer(peer_addr(&bars[g], (uint32_t)tid));
    };
    for (int pp = 0; pp < C; ++pp) {
      const int P0 = pp * R;
      if ((int)g == pp) {
        if (pp == 0) {  // later owners published while applying the previous panel
          if (warp == kInvWarp) {
            float d[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) d[e] = rows[(size_t)(pa0 + e) * Mp + P0 + pb];
            invert_publish(d);
          } else {
            for (int t = tid; t < R * Mp / 4; t += kWork)
              reinterpret_cast<float4*>(myslot)[t] = reinterpret_cast<const float4*>(rows)[t];
          }
          __syncthreads();
          signal_peers();
        }
        // own rows become the panel rows: D^-1 R outside the pivot columns, D^-1 inside
        for (int k = tid; k < Mp && tid < kWork; k += kWork) {
          float col[R], acc[R];
          const bool kin = (k >= P0 && k < P0 + R);
#pragma unroll
          for (int m = 0; m < R; ++m) {
            col[m] = rows[(size_t)m * Mp + k];
            acc[m] = 0.0f;
          }
          rank16_update(acc, Dm, col, 1.0f);
#pragma unroll
          for (int r = 0; r < R; ++r) rows[(size_t)r * Mp + k] = kin ? Dm[r * R + (k - P0)] : acc[r];
        }
        __syncthreads();
      } else {
        // wait for panel pp, then read R_pp and D_pp^-1 from its slot (L2)
        bool ok = true;
        if (tid == 0 && !failed) {
          ok = wait_cluster_bounded(&bars[pp], (unsigned)(j & 1), status);
          if (!ok) failed = 1;
        }
        __syncthreads();
        // D_pp^-1 to shared memory first; R_pp into registers, stored after W' (its latency overlaps W')
        const float4* src = reinterpret_cast<const float4*>(p.pbuf + (size_t)pp * slot);
        if (tid < R * R / 4) reinterpret_cast<float4*>(Dr)[tid] = __ldcg(src + R * Mp / 4 + tid);
        constexpr int kPer = (kRows * 16 * kRows / 4 + kWork - 1) / kWork;  // float4 per thread, Mp <= 16 R
        float4 rp[kPer];
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
          const int t = tid + u * kWork;
          if (tid < kWork && t < R * Mp / 4) rp[u] = __ldcg(src + t);
        }
        __syncthreads();
        if (tid < kWork) {  // W' = own rows[P] D_pp^-1, one element per thread
          const int a = tid >> 4, bcol = tid & 15;
          float w = 0.0f;
#pragma unroll
          for (int m = 0; m < R; ++m) w = fmaf(rows[(size_t)a * Mp + P0 + m], Dr[m * R + bcol], w);
          W[tid] = w;
#pragma unroll
          for (int u = 0; u < kPer; ++u) {
            const int t = tid + u * kWork;
            if (t < R * Mp / 4) reinterpret_cast<float4*>(pn)[t] = rp[u];
          }
        }
        __syncthreads();
        const bool ahead = (int)g == pp + 1;  // owner of the next panel
        const int P1 = P0 + R;
        if (ahead) {  // its pivot block after this panel, same operation order as the update below
          if (tid < kWork) {
            const int a = tid >> 4, bcol = tid & 15;
            float v = rows[(size_t)a * Mp + P1 + bcol];
#pragma unroll
            for (int m = 0; m < R; ++m) v = fmaf(-1.0f * W[a * R + m], pn[(size_t)m * Mp + P1 + bcol], v);
            Bp[tid] = v;
          }
          __syncthreads();
        }
        if (ahead && warp == kInvWarp) {
          float d[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) d[e] = Bp[(pa0 + e) * R + pb];
          invert_publish(d);
        } else {
          //   row <- row - W' R_pp outside the pivot columns, -W' inside; the next owner also
          //   publishes its updated rows as R_{pp+1}
          for (int k = tid; k < Mp && tid < kWork; k += kWork) {
            float col[R], acc[R];
            const bool kin = (k >= P0 && k < P0 + R);  // R_pp holds D there, not D^-1: the result is -W'
#pragma unroll
            for (int m = 0; m < R; ++m) {
              col[m] = pn[(size_t)m * Mp + k];
              acc[m] = rows[(size_t)m * Mp + k];
            }
            rank16_update(acc, W, col, -1.0f);
#pragma unroll
            for (int r = 0; r < R; ++r) {
              if (kin) acc[r] = -W[r * R + (k - P0)];
              rows[(size_t)r * Mp + k] = acc[r];
            }
            if (ahead)
#pragma unroll
              for (int r = 0; r < R; ++r) myslot[(size_t)r * Mp + k] = acc[r];
          }
        }
        __syncthreads();
        if (ahead) signal_peers();
      }
    }
    cluster_sync();  // every read of this step's slots is done before the next step rewrites them
  }
  {
    float* Xo = p.X + (size_t)(N - 1) * Mp * Mp + (size_t)r0 * Mp;
    for (int t = tid; t < R * Mp; t += kThreads) Xo[t] = rows[t];
  }
  cluster_sync();  // no block leaves while another may still read its shared memory
}

bool factor_cluster_supported(int Mp) { return Mp >= 2 * kRows && Mp <= 16 * kRows && Mp % kRows == 0; }

int factor_cluster_size(int Mp) { return Mp / kRows; }

cudaError_t launch_factor_cluster(const FactorParams<float>* maps_dev, int nmaps, int Mp, unsigned* status,
                                  cudaStream_t st) {
  const int C = factor_cluster_size(Mp);
  const size_t smem = factor_cluster_smem_bytes(Mp, kRows);
  cudaError_t err = cudaFuncSetAttribute(factor_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  if (C > 8) {
    err = cudaFuncSetAttribute(factor_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (err != cudaSuccess) return err;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nmaps * C);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, factor_cluster_kernel, maps_dev, C, status);
}

}  // namespace xbar
