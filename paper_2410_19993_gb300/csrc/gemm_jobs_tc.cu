// gemm_jobs_tc.cu -- job-list GEMMs of the cyclic-reduction factor on the tcgen05 tensor cores.
//
// The dense work of each reduction level is a batch of independent products of M x M blocks
// (couplings P = D^-1 L and Q = D^-1 U, Schur complements D - U P, the next level's couplings
// U Q, and the products of the 2 x 2 block inversion).  This kernel runs one such batch: a
// persistent grid over the SMs walks the 128 x TN output tiles of all jobs.
//
// Precision.  The operands are FP32; each K slab is split while it is staged into three BF16
// terms, x = x0 + x1 + x2 (each rounded to nearest; the differences are exact in FP32), and every
// K step of 16 issues the six products A_s B_t with s + t <= 2 into one FP32 accumulator in tensor
// memory (kind::f16).  The dropped products are below 2^-24 relative, so the result carries
// FP32-level accuracy, which the factor's refinement relies on; all operands of the factor are
// entrywise non-negative or non-positive blocks, so no product cancels.
//
// Roles (416 threads): warps 0-7 load the FP32 slabs of A (128 rows x 16) and B (TN columns x 16)
// with coalesced loads for either storage order, split them and store the terms in the no-swizzle
// K-major core-matrix layout of the MMA (8 rows x 16 bytes per core matrix) into a ring of stages;
// warp 8 issues the MMAs from one thread and frees each stage with tcgen05.commit; warps 9-12 drain
// the accumulator (tcgen05.ld, lane = row), apply C = Cin + alpha D and store.  The accumulator is
// double-buffered in tensor memory (2 TN columns), so one tile's epilogue overlaps the next tile's
// MMAs.  Every wait is bounded (XBAR_DEV_TIMEOUT); on expiry a role stops, and the MMA thread waits
// for its own issued MMAs before the block frees tensor memory.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "umma.cuh"

namespace xbar {

namespace gtc {
constexpr int kTM = 128, kKC = 16;
constexpr int kProd = 8, kEpi = 4;
constexpr int kThreads = (kProd + 1 + kEpi) * 32;
constexpr uint32_t kAterm = 2 * (kTM / 8) * 128;  // one BF16 term of the A slab: 4 KB
__host__ __device__ constexpr uint32_t bterm(int TN) { return 2u * (TN / 8) * 128; }
__host__ __device__ constexpr uint32_t stage_bytes(int TN) { return 3 * kAterm + 3 * bterm(TN); }
__host__ __device__ constexpr int nstages(int TN) { return TN == 256 ? 5 : 8; }
constexpr uint32_t kHdr = 1024;  // barriers and flags
__host__ __device__ constexpr size_t smem_bytes(int TN) { return kHdr + (size_t)nstages(TN) * stage_bytes(TN); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// x = x0 + x1 + x2 for 8 values -> three 16-byte rows of BF16
__device__ __forceinline__ void split8(const float (&v)[8], uint4 (&o)[3]) {
  uint32_t w[3][4];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(v[e], v[e + 1]);
    const float ra = v[e] - __low2float(h0), rb = v[e + 1] - __high2float(h0);
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(ra, rb);
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(ra - __low2float(h1), rb - __high2float(h1));
    w[0][e / 2] = *reinterpret_cast<const uint32_t*>(&h0);
    w[1][e / 2] = *reinterpret_cast<const uint32_t*>(&h1);
    w[2][e / 2] = *reinterpret_cast<const uint32_t*>(&h2);
  }
#pragma unroll
  for (int t = 0; t < 3; ++t) o[t] = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
}

}  // namespace gtc

template <int TN>
__global__ void __launch_bounds__(gtc::kThreads, 1)
    gemm_jobs_tc_kernel(const GemmJob<float>* __restrict__ jobs, int njobs, int m, int n, int tiles_n,
                        unsigned* status) {
  using namespace gtc;
  constexpr int NS = nstages(TN);
  constexpr uint32_t SB = stage_bytes(TN);
  constexpr uint32_t BT = bterm(TN);
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);  // [NS]   producer warps -> MMA
  uint64_t* empty = full + 8;                          // [NS]   MMA commit -> producers
  uint64_t* tfull = full + 16;                         // [2]    accumulator ready
  uint64_t* tempty = full + 18;                        // [2]    accumulator drained
  uint64_t* drain = full + 20;                         // [1]    MMA teardown
  uint32_t* tslot = reinterpret_cast<uint32_t*>(full + 21);
  volatile unsigned* fail = reinterpret_cast<volatile unsigned*>(full + 22);
  unsigned char* stages = smem + kHdr;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_m = (m + kTM - 1) / kTM;
  const int tpj = tiles_m * tiles_n;
  const int ntiles = njobs * tpj;
  const uint64_t limit = wait_limit(status);

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], kProd);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], kEpi);
    }
    mbar_init(drain, 1);
    *fail = 0;
    fence_mbar_init();
  }
  if (warp == 0) umma::alloc(tslot, 2 * TN);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tbase = *tslot;

  // tile t -> (job, i0, j0)
  auto tile_of = [&](int t, int& job, int& i0, int& j0) {
    job = t / tpj;
    const int r = t - job * tpj;
    i0 = (r / tiles_n) * kTM;
    j0 = (r % tiles_n) * TN;
  };

  if (warp < kProd) {
    // ---- producers: load, split and stage the A and B slabs --------------------------------------
    // The raw values of the next K slab are loaded before the current one is split and stored, so
    // their latency overlaps that work and the wait for a free stage.
    const int pt = tid;  // 0..255
    struct Pos {
      int t, s, k0;
    };
    auto valid = [&](const Pos& q) { return q.t < ntiles; };
    auto next = [&](Pos q) {
      const GemmJob<float>& jb = jobs[q.t / tpj];
      q.k0 += kKC;
      if (q.k0 >= jb.k[q.s]) {
        q.k0 = 0;
        if (++q.s >= jb.nseg) {
          q.s = 0;
          q.t += gridDim.x;
        }
      }
      return q;
    };
    auto load = [&](const Pos& q, float (&av)[8], float (&bv)[TN / 128][8]) {
      int job, i0, j0;
      tile_of(q.t, job, i0, j0);
      const GemmJob<float>& jb = jobs[job];
      const float* A = jb.A[q.s];
      const float* B = jb.B[q.s];
      const int lda = jb.lda[q.s], ldb = jb.ldb[q.s], ta = jb.ta[q.s], tb = jb.tb[q.s];
      {
        const int r = pt & 127, o = pt >> 7;  // A item: row r, K octet o
        const int gi = i0 + r, gk = q.k0 + 8 * o;
        if (gi < m) {
          if (!ta) {
            const float4* src = reinterpret_cast<const float4*>(A + (size_t)gi * lda + gk);
            const float4 x = src[0], y = src[1];
            av[0] = x.x; av[1] = x.y; av[2] = x.z; av[3] = x.w;
            av[4] = y.x; av[5] = y.y; av[6] = y.z; av[7] = y.w;
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) av[e] = A[(size_t)(gk + e) * lda + gi];
          }
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) av[e] = 0.0f;
        }
      }
#pragma unroll
      for (int u = 0; u < TN / 128; ++u) {  // B items: column col, K octet o
        const int item = pt + 256 * u;
        const int col = item % TN, o = item / TN;
        const int gj = j0 + col, gk = q.k0 + 8 * o;
        if (gj < n) {
          if (tb) {
            const float4* src = reinterpret_cast<const float4*>(B + (size_t)gj * ldb + gk);
            const float4 x = src[0], y = src[1];
            bv[u][0] = x.x; bv[u][1] = x.y; bv[u][2] = x.z; bv[u][3] = x.w;
            bv[u][4] = y.x; bv[u][5] = y.y; bv[u][6] = y.z; bv[u][7] = y.w;
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) bv[u][e] = B[(size_t)(gk + e) * ldb + gj];
          }
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) bv[u][e] = 0.0f;
        }
      }
    };
    int st = 0, use = 0;
    long long c = 0;
    Pos cur{(int)blockIdx.x, 0, 0};
    float av[8], bv[TN / 128][8], av2[8], bv2[TN / 128][8];
    if (valid(cur)) load(cur, av, bv);
    while (valid(cur)) {
      const Pos nx = next(cur);
      if (valid(nx)) load(nx, av2, bv2);
      if (c >= NS && !mbar_spin_bounded(&empty[st], (unsigned)((use - 1) & 1), status, limit, 32)) {
        *fail = 1;
        break;
      }
      if (*fail) break;
      unsigned char* sb = stages + (size_t)st * SB;
      {
        const int r = pt & 127, o = pt >> 7;
        uint4 w[3];
        split8(av, w);
        const uint32_t off = (uint32_t)o * (kTM / 8) * 128 + (uint32_t)(r >> 3) * 128 + (uint32_t)(r & 7) * 16;
#pragma unroll
        for (int q = 0; q < 3; ++q) *reinterpret_cast<uint4*>(sb + q * kAterm + off) = w[q];
      }
#pragma unroll
      for (int u = 0; u < TN / 128; ++u) {
        const int item = pt + 256 * u;
        const int col = item % TN, o = item / TN;
        uint4 w[3];
        split8(bv[u], w);
        const uint32_t off =
            3 * kAterm + (uint32_t)o * (TN / 8) * 128 + (uint32_t)(col >> 3) * 128 + (uint32_t)(col & 7) * 16;
#pragma unroll
        for (int q = 0; q < 3; ++q) *reinterpret_cast<uint4*>(sb + off + q * BT) = w[q];
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[st]);
      if (++st == NS) { st = 0; ++use; }
      ++c;
      cur = nx;
#pragma unroll
      for (int e = 0; e < 8; ++e) av[e] = av2[e];
#pragma unroll
      for (int u = 0; u < TN / 128; ++u)
#pragma unroll
        for (int e = 0; e < 8; ++e) bv[u][e] = bv2[u][e];
    }
  } else if (warp == kProd) {
    // ---- MMA issuer --------------------------------------------------------------------------------
    if (lane == 0) {
      constexpr uint32_t idesc = umma::idesc_bf16(kTM, TN);
      const uint32_t sbase = smem_addr(stages);
      int st = 0, use = 0, lt = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++lt) {
        int job, i0, j0;
        tile_of(t, job, i0, j0);
        const GemmJob<float>& jb = jobs[job];
        const int ab = lt & 1;
        if (lt >= 2 && !mbar_spin_bounded(&tempty[ab], (unsigned)(((lt >> 1) - 1) & 1), status, limit, 0)) {
          ok = false;
          break;
        }
        umma::fence_after();
        const uint32_t dt = tbase + (uint32_t)(ab * TN);
        bool first = true;
        for (int s = 0; s < jb.nseg && ok; ++s) {
          for (int k0 = 0; k0 < jb.k[s]; k0 += kKC) {
            if (!mbar_spin_bounded(&full[st], (unsigned)(use & 1), status, limit, 0) || *fail) {
              ok = false;
              break;
            }
            umma::fence_after();
            const uint32_t sa = sbase + (uint32_t)st * SB;
            const uint32_t sbb = sa + 3 * kAterm;
            uint64_t ad[3], bd[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              ad[q] = umma::sdesc(sa + q * kAterm, (kTM / 8) * 128, 128);
              bd[q] = umma::sdesc(sbb + q * BT, (TN / 8) * 128, 128);
            }
            umma::mma_bf16(dt, ad[0], bd[0], idesc, first ? 0u : 1u);
            umma::mma_bf16(dt, ad[0], bd[1], idesc, 1u);
            umma::mma_bf16(dt, ad[1], bd[0], idesc, 1u);
            umma::mma_bf16(dt, ad[0], bd[2], idesc, 1u);
            umma::mma_bf16(dt, ad[1], bd[1], idesc, 1u);
            umma::mma_bf16(dt, ad[2], bd[0], idesc, 1u);
            first = false;
            umma::commit(&empty[st]);
            if (++st == NS) { st = 0; ++use; }
          }
        }
        if (!ok) break;
        umma::commit(&tfull[ab]);
      }
      if (!ok) {
        *fail = 1;
        // wait for every MMA issued so far before the block may free tensor memory
        umma::commit(drain);
        mbar_wait_bounded(drain, 0u, status, limit);
        for (int a = 0; a < 2; ++a) mbar_arrive(&tfull[a]);  // release waiting epilogue warps
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue: TMEM lane quarter (warp % 4) = 32 rows of the tile ------------------------------
    const int quarter = warp & 3;
    const int r = quarter * 32 + lane;
    int lt = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
      int job, i0, j0;
      tile_of(t, job, i0, j0);
      const GemmJob<float>& jb = jobs[job];
      const int ab = lt & 1;
      if (!mbar_spin_bounded(&tfull[ab], (unsigned)((lt >> 1) & 1), status, limit, 64) || *fail) break;
      umma::fence_after();
      const int gi = i0 + r;
      const float alpha = jb.alpha;
      float* crow = jb.C + (size_t)gi * jb.ldc;
      const float* cin = jb.Cin ? jb.Cin + (size_t)gi * jb.ldcin : nullptr;
#pragma unroll 1
      for (int cc = 0; cc < TN; cc += 32) {
        float v[32];
        umma::ld32(tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ab * TN + cc), v);
        const int gj = j0 + cc;
        if (gi < m) {
          if (gj + 32 <= n) {
#pragma unroll
            for (int e = 0; e < 32; e += 4) {
              float4 o = make_float4(alpha * v[e], alpha * v[e + 1], alpha * v[e + 2], alpha * v[e + 3]);
              if (cin) {
                const float4 ci = *reinterpret_cast<const float4*>(cin + gj + e);
                o.x += ci.x; o.y += ci.y; o.z += ci.z; o.w += ci.w;
              }
              *reinterpret_cast<float4*>(crow + gj + e) = o;
            }
          } else {
#pragma unroll
            for (int e = 0; e < 32; ++e)
              if (gj + e < n) crow[gj + e] = alpha * v[e] + (cin ? cin[gj + e] : 0.0f);
          }
        }
      }
      umma::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[ab]);
    }
  }
  // ---- teardown --------------------------------------------------------------------------------------
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  if (warp == 0) umma::dealloc(tbase, 2 * TN);
}

cudaError_t launch_gemm_jobs_tc(const GemmJob<float>* jobs_dev, int njobs, int m, int n, int tn, int nsm,
                                unsigned* status, cudaStream_t st) {
  if (njobs <= 0 || m <= 0 || n <= 0) return cudaSuccess;
  if (tn != 128 && tn != 256) return cudaErrorInvalidValue;
  const int tiles_m = (m + gtc::kTM - 1) / gtc::kTM, tiles_n = (n + tn - 1) / tn;
  const long long ntiles = (long long)njobs * tiles_m * tiles_n;
  if (ntiles > (1ll << 30)) return cudaErrorInvalidValue;
  const int grid = (int)(ntiles < nsm ? ntiles : nsm);
  const size_t smem = gtc::smem_bytes(tn);
  auto kern = tn == 256 ? gemm_jobs_tc_kernel<256> : gemm_jobs_tc_kernel<128>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  kern<<<grid, gtc::kThreads, smem, st>>>(jobs_dev, njobs, m, n, tiles_n, status);
  return cudaGetLastError();
}

}  // namespace xbar
