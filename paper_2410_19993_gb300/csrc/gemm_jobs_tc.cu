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
// Roles: 12 producer warps copy the FP32 slabs of A (128 rows x 16)
// and B (TN columns x 16) for either storage order, split them and store the terms in the no-swizzle
// K-major core-matrix layout of the MMA (8 rows x 16 bytes per core matrix) into a ring of stages;
// the next warp issues the MMAs from one thread and frees each stage with tcgen05.commit; the last
// four drain the accumulator (tcgen05.ld, lane = row), apply C = Cin + alpha D and store.  The accumulator is
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
constexpr int kEpi = 4;
// producer warps: the 32-item groups of a chunk (8 of A, TN / 16 of B) are dealt round-robin
__host__ __device__ constexpr int ngroups(int TN) { return 8 + TN / 16; }
#ifndef XBAR_GTC_NP256
#define XBAR_GTC_NP256 12
#endif
#ifndef XBAR_GTC_NP128
#define XBAR_GTC_NP128 12
#endif
#ifndef XBAR_GTC_NS256
#define XBAR_GTC_NS256 3
#endif
#ifndef XBAR_GTC_RS256
#define XBAR_GTC_RS256 2
#endif
#ifndef XBAR_GTC_SPIN_NS
#define XBAR_GTC_SPIN_NS 0
#endif
__host__ __device__ constexpr int nprod(int TN) { return TN == 256 ? XBAR_GTC_NP256 : XBAR_GTC_NP128; }
__host__ __device__ constexpr int nthreads(int TN) { return (nprod(TN) + 1 + kEpi) * 32; }
__host__ __device__ constexpr int groups_per_warp(int TN) { return (ngroups(TN) + nprod(TN) - 1) / nprod(TN); }
constexpr uint32_t kAterm = 2 * (kTM / 8) * 128;  // one BF16 term of the A slab: 4 KB
__host__ __device__ constexpr uint32_t bterm(int TN) { return 2u * (TN / 8) * 128; }
__host__ __device__ constexpr uint32_t stage_bytes(int TN) { return 3 * kAterm + 3 * bterm(TN); }
__host__ __device__ constexpr int nstages(int TN) { return TN == 256 ? XBAR_GTC_NS256 : 3; }
// Raw FP32 slabs arrive by cp.async into a ring of RS stages.  Every producer warp has a private
// slice of each stage: per group of 32 items (rows of A or columns of B) 8 K values each, either as
// [item][k] at a pitch of 12 floats (K contiguous in the source; the pitch keeps 16-byte reads of
// consecutive items in different banks) or as [k][item] (items contiguous in the source).  Either
// order fits the same 384 floats, so a warp never touches another warp's bytes, whichever
// operand order the chunks of different segments use.
constexpr int kPitch = 12;
constexpr uint32_t kGroupFloats = 32 * kPitch;  // >= 8 x 32
__host__ __device__ constexpr uint32_t warp_raw_floats(int TN) { return kGroupFloats * groups_per_warp(TN); }
__host__ __device__ constexpr uint32_t raw_bytes(int TN) { return (uint32_t)nprod(TN) * warp_raw_floats(TN) * 4; }
__host__ __device__ constexpr int rstages(int TN) { return TN == 256 ? XBAR_GTC_RS256 : 3; }
constexpr uint32_t kHdr = 1024;  // barriers and flags
// epilogue transpose buffers: per epilogue warp 32 rows x 32 columns at a pitch of 36 floats
constexpr int kEpiPitch = 36;
constexpr uint32_t kEpiBytes = kEpi * 32 * kEpiPitch * 4;
__host__ __device__ constexpr size_t smem_bytes(int TN) {
  return kHdr + (size_t)nstages(TN) * stage_bytes(TN) + (size_t)rstages(TN) * raw_bytes(TN) + kEpiBytes;
}

// 16-byte asynchronous copy global -> shared (L2 only); src_bytes = 0 fills zeros
__device__ __forceinline__ void cp_async16(void* dst, const void* src, unsigned src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// named barrier over the 8 producer warps; the _or form also returns whether any thread passed true
__device__ __forceinline__ void prod_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ bool prod_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, 256, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// x = x0 + x1 + x2 for 8 values -> three 16-byte rows of BF16, each term rounded to nearest (the
// differences are exact in FP32; |x - x0 - x1 - x2| <= 2^-24 |x| or so).  A pair of elements is
// converted by one cvt.rn.bf16x2; the FP32 values of the rounded terms are read back from the packed
// word with a shift and a mask.
__device__ __forceinline__ uint32_t bf16x2_rn(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ void split8(const float (&v)[8], uint4 (&o)[3]) {
  uint32_t w[3][4];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    const uint32_t p0 = bf16x2_rn(v[e], v[e + 1]);
    const float ra = v[e] - __uint_as_float(p0 << 16), rb = v[e + 1] - __uint_as_float(p0 & 0xffff0000u);
    const uint32_t p1 = bf16x2_rn(ra, rb);
    const float sa = ra - __uint_as_float(p1 << 16), sb = rb - __uint_as_float(p1 & 0xffff0000u);
    w[0][e / 2] = p0;
    w[1][e / 2] = p1;
    w[2][e / 2] = bf16x2_rn(sa, sb);
  }
#pragma unroll
  for (int t = 0; t < 3; ++t) o[t] = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
}

}  // namespace gtc

template <int TN>
__global__ void __launch_bounds__(gtc::nthreads(TN), 1)
    gemm_jobs_tc_kernel(const GemmJob<float>* __restrict__ jobs, int njobs, int m, int n, int tiles_n,
                        unsigned* status) {
  using namespace gtc;
  constexpr int NS = nstages(TN), NP = nprod(TN);
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
      mbar_init(&full[s], nprod(TN));
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

  if (warp < NP) {
    // ---- producers -------------------------------------------------------------------------------
    // The chunk's items (A: 128 rows, B: TN columns, each 16 K values) form 32-item groups with one
    // K octet each: A group a < 8 holds rows 32 (a % 4) .. +31, octet a / 4; B group b holds columns
    // 32 (b % (TN/32)) .. +31, octet b / (TN/32).  Warp w owns groups w, w + NP, ...: it copies by
    // cp.async exactly the raw FP32 values of its groups, D = RS - 1 chunks ahead, into its own slice
    // of raw stage c % RS ([item][k] at a pitch of 12 floats when K is contiguous in the source,
    // [k][item] otherwise).  Nothing crosses warps, so a warp needs only its own wait_group and
    // __syncwarp before splitting: the warps run independently.  The split writes three BF16 terms
    // in the MMA's K-major core-matrix layout; lane 0 of each warp then arrives on the stage's
    // barrier.
    constexpr int RS = rstages(TN), D = RS - 1, GPW = groups_per_warp(TN), NG = ngroups(TN);
    float* raw = reinterpret_cast<float*>(stages + (size_t)NS * SB) + (size_t)warp * warp_raw_floats(TN);
    constexpr uint32_t RSF = raw_bytes(TN) / 4;  // floats per raw stage (all warps)
    struct Cursor {
      int t, s, k0, nseg, K, i0, j0, lda, ldb, ta, tb;
      const float* A;
      const float* B;
    };
    auto load_seg = [&](Cursor& q) {
      int job;
      tile_of(q.t, job, q.i0, q.j0);
      const GemmJob<float>& jb = jobs[job];
      q.nseg = jb.nseg;
      q.K = jb.k[q.s];
      q.A = jb.A[q.s];
      q.B = jb.B[q.s];
      q.lda = jb.lda[q.s];
      q.ldb = jb.ldb[q.s];
      q.ta = jb.ta[q.s];
      q.tb = jb.tb[q.s];
    };
    auto advance = [&](Cursor& q) {
      q.k0 += kKC;
      if (q.k0 < q.K) return;
      q.k0 = 0;
      if (++q.s >= q.nseg) {
        q.s = 0;
        q.t += gridDim.x;
      }
      if (q.t < ntiles) load_seg(q);
    };
    // group g -> operand (A: g < 8), first item within the tile, K octet
    auto group = [&](int g, bool& isA, int& base, int& oc) {
      isA = g < 8;
      if (isA) {
        base = 32 * (g & 3);
        oc = g >> 2;
      } else {
        const int b = g - 8;
        base = 32 * (b % (TN / 32));
        oc = b / (TN / 32);
      }
    };
    // Copies of this warp's groups for the chunk at the `ahead` cursor.  Per group and lane two
    // 16-byte granules: K contiguous in the source -> item 16 u + lane / 2, granule lane % 2 of the
    // octet, stored [item][k] at a pitch of 12 floats; otherwise K row 4 u + lane / 8, item granule
    // lane % 8, stored [k][item].  Source addresses are formed once per segment (set_groups) and
    // advance by a fixed stride per chunk.
    const float* gptr[GPW][2];
    long long gstep[GPW];
    uint32_t gdst[GPW][2], gbytes[GPW][2];
    auto set_groups = [&](const Cursor& q) {
#pragma unroll
      for (int gi = 0; gi < GPW; ++gi) {
        const int g = warp + NP * gi;
        bool isA;
        int base, oc;
        group(g < NG ? g : 0, isA, base, oc);
        const float* src = isA ? q.A : q.B;
        const int ld = isA ? q.lda : q.ldb;
        const int kcontig = isA ? !q.ta : q.tb;
        const int first = (isA ? q.i0 : q.j0) + base, nitems = isA ? m : n;
        gstep[gi] = kcontig ? kKC : (long long)kKC * ld;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          if (kcontig) {
            const int it = 16 * u + (lane >> 1), kg = lane & 1, x = first + it;
            gptr[gi][u] = src + (size_t)(x < nitems ? x : 0) * ld + q.k0 + 8 * oc + 4 * kg;
            gdst[gi][u] = it * kPitch + 4 * kg;
            gbytes[gi][u] = x < nitems ? 16u : 0u;
          } else {
            const int e = 4 * u + (lane >> 3), ig = lane & 7, x = first + 4 * ig;
            gptr[gi][u] = src + (size_t)(q.k0 + 8 * oc + e) * ld + (x < nitems ? x : 0);
            gdst[gi][u] = e * 32 + 4 * ig;
            gbytes[gi][u] = x < nitems ? 16u : 0u;
          }
        }
      }
    };
    auto issue = [&](const Cursor& q, int rs) {
      if (q.t >= ntiles) return;
      float* w = raw + (size_t)rs * RSF;
#pragma unroll
      for (int gi = 0; gi < GPW; ++gi) {
        if (warp + NP * gi >= NG) break;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          cp_async16(w + kGroupFloats * gi + gdst[gi][u], gptr[gi][u], gbytes[gi][u]);
          gptr[gi][u] += gstep[gi];
        }
      }
    };
    // the ahead cursor: a new segment or tile re-forms the group addresses
    auto advance_ahead = [&](Cursor& q) {
      const int s0 = q.s, t0 = q.t;
      advance(q);
      if (q.t < ntiles && (q.s != s0 || q.t != t0)) set_groups(q);
    };
    // the 8 K values of this lane's item in a group (layout as copied)
    auto read_group = [&](const float* src, int kcontig, float (&v)[8]) {
      if (kcontig) {
        const float4 x = *reinterpret_cast<const float4*>(src + lane * kPitch);
        const float4 y = *reinterpret_cast<const float4*>(src + lane * kPitch + 4);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w; v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = src[e * 32 + lane];
      }
    };
    Cursor ahead;
    ahead.t = blockIdx.x;
    ahead.s = 0;
    ahead.k0 = 0;
    if (ahead.t < ntiles) {
      load_seg(ahead);
      set_groups(ahead);
    }
    Cursor cur = ahead;
#pragma unroll 1
    for (int r = 0; r < D; ++r) {
      issue(ahead, r);
      cp_async_commit();
      if (ahead.t < ntiles) advance_ahead(ahead);
    }
    int st = 0, use = 0;
    long long c = 0;
    while (cur.t < ntiles) {
      issue(ahead, (int)((c + D) % RS));  // this warp's slice, last read while splitting chunk c - 1
      cp_async_commit();
      if (ahead.t < ntiles) advance_ahead(ahead);
      cp_async_wait<D>();  // this lane's copies of chunk c have landed
      __syncwarp();        // ... and every lane's, visible to the whole warp
      bool ok = true;
      if (lane == 0 && c >= NS)
        ok = mbar_spin_bounded(&empty[st], (unsigned)((use - 1) & 1), status, limit, XBAR_GTC_SPIN_NS);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok || *fail) {
        *fail = 1;
        break;
      }
      const float* w = raw + (size_t)(c % RS) * RSF;
      unsigned char* sb = stages + (size_t)st * SB;
#pragma unroll
      for (int gi = 0; gi < GPW; ++gi) {
        const int g = warp + NP * gi;
        if (g >= NG) break;
        bool isA;
        int base, oc;
        group(g, isA, base, oc);
        const int it = base + lane;  // this lane's item (row of A or column of B)
        float v[8];
        read_group(w + kGroupFloats * gi, isA ? !cur.ta : cur.tb, v);
        uint4 t3[3];
        split8(v, t3);
        if (isA) {
          const uint32_t off = (uint32_t)oc * (kTM / 8) * 128 + (uint32_t)(it >> 3) * 128 + (uint32_t)(it & 7) * 16;
#pragma unroll
          for (int q = 0; q < 3; ++q) *reinterpret_cast<uint4*>(sb + q * kAterm + off) = t3[q];
        } else {
          const uint32_t off =
              3 * kAterm + (uint32_t)oc * (TN / 8) * 128 + (uint32_t)(it >> 3) * 128 + (uint32_t)(it & 7) * 16;
#pragma unroll
          for (int q = 0; q < 3; ++q) *reinterpret_cast<uint4*>(sb + off + q * BT) = t3[q];
        }
      }
      fence_proxy_async_smem();
      __syncwarp();  // the warp's reads of its raw slice and its BF16 stores are done
      if (lane == 0) mbar_arrive(&full[st]);
      if (++st == NS) { st = 0; ++use; }
      ++c;
      advance(cur);
    }
    cp_async_wait<0>();  // no copy of this block may still be in flight when it exits
  } else if (warp == NP) {
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
            if (!mbar_spin_bounded(&full[st], (unsigned)(use & 1), status, limit, XBAR_GTC_SPIN_NS) || *fail) {
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
    // Each 32 x 32 block of the accumulator goes through this warp's shared-memory buffer, so that
    // C (and Cin) are accessed as 4 rows x 128 contiguous bytes per warp instruction.
    const int quarter = warp & 3;
    float* tb32 = reinterpret_cast<float*>(smem + smem_bytes(TN) - kEpiBytes) + (warp - NP - 1) * 32 * kEpiPitch;
    int lt = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
      int job, i0, j0;
      tile_of(t, job, i0, j0);
      const GemmJob<float>& jb = jobs[job];
      const int ab = lt & 1;
      if (!mbar_spin_bounded(&tfull[ab], (unsigned)((lt >> 1) & 1), status, limit, 64) || *fail) break;
      umma::fence_after();
      const float alpha = jb.alpha;
      float* C = jb.C;
      const float* Cin = jb.Cin;
      const int ldc = jb.ldc, ldcin = jb.ldcin;
      const int rsub = lane >> 3, c4 = (lane & 7) * 4;  // transposed access: row 4 it + rsub, columns c4..c4+3
#pragma unroll 1
      for (int cc = 0; cc < TN; cc += 32) {
        float v[32];
        umma::ld32(tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ab * TN + cc), v);
#pragma unroll
        for (int e = 0; e < 32; e += 4)
          *reinterpret_cast<float4*>(tb32 + lane * kEpiPitch + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
        __syncwarp();
        const int gj = j0 + cc + c4;
#pragma unroll
        for (int it = 0; it < 8; ++it) {
          const int r = 4 * it + rsub, gi = i0 + quarter * 32 + r;
          const float4 a = *reinterpret_cast<const float4*>(tb32 + r * kEpiPitch + c4);
          if (gi < m) {
            if (gj + 4 <= n) {
              float4 o = make_float4(alpha * a.x, alpha * a.y, alpha * a.z, alpha * a.w);
              if (Cin) {
                const float4 ci = *reinterpret_cast<const float4*>(Cin + (size_t)gi * ldcin + gj);
                o.x += ci.x; o.y += ci.y; o.z += ci.z; o.w += ci.w;
              }
              *reinterpret_cast<float4*>(C + (size_t)gi * ldc + gj) = o;
            } else {
              const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
              for (int e = 0; e < 4; ++e)
                if (gj + e < n) C[(size_t)gi * ldc + gj + e] = alpha * av[e] + (Cin ? Cin[(size_t)gi * ldcin + gj + e] : 0.0f);
            }
          }
        }
        __syncwarp();  // the buffer is rewritten by the next block
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
  kern<<<grid, tn == 256 ? gtc::nthreads(256) : gtc::nthreads(128), smem, st>>>(jobs_dev, njobs, m, n, tiles_n,
                                                                                status);
  return cudaGetLastError();
}

}  // namespace xbar
