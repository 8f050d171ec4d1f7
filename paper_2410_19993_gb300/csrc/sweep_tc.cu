// sweep_tc.cu -- forward/back substitution on the 5th-generation tensor cores (tcgen05).
//
// Same recurrences as sweep.cu (Sec. II-C substitutions after block Thomas):
//     z_0 = X_0 r_0,  z_j = X_j (r_j + e_{j-1} o z_{j-1});   w_{N-1} = z_{N-1},
//     w_j = z_j + X_j (e_j o w_{j+1});   I_j = hs_j . w_j,
// for a panel of 64 input vectors per block.  Each step is D[Mt x 64] = X_j[Mt x Mt] . v[Mt x 64]
// computed from three-term BF16 splits (x = x0 + x1 + x2, each BF16: together 24+ significant bits,
// FP32-level accuracy; a plain BF16 or TF32 product would cost the refinement extra passes).  With
// KP leading terms used, each K step of 16 issues A_p v_q for every p + q < KP (N = 64 each) into
// one FP32 accumulator: (A0 + A1 + A2)(v0 + v1 + v2) without A1 v2, A2 v1, A2 v2 (each below
// 2^-26 relative) for KP = 3, A0 v0 + A0 v1 + A1 v0 (~2^-17) for KP = 2.  One accumulator leaves
// the epilogue a single tensor-memory read per column block on its critical path.
// Against a split-TF32 product (x = hi + lo, four K=8 products per 16 K) this moves 6 instead of
// 8 bytes per element of X_j, issues 96 instead of 128 MMAs per step and does 25% less tensor work.
//
// Operands.  A = X_j, split and pre-tiled in global memory (sweep_tc_tile_kernel) in the
// no-swizzle K-major core-matrix order of the MMA (8 rows x 16 bytes per core matrix), chunk by
// chunk of 16 K-elements (one MMA K step), the three parts adjacent, so one 1-D bulk copy per chunk
// lands MMA-ready data in shared memory.  B = the running vector of the panel, written by the
// epilogue threads in MN-major core-matrix order (8 nodes x 8 columns per core matrix, columns
// contiguous), so each thread stores 8 columns of its node at once.  D = tcgen05 tensor memory,
// one 192-column slab per 128-row half of X_j.
//
// z (the forward result kept for the back substitution) never leaves this kernel, so it is stored
// in the order the epilogue holds it -- thread = row, four columns per 16-byte access -- as
// z[j][panel][column/4][row][4]: a warp's access then covers 512 contiguous bytes instead of 32
// rows 32 KB apart.
//
// Roles: a producer warp streams the chunks through a ring of stages (one 1-D bulk copy each,
// completion on mbarriers) as far ahead as free stages allow; one thread of the MMA warp issues
// the MMAs, frees each stage with tcgen05.commit and signals the finished D; 8 epilogue warps
// (named barrier 1, which neither of the others joins) drain D from tensor memory, write the next
// step's vector split into hi/lo and release the next step's MMAs (mbarrier, one arrival per warp)
// before the work the next step does not need -- z and w stores, current dot products by warp
// transpose-reduction -- so that this work overlaps the next step's MMAs.  Every wait is bounded;
// on expiry the block records XBAR_DEV_TIMEOUT, drains and frees its tensor memory before returning.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "kernels.h"
#include "umma.cuh"

namespace xbar {

namespace tc {

constexpr int kBP = 64;       // input vectors per panel
constexpr int kKC = 16;       // K elements per bulk-copied chunk (one BF16 MMA K step)
constexpr int kParts = 3;     // x = x0 + x1 + x2
constexpr int kThreads = 256;
// B operand = [v0 | v1 | v2] stacked along N (24 groups of 8 columns), MN-major: a core matrix is 8
// nodes x 8 consecutive columns (16 bytes), so a thread (= node) writes 8 columns per 16-byte store;
// node groups of 8 are 128 bytes apart, column groups (Mt/8)*128 bytes apart
__host__ __device__ constexpr uint32_t lbo_b(int Mt) { return (uint32_t)(Mt / 8) * 128; }  // column-group stride
// tensor-memory columns for NH halves of KP * 64 columns (allocations are powers of two >= 32)
// two accumulators (steps alternate) of NH x 64 columns each.  (Issuing A_0 [v_0 | v_1] as one
// N = 128 product, with the epilogue adding the two 64-column halves, reads A_0 once per K step
// instead of twice, but the extra accumulator reads on the epilogue's critical path cost more:
// measured 5% slower per step.)
__host__ __device__ constexpr uint32_t tmem_cols(int NH) { return NH == 1 ? 128u : 256u; }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// 32 consecutive 32-bit TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// x = x0 + x1 + x2 + O(2^-27 |x|), each term BF16 rounded to nearest (the differences are exact in FP32)
__device__ __forceinline__ void split3(float x, __nv_bfloat16& x0, __nv_bfloat16& x1, __nv_bfloat16& x2) {
  x0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(x0);
  x1 = __float2bfloat16_rn(r1);
  x2 = __float2bfloat16_rn(r1 - __bfloat162float(x1));
}

// sum over the 32 lanes of column `lane` of v[0..31] (v is destroyed)
__device__ __forceinline__ float transpose_sum32(float (&v)[32], int lane) {
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const bool up = (lane & w) != 0;
#pragma unroll
    for (int m = 0; m < w; ++m) {
      const float send = up ? v[m] : v[m + w];
      const float keep = up ? v[m + w] : v[m];
      v[m] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
  }
  return v[0];
}

}  // namespace tc

// X_j (FP32 [N][Mp][Mp]) -> three-term BF16 split in the MMA's chunked core-matrix order
// Xt[j][kc][part][kcol][g][r][e], kc < Mt/16, part < 3, kcol < 2, g < Mt/8, r < 8, e < 8;
// element (row n, column k) of X_j with n = 8g + r, k = 16 kc + 8 kcol + e; rows/cols >= Mp are zero.
__global__ void sweep_tc_tile_kernel(const float* __restrict__ X, __nv_bfloat16* __restrict__ Xt, int Mp, int Mt,
                                     int N) {
  const size_t per = (size_t)Mt * Mt;
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= per * N) return;
  const int j = (int)(idx / per);
  const int rem = (int)(idx - (size_t)j * per);
  const int n = rem / Mt, k = rem - n * Mt;
  const float x = (n < Mp && k < Mp) ? X[((size_t)j * Mp + n) * Mp + k] : 0.0f;
  __nv_bfloat16 x0, x1, x2;
  tc::split3(x, x0, x1, x2);
  const int kc = k / tc::kKC, kk = k % tc::kKC, kcol = kk / 8, e = kk % 8, g = n / 8, r = n % 8;
  const size_t part = (size_t)2 * (Mt / 8) * 64;  // elements in one part of a chunk
  const size_t base = ((size_t)j * (Mt / tc::kKC) + kc) * tc::kParts * part;
  const size_t off = ((size_t)kcol * (Mt / 8) + g) * 64 + r * 8 + e;
  Xt[base + off] = x0;
  Xt[base + part + off] = x1;
  Xt[base + 2 * part + off] = x2;
}

// named barrier over the 8 epilogue warps (the producer warp never joins it)
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ bool epi_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, 256, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

// Operand stages: each holds tc_sub consecutive 16-wide K chunks, a chunk slot only the KP terms a
// sweep copies, so there is one full/empty hand-off (wait, fence, commit) per tc_sub chunks; as many
// stages (2 to 8) as the shared memory beside the KP-term vector operand holds.  (Five stages of two
// chunks for a two-term 256-row step ran no faster than two of four: the ring is not what limits
// the K loop.)
__host__ __device__ constexpr int tc_sub(int Mt, int KP) { return (Mt == 256 && KP == 3) ? 2 : 4; }
__host__ __device__ constexpr uint32_t tc_slot(int Mt, int KP) { return (uint32_t)KP * tc::kKC * Mt * 2; }
__host__ __device__ constexpr int tc_vbytes(int Mt, int KP) { return KP * (tc::kBP / 8) * (int)tc::lbo_b(Mt); }
// 32 floats per epilogue thread: with 256-row blocks, the second 32-column block of the next step's
// z or right-hand side, copied in ahead of the accumulator wait; in every sweep, the staging of the
// w tiles (4 KB per warp) between those copies
__host__ __device__ constexpr int tc_prebytes(int Mt) { return tc::kThreads * 32 * 4; }
__host__ __device__ constexpr int tc_fixed(int Mt, int KP) { return 2304 + tc_vbytes(Mt, KP) + tc_prebytes(Mt); }
__host__ __device__ constexpr int tc_stages(int Mt, int KP) {
  return (232448 - tc_fixed(Mt, KP)) / (int)(tc_sub(Mt, KP) * tc_slot(Mt, KP)) > 8
             ? 8
             : (232448 - tc_fixed(Mt, KP)) / (int)(tc_sub(Mt, KP) * tc_slot(Mt, KP));
}
static_assert(tc_stages(256, 1) == 5 && tc_stages(256, 2) == 2 && tc_stages(256, 3) == 2 &&
                  tc_stages(128, 2) == 5 && tc_stages(128, 3) == 3,
              "stage rings");

// NH = number of 128-row halves of X_j (Mt = 128 NH); KP = number of BF16 terms of the split used
// (1..3; the tiles always hold three, a sweep with fewer copies and multiplies only the leading
// ones).  Every size the MMA issue loop touches is a compile-time constant: the single issuing
// thread then spends no dependent integer work per MMA (runtime offsets in that loop tripled its
// cost per MMA).
template <int NH, int KP>
__global__ void __launch_bounds__(tc::kThreads + 64, 1)
    sweep_tc_kernel(SweepParams<float> p, const __nv_bfloat16* __restrict__ Xt) {
  using namespace tc;
  constexpr int BP = kBP, KC = kKC;
  constexpr int Mt = 128 * NH, nh = NH;
  constexpr int NS = tc_stages(Mt, KP), kSub = tc_sub(Mt, KP);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b0 = blockIdx.x * BP;
  const uint64_t wlim = wait_limit(p.status);  // read once: the waits below sit on critical paths

  const int N = p.N, Mp = p.Mp, Bpad = p.Bpad;

  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);  // [NS]
  uint64_t* empty = full + 8;                          // [NS]
  uint64_t* dfull = full + 16;                         // [1] D of the step is complete
  uint64_t* vfull = full + 17;                         // [1] v of the step is written (8 warp arrivals)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(full + 18);
  unsigned* fail = reinterpret_cast<unsigned*>(full + 19);
  float* red = reinterpret_cast<float*>(smem + 256);   // [8][64]
  unsigned char* xs = smem + 256 + 8 * 64 * 4;         // [NS stages][hi | lo]
  constexpr uint32_t part_bytes = (uint32_t)KC * Mt * 2;  // one BF16 part of a chunk
  constexpr uint32_t chunk_bytes = kParts * part_bytes;
  constexpr uint32_t slot_bytes = tc_slot(Mt, KP);  // one chunk's KP terms in shared memory
  constexpr uint32_t stage_bytes = kSub * slot_bytes;
  static_assert((Mt / KC) % kSub == 0, "a stage must not span two column steps");
  unsigned char* vb = xs + (size_t)NS * stage_bytes;   // 8 KP column groups of lbo_b(Mt) bytes: [v0 | v1 | v2]
  constexpr uint32_t LBO_B = lbo_b(Mt);
  // [8 float4][kThreads]: thread t's 16-byte piece k at k * kThreads + t (conflict-free reads)
  float4* pres = reinterpret_cast<float4*>(vb + tc_vbytes(Mt, KP));

  constexpr int cps = Mt / KC;  // chunks per step
  const int nsteps = 2 * N - 1;
  const long long nchunks = (long long)nsteps * cps;
  // accumulators: per 128-row half, 64 columns; two sets, for even and odd steps, so that the
  // epilogue can re-read this step's D while the next step's MMAs accumulate into the other set
  constexpr uint32_t ncols = tmem_cols(NH);
  constexpr int dcols = BP;
  constexpr uint32_t dset = NH * dcols;
  constexpr uint32_t copy_bytes = KP * part_bytes;  // leading KP terms of each chunk
  constexpr uint32_t kBMajorMN = 1u << 16;          // instruction descriptor: B is MN-major
  constexpr uint32_t LBO_A = (uint32_t)(Mt / 8) * 128, SBO = 128;

  if (p.skip && *p.skip) return;  // uniform: before any barrier or tensor-memory allocation
  if ((int)blockDim.x != kThreads + 64 || b0 + BP > Bpad) {
    if (tid == 0) set_status(p.status, XBAR_DEV_BADLAUNCH);
    return;
  }
  if (tid == 0) {
    for (int st = 0; st < NS; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    mbar_init(dfull, 1);
    mbar_init(vfull, kThreads / 32);
    *fail = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tslot, ncols);
    tmem_relinquish();
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = *tslot;

  if (warp == 8) {
    // ---- producer: stream X chunks into the stage ring, as far ahead as free stages allow ----
    if (lane == 0) {
      long long issued = 0;
      int st = 0, use = 0, s = 0, kc = 0;  // stage, uses of this stage so far, step, chunk in step
      const long long nstg = nchunks / kSub;  // cps is a multiple of kSub: a stage never spans two steps
      for (long long c = 0; c < nstg; ++c) {
        if (c >= NS && !mbar_spin_bounded(&empty[st], (unsigned)((use - 1) & 1), p.status, wlim, 0))
          break;
        issued = c + 1;
        const int j = s < N ? s : 2 * N - 2 - s;
        mbar_arrive_expect_tx(&full[st], kSub * copy_bytes);
#pragma unroll
        for (int sub = 0; sub < kSub; ++sub)
          bulk_g2s(xs + (size_t)st * stage_bytes + sub * slot_bytes,
                   Xt + ((size_t)j * cps + kc + sub) * (chunk_bytes / 2), copy_bytes, &full[st]);
        kc += kSub;
        if (kc == cps) { kc = 0; ++s; }
        if (++st == NS) { st = 0; ++use; }
      }
      // before the block may exit: the last copy into each stage has landed (bounded wait)
      for (long long c = (issued > NS ? issued - NS : 0); c < issued; ++c)
        mbar_wait_bounded(&full[c % NS], (unsigned)((c / NS) & 1), p.status, wlim);
    }
    __syncwarp();
  } else if (warp == 9) {
    // ---- MMA issuer: step s starts once the epilogue has written its v (and read step s-1's D) ----
    if (lane == 0) {
      // stage ring position and descriptors (descriptor address fields are the low bits, so stage /
      // half / lo offsets are plain adds)
      int mst = 0, muse = 0;
      const uint64_t adesc0 = umma::sdesc(smem_addr(xs), LBO_A, SBO);
      // MN-major, no swizzle: the descriptor's leading byte offset is the stride between groups of
      // 8 nodes (K), the stride byte offset the stride between groups of 8 columns (N)
      const uint64_t bdesc0 = umma::sdesc(smem_addr(vb), 128, LBO_B);
      constexpr uint64_t a_stage = stage_bytes >> 4, a_chunk = slot_bytes >> 4, a_half = (16 * 128) >> 4,
                         a_part = part_bytes >> 4;
      constexpr uint64_t b_term = ((uint64_t)(kBP / 8) * LBO_B) >> 4;  // v_q: 8 column groups per term
      uint64_t ast = adesc0;  // descriptor of stage mst
      for (int s = 0; s < nsteps; ++s) {
        bool ok = mbar_spin_bounded(vfull, (unsigned)(s & 1), p.status, wlim, 0);
        fence_after();
        uint64_t bdesc = bdesc0;  // advances by one K-step (2 node groups of 128 bytes) per chunk
        for (int kc0 = 0; kc0 < cps && ok; kc0 += kSub) {
          if (!mbar_spin_bounded(&full[mst], (unsigned)(muse & 1), p.status, wlim, 0)) {
            ok = false;
            break;
          }
          fence_after();
#pragma unroll
          for (int sub = 0; sub < kSub; ++sub) {
            const uint64_t ac = ast + sub * a_chunk;
#pragma unroll
            for (int pt = 0; pt < KP; ++pt)  // A_pt v_q for pt + q < KP, all into the one accumulator
#pragma unroll
              for (int qv = 0; qv + pt < KP; ++qv)
#pragma unroll
                for (int hh = 0; hh < NH; ++hh)
                  umma::mma_bf16(tbase + (s & 1) * dset + hh * dcols, ac + pt * a_part + hh * a_half,
                                 bdesc + qv * b_term, umma::idesc_bf16(128, BP) | kBMajorMN,
                                 (kc0 + sub > 0 || pt > 0 || qv > 0) ? 1u : 0u);
            bdesc += (uint64_t)((2 * 128) >> 4);
          }
          mma_commit(&empty[mst]);
          ast += a_stage;
          if (++mst == NS) { mst = 0; ++muse; ast = adesc0; }
        }
        if (ok) {
          mma_commit(dfull);
        } else {
          *fail = 1;
          mbar_arrive(dfull);  // release the epilogue threads
          break;
        }
      }
    }
    __syncwarp();
  } else {
    // ---- 8 epilogue warps --------------------------------------------------------------------
    // mapping: warp -> TMEM lane quarter q and either a 128-row half (nh = 2, all 64 columns)
    // or a 32-column half (nh = 1, rows 0..127)
    const int q = warp & 3, sub = warp >> 2;
    const int h = (nh == 2) ? sub : 0;
    const int cb = (nh == 2) ? 0 : sub * 32;
    constexpr int ncb = (nh == 2) ? 2 : 1;
    const int i = h * 128 + q * 32 + lane;
    const bool real = i < Mp;

    // B-operand byte offset of (node i, column n): column group n/8 (LBO_B apart), node group i/8
    // (128 bytes apart), node i%8 (16 bytes), column n%8 (2 bytes); part p of the split is column
    // col + 64 p.  Columns col0 .. col0+7 (col0 % 8 == 0) of this node, three 16-byte stores.
    unsigned char* vrow = vb + (uint32_t)(i >> 3) * 128 + (uint32_t)(i & 7) * 16;
    auto put_v8 = [&](int col0, const float (&v)[8]) {
      uint32_t w[3][4];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {  // the split of split3 (leading KP terms), two columns per conversion
        const __nv_bfloat162 h0 = __floats2bfloat162_rn(v[e], v[e + 1]);
        w[0][e / 2] = *reinterpret_cast<const uint32_t*>(&h0);
        if (KP > 1) {
          const float ra = v[e] - __low2float(h0), rb = v[e + 1] - __high2float(h0);
          const __nv_bfloat162 h1 = __floats2bfloat162_rn(ra, rb);
          w[1][e / 2] = *reinterpret_cast<const uint32_t*>(&h1);
          if (KP > 2) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(ra - __low2float(h1), rb - __high2float(h1));
            w[2][e / 2] = *reinterpret_cast<const uint32_t*>(&h2);
          }
        }
      }
      unsigned char* a = vrow + (uint32_t)(col0 >> 3) * LBO_B;
#pragma unroll
      for (int q2 = 0; q2 < KP; ++q2)
        *reinterpret_cast<uint4*>(a + (uint32_t)q2 * (kBP / 8) * LBO_B) = make_uint4(w[q2][0], w[q2][1], w[q2][2], w[q2][3]);
    };
    // v written and this thread's reads of D done: release the next step's MMAs (one arrival per warp)
    auto release_v = [&]() {
      fence_proxy_async_smem();
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(vfull);
    };

    for (int blk = 0; blk < ncb; ++blk)
      for (int n0 = 0; n0 < 32; n0 += 8) {
        float v[8];
        for (int e = 0; e < 8; ++e) {
          const int b = b0 + cb + blk * 32 + n0 + e;
          v[e] = 0.0f;
          if (p.V) {
            if (i < p.M && b < p.B) v[e] = p.src[i] * (float)p.V[(size_t)b * p.M + i];
          } else if (real) {
            v[e] = p.rhs[(size_t)i * Bpad + b];
          }
        }
        put_v8(cb + blk * 32 + n0, v);
      }
    release_v();

    // warm L2 with the global operands step s2's epilogue reads before its accumulator wait: z of
    // step s2 (back substitution) or the right-hand side of the column after it (forward).  Issued
    // as soon as step s2 - 1 has released its vector, so the copies overlap that step's stores.
    auto warm_l2 = [&](int s2) {
      const bool fwd2 = s2 < N;
      const int j2 = fwd2 ? s2 : 2 * N - 2 - s2;
      const float* zp2 = p.z + ((size_t)j2 * (Bpad / BP) + blockIdx.x) * (size_t)Mp * BP;
      const int i0 = i - lane + (lane & 3) * 8;  // this lane's quarter of the warp's 32 rows
      for (int blk = 0; blk < ncb; ++blk) {
        if (!fwd2 && i0 < Mp)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(zp2 + ((size_t)((cb + blk * 32) / 4 + (lane >> 2)) * Mp + i0) * 4));
        if (real && s2 + 1 < N && p.rhs)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(p.rhs + ((size_t)(j2 + 1) * Mp + i) * Bpad + b0 + cb + blk * 32));
      }
    };
    warm_l2(0);
    // the warp's 32 x 32 tile v (lane = row) times sc to rows (i - lane) + r of dst (row stride
    // Bpad), r < 32, columns 0..31, staged in pres so that each store instruction writes 4 whole
    // rows.  Float4 q of row r goes to pres[(r & 7) kThreads + 32 warp + ((r & 24) | ((r + q) & 7))]:
    // only the pieces of this warp's own threads' copies (each thread has consumed its own, and
    // the next step's copies follow in program order), so no other warp shares the slice; the skew
    // keeps both the row writes and the chunk reads free of bank conflicts.
    float4* wst = pres + 32 * warp;
    auto store_rows = [&](float* dst, const float (&v)[32], float sc) {
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 8; ++q)
        wst[(lane & 7) * kThreads + ((lane & 24) | ((lane + q) & 7))] =
            make_float4(sc * v[4 * q], sc * v[4 * q + 1], sc * v[4 * q + 2], sc * v[4 * q + 3]);
      __syncwarp();
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int r = 4 * m + (lane >> 3), q = lane & 7;
        const float4 x = wst[(r & 7) * kThreads + ((r & 24) | ((r + q) & 7))];
        if (i - lane + r < Mp) *reinterpret_cast<float4*>(dst + (size_t)r * Bpad + 4 * q) = x;
      }
      __syncwarp();
    };
    float local_max = 0.0f;
    for (int s = 0; s < nsteps; ++s) {
      const bool fwd = s < N;
      const int j = fwd ? s : 2 * N - 2 - s;
      const bool nfwd = s + 1 < N;
      float* zp = p.z + ((size_t)j * (Bpad / BP) + blockIdx.x) * (size_t)Mp * BP;  // z panel of step j
      const float ej = real ? (nfwd ? p.e[(size_t)j * Mp + i] : (j > 0 ? p.e[(size_t)(j - 1) * Mp + i] : 0.0f))
                            : 0.0f;
      const float hj = real ? p.hs[(size_t)j * Mp + i] : 0.0f;
      const float sj = (real && p.w1out) ? p.s32[(size_t)j * Mp + i] : 0.0f;
      const size_t rowoff = ((size_t)j * Mp + (real ? i : 0)) * Bpad + b0 + cb;
      const bool have_w = !fwd || s == N - 1;
      const bool more = s + 1 < nsteps;
      // the current this step adds to, read now so that its latency overlaps the accumulator wait
      double Iold = 0.0;
      if (have_w && p.accumulate && tid < BP && b0 + tid < p.B) Iold = p.I[(size_t)(b0 + tid) * N + j];
      // the next input's operands that do not depend on D -- z of this step (back substitution) or
      // the next column's right-hand side (forward) -- are loaded before the wait: column block 0
      // now, block 1 right after it, so their latency leaves the step's critical path
      const bool use_z = !fwd && real;
      const bool use_r = more && nfwd && p.rhs && real;
      float pre[ncb][32];
      // block 1 (nh == 2): 16-byte cp.async copies into this thread's slice of pres, waited for
      // after the accumulator wait, so their latency overlaps it
      auto async_pre1 = [&]() {
        if (use_z) {
          const float4* zrow = reinterpret_cast<const float4*>(zp) + (size_t)((cb + 32) / 4) * Mp + i;
#pragma unroll
          for (int n = 0; n < 32; n += 4)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_addr(pres + (n / 4) * kThreads + tid)),
                         "l"(zrow + (size_t)(n / 4) * Mp)
                         : "memory");
        } else if (use_r) {
          const float* rn = p.rhs + rowoff + 32 + (size_t)Mp * Bpad;
#pragma unroll
          for (int n = 0; n < 32; n += 4)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_addr(pres + (n / 4) * kThreads + tid)),
                         "l"(rn + n)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
      };
      auto take_pre1 = [&]() {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        if (use_z || use_r) {
#pragma unroll
          for (int n = 0; n < 32; n += 4) {
            const float4 v4 = pres[(n / 4) * kThreads + tid];
            pre[ncb - 1][n] = v4.x;
            pre[ncb - 1][n + 1] = v4.y;
            pre[ncb - 1][n + 2] = v4.z;
            pre[ncb - 1][n + 3] = v4.w;
          }
        }
      };
      auto load_pre = [&](int blk) {
        if (use_z) {
          const float4* zrow = reinterpret_cast<const float4*>(zp) + (size_t)((cb + blk * 32) / 4) * Mp + i;
#pragma unroll
          for (int n = 0; n < 32; n += 4) {
            const float4 zz = zrow[(size_t)(n / 4) * Mp];
            pre[blk][n] = zz.x;
            pre[blk][n + 1] = zz.y;
            pre[blk][n + 2] = zz.z;
            pre[blk][n + 3] = zz.w;
          }
        } else if (use_r) {
          const float* rn = p.rhs + rowoff + blk * 32 + (size_t)Mp * Bpad;
#pragma unroll
          for (int n = 0; n < 32; n += 4) {
            const float4 r4 = *reinterpret_cast<const float4*>(rn + n);
            pre[blk][n] = r4.x;
            pre[blk][n + 1] = r4.y;
            pre[blk][n + 2] = r4.z;
            pre[blk][n + 3] = r4.w;
          }
        }
      };
      load_pre(0);
      if (nh == 2) async_pre1();
      // one thread polls the accumulator barrier; the others wait on the named hardware barrier so
      // that no shared-memory polling competes with the tensor core's operand reads
      bool okd = true;
      if (tid == 32) okd = mbar_spin_bounded(dfull, (unsigned)(s & 1), p.status, wlim, 64);
      if (!okd) atomicExch(fail, 1u);
      if (epi_sync_or(*fail != 0)) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");  // no copy outlives the loop
        break;
      }
      fence_after();
      if (nh == 2) take_pre1();

      // (1) D of this step per column block (z added in the back substitution), then (2) the next
      // step's input from it, split into BF16 terms; then the next step's MMAs may start
      const uint32_t tstep = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)((s & 1) * dset + h * dcols + cb);
      if (more) {
#pragma unroll
        for (int blk = 0; blk < ncb; ++blk) {
          float a[32];
          tmem_ld32(tstep + blk * 32, a);
#pragma unroll
          for (int n = 0; n < 32; n += 8) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const float x = use_z ? a[n + e] + pre[blk][n + e] : a[n + e];
              v[e] = use_r ? fmaf(ej, x, pre[blk][n + e]) : ej * x;
            }
            put_v8(cb + blk * 32 + n, v);
          }
        }
        release_v();
        warm_l2(s + 1);
      }
      // (3) while the next step's MMAs run: z (forward), w and the current (back substitution)
      float dots[ncb];
#pragma unroll
      for (int blk = 0; blk < ncb; ++blk) {
        float a[32];  // this step's D again (its accumulator set is not written until step s + 2)
        tmem_ld32(tstep + blk * 32, a);
        if (use_z)
#pragma unroll
          for (int n = 0; n < 32; ++n) a[n] += pre[blk][n];
        if (fwd && real) {
          float4* zrow = reinterpret_cast<float4*>(zp) + (size_t)((cb + blk * 32) / 4) * Mp + i;
#pragma unroll
          for (int n = 0; n < 32; n += 4)
            zrow[(size_t)(n / 4) * Mp] = make_float4(a[n], a[n + 1], a[n + 2], a[n + 3]);
        }
        if (have_w) {
          // w (or the refinement state s o w, FP32: the float pairs' low part is 0) of this block's
          // 32 rows x 32 columns, written as whole 128-byte row segments through the warp's slice of
          // pres (free until the next step's copies, which follow the epi_sync below)
          if (p.w || p.w1out)
            store_rows((p.w ? p.w : p.w1out) + ((size_t)j * Mp + (i - lane)) * Bpad + b0 + cb + blk * 32, a,
                       p.w ? 1.0f : sj);
#pragma unroll
          for (int n = 0; n < 32; ++n) a[n] *= hj;
          dots[blk] = transpose_sum32(a, lane);
        }
      }
      if (have_w)
#pragma unroll
        for (int blk = 0; blk < ncb; ++blk) red[warp * 64 + cb + blk * 32 + lane] = dots[blk];
      epi_sync();
      if (have_w && tid < BP) {
        float sum = 0.0f;
        if (nh == 2) {
          for (int w = 0; w < 8; ++w) sum += red[w * 64 + tid];
        } else {
          const int s0 = (tid >> 5) * 4;  // warps covering this column block
          for (int w = s0; w < s0 + 4; ++w) sum += red[w * 64 + tid];
        }
        const int b = b0 + tid;
        if (b < p.B) {
          double* Ip = p.I + (size_t)b * N + j;
          const double dI = (double)sum;
          if (!isfinite(dI)) set_status(p.status, XBAR_DEV_NONFINITE);
          if (p.accumulate) {
            const double In = Iold + dI;
            *Ip = In;
            local_max = fmaxf(local_max, (float)(fabs(dI) / fmax(fabs(In), 1e-300)));
          } else {
            *Ip = dI;
          }
        }
      }
    }
    if (p.max_rel) {
      for (int o = 16; o > 0; o >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
      if (lane == 0 && local_max > 0.0f) atomic_max_nonneg(p.max_rel, local_max);
    }
  }
  // ---- teardown: all 10 warps; free tensor memory ------------------------------------------------
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) tmem_dealloc(tbase, ncols);
}

size_t sweep_tc_smem_bytes(int Mt, int KP) {
  return 256 + 8 * 64 * 4 + (size_t)tc_stages(Mt, KP) * tc_sub(Mt, KP) * tc_slot(Mt, KP) + tc_vbytes(Mt, KP) +
         tc_prebytes(Mt);
}

bool sweep_tc_supported(int Mp) { return Mp <= 256; }

int sweep_tc_rows(int Mp) { return Mp <= 128 ? 128 : 256; }

size_t sweep_tc_tile_bytes(int Mp, int N) {
  const int Mt = sweep_tc_rows(Mp);
  return (size_t)N * Mt * Mt * tc::kParts * sizeof(__nv_bfloat16);
}

cudaError_t launch_sweep_tc_tile(const float* X, void* Xt, int Mp, int N, cudaStream_t st) {
  const int Mt = sweep_tc_rows(Mp);
  const size_t n = (size_t)Mt * Mt * N;
  sweep_tc_tile_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(X, static_cast<__nv_bfloat16*>(Xt), Mp, Mt,
                                                                    N);
  return cudaGetLastError();
}

cudaError_t launch_sweep_tc(const SweepParams<float>& p, const void* Xt, int terms, cudaStream_t st) {
  const int Mt = sweep_tc_rows(p.Mp);
  if (p.Bp != tc::kBP || p.Bpad % tc::kBP) return cudaErrorInvalidValue;
  const int blocks = (p.B + tc::kBP - 1) / tc::kBP;
  if (blocks == 0) return cudaSuccess;
  if (terms < 1 || terms > tc::kParts) return cudaErrorInvalidValue;
  const size_t smem = sweep_tc_smem_bytes(Mt, terms);
  using Kern = void (*)(SweepParams<float>, const __nv_bfloat16*);
  const Kern kerns[2][3] = {{sweep_tc_kernel<1, 1>, sweep_tc_kernel<1, 2>, sweep_tc_kernel<1, 3>},
                            {sweep_tc_kernel<2, 1>, sweep_tc_kernel<2, 2>, sweep_tc_kernel<2, 3>}};
  const Kern kern = kerns[Mt == 128 ? 0 : 1][terms - 1];
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  kern<<<blocks, tc::kThreads + 64, smem, st>>>(p, static_cast<const __nv_bfloat16*>(Xt));
  return cudaGetLastError();
}

}  // namespace xbar
