// common.cuh -- device helpers shared by the libxbar kernels (sm_103a).
//
// Every wait in these kernels is bounded: a spin on a flag, a cross-block
// barrier or an mbarrier gives up after kWaitLimitNs of %globaltimer time,
// records XBAR_DEV_TIMEOUT in the caller-visible status word and lets the
// kernel return, so a stuck wait surfaces as XBAR_ETIMEOUT on the host instead
// of hanging the GPU.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace xbar {

// bits of the device status word (one unsigned per handle)
enum : unsigned {
  XBAR_DEV_TIMEOUT = 1u,    // a bounded wait expired
  XBAR_DEV_NONFINITE = 2u,  // a NaN/Inf was produced where none may appear
  XBAR_DEV_BADLAUNCH = 4u,  // a kernel found its launch shape inconsistent with its arguments
  XBAR_DEV_BADINPUT = 8u    // an input checked on the device was invalid (negative or non-finite G)
};

// default limit of every device-side wait: 2 s
#ifndef XBAR_WAIT_LIMIT_NS
#define XBAR_WAIT_LIMIT_NS 2000000000ull
#endif

// Device status block of a handle (16 bytes, the `status` pointer the kernels receive points at
// its first word): status bits, padding, then the wait limit in nanoseconds (0 = the default).
struct DevStatus {
  unsigned bits;
  unsigned pad;
  unsigned long long wait_ns;
};

// limit of the bounded waits of a kernel launched with this status block
__device__ __forceinline__ uint64_t wait_limit(const unsigned* status) {
  if (!status) return XBAR_WAIT_LIMIT_NS;
  const uint64_t v = *reinterpret_cast<const volatile unsigned long long*>(status + 2);
  return v ? v : XBAR_WAIT_LIMIT_NS;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void set_status(unsigned* status, unsigned bits) {
  if (status) atomicOr(status, bits);
}

// Cross-block barrier among `nblocks` co-resident blocks (cooperative launch).
// Sense reversal on a generation counter; `bar` points at two unsigned words
// {count, generation} zeroed before the first use.  Returns false (and sets
// XBAR_DEV_TIMEOUT) if the other blocks did not arrive within limit_ns.
// Must be called by every thread of the block.
__device__ __forceinline__ bool group_barrier(unsigned* bar, unsigned nblocks, unsigned* status,
                                              uint64_t limit_ns, unsigned* flag_smem) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned ok = 1;
    if (nblocks > 1) {
      volatile unsigned* vgen = bar + 1;
      const unsigned gen = *vgen;
      __threadfence();
      const unsigned arrived = atomicAdd(bar, 1u);
      if (arrived == nblocks - 1) {
        atomicExch(bar, 0u);
        __threadfence();
        atomicAdd(bar + 1, 1u);
      } else {
        const uint64_t t0 = globaltimer_ns();
        while (*vgen == gen) {
          __nanosleep(16);
          if (globaltimer_ns() - t0 > limit_ns) {
            ok = 0;
            set_status(status, XBAR_DEV_TIMEOUT);
            break;
          }
        }
      }
      __threadfence();
    }
    *flag_smem = ok;
  }
  __syncthreads();
  return *flag_smem != 0;
}

// ---------------------------------------------------------------------------------------------
// mbarrier + 1-D bulk copy (TMA engine) helpers
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// one bulk copy global -> shared, completion counted on `bar` (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, unsigned bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait for phase `parity` of `bar`; false (and XBAR_DEV_TIMEOUT) on expiry
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned* status,
                                                  uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > limit_ns) {
      set_status(status, XBAR_DEV_TIMEOUT);
      return false;
    }
  }
  return true;
}

// non-suspending probe of phase `parity`
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded spin on phase `parity` with test_wait (no suspension, so the waiter resumes as soon as
// the phase completes); sleep_ns > 0 backs off between probes for waiters that are not latency
// critical.  false (and XBAR_DEV_TIMEOUT) on expiry.
__device__ __forceinline__ bool mbar_spin_bounded(uint64_t* bar, unsigned parity, unsigned* status,
                                                  uint64_t limit_ns, unsigned sleep_ns) {
  if (mbar_test_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  unsigned k = 0;
  while (!mbar_test_wait(bar, parity)) {
    if (sleep_ns) __nanosleep(sleep_ns);
    if ((++k & 255u) == 0 && globaltimer_ns() - t0 > limit_ns) {
      set_status(status, XBAR_DEV_TIMEOUT);
      return false;
    }
  }
  return true;
}

// atomic max for non-negative floats through their ordered bit patterns
__device__ __forceinline__ void atomic_max_nonneg(float* addr, float v) {
  if (!(v >= 0.0f)) v = __int_as_float(0x7f800000);  // NaN -> +inf so it is noticed
  atomicMax(reinterpret_cast<int*>(addr), __float_as_int(v));
}

template <typename T>
__device__ __forceinline__ T ld_cg(const T* p) {
  return __ldcg(p);
}

}  // namespace xbar
