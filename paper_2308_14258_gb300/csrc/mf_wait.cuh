// Bounded waits on shared-memory mbarriers, shared by the tensor-core SDNet kernel and
// the failure-detection self-test (which runs these same routines against a phase that
// never completes). A wait gives up after limit_ns of %globaltimer (default 1 s): it
// records kDevErrTimeout in the device status word, raises the CTA's abort flag so the
// other roles of the CTA stop waiting too, and returns false. No wait traps or asserts.
#pragma once
#include <stdint.h>

#include "mf_internal.cuh"

namespace mf {
namespace {

constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint32_t bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase; false once the CTA is aborting or after the limit.
// The _inl forms are for kernels that reallocate registers between warpgroups (a called
// function has one register budget); the others are out-of-line copies of the same loop.
__device__ __forceinline__ bool wait_bounded_inl(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status,
                                                 bool honour_abort, unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (honour_abort && *abort_flag) return false;
    if (globaltimer() - t0 > limit_ns) {
      *abort_flag = 1;
      atomicExch(status, kDevErrTimeout);
      return false;
    }
  }
}
__device__ __noinline__ bool wait_bounded(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status,
                                          bool honour_abort, unsigned long long limit_ns = kWaitLimitNs) {
  return wait_bounded_inl(bar, parity, abort_flag, status, honour_abort, limit_ns);
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Spinning bounded wait: polls the phase without suspending (a suspended try_wait wakes
// a few hundred cycles after the phase completes, which sits on the critical path);
// the abort flag and the time limit are checked every 64 polls.
__device__ __forceinline__ bool wait_spin_inl(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status,
                                              unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t i = 1;; ++i) {
    if (mbar_test(bar, parity)) return true;
    if ((i & 63u) == 0u) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > limit_ns) {
        *abort_flag = 1;
        atomicExch(status, kDevErrTimeout);
        return false;
      }
    }
  }
}
__device__ __noinline__ bool wait_spin(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status,
                                       unsigned long long limit_ns = kWaitLimitNs) {
  return wait_spin_inl(bar, parity, abort_flag, status, limit_ns);
}

// Spinning bounded wait with a short sleep between polls, for waits that are not on the
// critical path: the waiting warps then leave the issue slots to the warps that work.
__device__ __forceinline__ bool wait_nap_inl(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status,
                                             unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    __nanosleep(32);
    if (mbar_test(bar, parity)) return true;
    if (*abort_flag) return false;
    if (globaltimer() - t0 > limit_ns) {
      *abort_flag = 1;
      atomicExch(status, kDevErrTimeout);
      return false;
    }
  }
}

// Warp-uniform form: every lane waits, and the warp continues only if all lanes saw
// the phase complete (the .sync.aligned tcgen05 loads that follow need the whole warp).
__device__ __forceinline__ bool wait_warp(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status) {
  const bool ok = wait_spin(bar, parity, abort_flag, status);
  return __all_sync(0xffffffffu, ok);
}
// The same with the spin inline: no call on the hot path (a phase that is already
// complete costs one test instead of a call and return).
__device__ __forceinline__ bool wait_warp_inl(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status) {
  return __all_sync(0xffffffffu, wait_spin_inl(bar, parity, abort_flag, status));
}

}  // namespace
}  // namespace mf
