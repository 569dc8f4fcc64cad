// mbarrier, bulk-copy (TMA) and named-barrier helpers (inline PTX, sm_90+ forms used on sm_103a).
//
// Every wait is bounded by wall-clock time (the %globaltimer register, nanoseconds): a wait that runs
// out returns false, and the caller records LEB_ASYNC_TIMEOUT and leaves its loop instead of hanging.
#pragma once
#include <cstdint>

namespace leb {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// The same test with a suspend-time hint: a thread whose phase has not completed is suspended until it
// completes or about hint_ns have passed, instead of returning at once, so that a waiting warp takes no
// issue slots from the warps that work.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

constexpr uint32_t kWaitSleepNs = 100000;   // suspend-time hint of a wait's retries (100 us)

// Wait until the phase with the given parity has completed; false if limit_ns ran out first.
__device__ __forceinline__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait_sleep(bar, parity, kWaitSleepNs)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// Waits that poll without suspending (bounded like the others), for the single threads that hand weight
// tiles from TMA to the tensor cores: a suspended thread resumes some time after the phase completes, a
// delay that a chain of such hand-offs would pay on every tile. The cluster form acquires at cluster
// scope, for phases completed by arrivals from another CTA of the cluster.
__device__ __forceinline__ bool mbar_try_wait_cl(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
template <bool kCluster>
__device__ __forceinline__ bool mbar_wait_spin(uint64_t* bar, uint32_t parity) {
  auto test = [&]() { return kCluster ? mbar_try_wait_cl(bar, parity) : mbar_try_wait(bar, parity); };
  if (test()) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (test()) return true;
    if (global_ns() - t0 > kWaitLimitNs) return false;
  }
}
// A sleeping wait with acquire at cluster scope (phases completed from another CTA of the cluster).
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait_cl(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait_cluster(bar, parity, kWaitSleepNs)) return true;
    if (global_ns() - t0 > kWaitLimitNs) return false;
  }
}

// The kernels' wait: the same, with the library's limit.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  return mbar_wait_for(bar, parity, kWaitLimitNs);
}

// A wait that all 32 lanes of a warp make together (each lane waits, so each has its own acquire of the
// phase): the result is the same in every lane. Without the vote, lanes whose waits end on either side of
// the limit would take different branches, and a later warp-wide shuffle or __syncwarp would wait for
// lanes that have left.
__device__ __forceinline__ bool mbar_wait_warp_for(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  return __all_sync(0xffffffffu, mbar_wait_for(bar, parity, limit_ns));
}
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* bar, uint32_t parity) {
  return mbar_wait_warp_for(bar, parity, kWaitLimitNs);
}

// Bulk (non-tensor) async copy global -> shared, completion counted in bytes on an mbarrier.
// Source, destination and size must be multiples of 16 bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Named barrier among `count` threads (a multiple of 32) that also ORs a predicate across them.
__device__ __forceinline__ bool bar_sync_or(int id, int count, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "barrier.cta.red.or.pred p, %2, %3, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void bar_sync(int id, int count) {
  asm volatile("barrier.cta.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Barrier among the warps of a group (one arrival per warp, the mbarrier initialised with the group's
// warp count) whose wait is bounded, unlike a named barrier: if a warp of the group has left after a
// wait of its own ran out, the others give up after the limit too instead of waiting forever. It also
// ORs a per-thread predicate over the group. The OR words rotate over three phases: the word of phase
// p + 2 is cleared after phase p completes, when no warp can still read it (its readers all arrived
// at phase p) and none can write it yet (its writers must first pass phase p + 1).
struct GroupBar {
  uint64_t bar;
  int orw[3];
};

__device__ __forceinline__ void group_bar_init(GroupBar* g, uint32_t warps) {
  mbar_init(&g->bar, warps);
  g->orw[0] = g->orw[1] = g->orw[2] = 0;
}

// Every lane of every warp of the group calls this with the same phase counter (advanced here).
// Returns the OR of every thread's bits over the group; *ok = false if the wait ran out (the result is
// then unusable).
__device__ __forceinline__ uint32_t group_sync_or(GroupBar* g, uint32_t& phase, uint32_t bits, bool* ok,
                                                  unsigned long long limit_ns) {
  const uint32_t wor = __reduce_or_sync(0xffffffffu, bits);
  const int slot = (int)(phase % 3u);
  if ((threadIdx.x & 31) == 0) {
    if (wor) atomicOr(&g->orw[slot], (int)wor);
    mbar_arrive(&g->bar);
  }
  *ok = mbar_wait_warp_for(&g->bar, phase & 1u, limit_ns);
  const uint32_t res = (uint32_t)*(volatile int*)&g->orw[slot];
  if ((threadIdx.x & 31) == 0) g->orw[(slot + 2) % 3] = 0;
  ++phase;
  return res;
}

}  // namespace leb
