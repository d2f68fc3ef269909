// Asynchronous copies between global and shared memory for sm_103a: the
// bulk-copy engine (TMA, cp.async.bulk) for the 16-byte-aligned interior of a
// contiguous window, cp.async for the few unaligned elements at its ends, and
// an mbarrier that completes when both have landed.  Every wait is bounded.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace hs {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make initialised barriers visible to the asynchronous proxy
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this thread's generic-proxy shared-memory accesses before later
// asynchronous-proxy (bulk copy) accesses
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// one plain arrival (no transaction bytes)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Wait for phase `parity` of `bar` to complete; gives up after `limit_ns` of
// globaltimer time (or an iteration count of the same order), sets kErrTimeout
// and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t* err, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint64_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 0) {
      const uint64_t now = globaltimer_ns();
      if (now - t0 > limit_ns || it > (limit_ns >> 3)) {
        atomicOr(err, kErrTimeout);
        return false;
      }
    }
  }
}

// Bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16),
// completing as transaction bytes on `bar`.
__device__ __forceinline__ void bulk_g2s(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(sdst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Bulk copy shared -> global (both 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_s2g(void* gdst, const void* ssrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_u32(ssrc)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory sources of this thread's bulk stores have been read
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// this thread's bulk stores are complete (visible in global memory)
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* sdst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(sdst)), "l"(gsrc), "n"(BYTES) : "memory");
}
// `bar` tracks completion of this thread's earlier cp.async copies (adds one
// pending arrival now, which the copies' completion performs).
__device__ __forceinline__ void cp_async_mbar_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Plan of one contiguous window of `cnt` elements of E bytes at global
// address g: the 16-byte-aligned interior [g_lo, g_hi) and the element counts
// before (head) and after (tail) it.  `phase` = elements between the 16-byte
// boundary below g and g: placing element 0 at shared index `phase` of a
// 16-byte-aligned region aligns the interior on both sides.
struct Window {
  uint32_t phase, head, body_bytes, tail;
};
template <int E>
__device__ __forceinline__ Window plan_window(const void* g, uint32_t cnt) {
  Window w;
  const uintptr_t a = reinterpret_cast<uintptr_t>(g);
  const uintptr_t end = a + static_cast<uintptr_t>(cnt) * E;
  w.phase = static_cast<uint32_t>((a & 15u) / E);
  const uintptr_t lo = (a + 15u) & ~static_cast<uintptr_t>(15u);
  const uintptr_t hi = end & ~static_cast<uintptr_t>(15u);
  if (cnt == 0 || lo >= hi) {  // no aligned interior: every element goes one by one
    w.head = cnt;
    w.body_bytes = 0;
    w.tail = 0;
  } else {
    w.head = static_cast<uint32_t>((lo - a) / E);
    w.body_bytes = static_cast<uint32_t>(hi - lo);
    w.tail = static_cast<uint32_t>((end - hi) / E);
  }
  return w;
}

}  // namespace hs
