// Device-wide exclusive prefix sum of uint32 counts, in place, as three
// plain kernels (reduce chunks, scan the chunk sums, rescan the chunks with
// their carry-in).  No kernel waits on another CTA.  The element count is read
// from device memory (`*m_ptr`, multiplied by `mult`) so the host never needs
// it; the host only sizes the partials array (kScanChunks entries).
#pragma once
#include "common.cuh"

namespace hs {

constexpr int kScanBlock = 256;
constexpr int kScanChunks = 1024;  // CTAs of the reduce and rescan kernels

__device__ __forceinline__ uint32_t block_incl_scan(uint32_t v, uint32_t* s_warp) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t x = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += x;
  }
  if (lane == 31) s_warp[wid] = v;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = (lane < (kScanBlock >> 5)) ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += x;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  const uint32_t r = v + (wid ? s_warp[wid - 1] : 0u);
  __syncthreads();
  return r;
}

__device__ __forceinline__ void chunk_range(uint64_t m, uint32_t c, uint64_t& lo, uint64_t& hi) {
  const uint64_t per = (m + kScanChunks - 1) / kScanChunks;
  lo = min64(m, static_cast<uint64_t>(c) * per);
  hi = min64(m, lo + per);
}

// 1. partials[c] = sum of chunk c
static __global__ void __launch_bounds__(kScanBlock) k_scan_reduce(const uint32_t* __restrict__ a,
                                                                    const uint32_t* __restrict__ m_ptr, uint32_t mult,
                                                                    uint32_t* __restrict__ partials) {
  griddep_open();
  __shared__ uint32_t s_warp[32];
  const uint64_t m = static_cast<uint64_t>(*m_ptr) * mult;
  uint64_t lo, hi;
  chunk_range(m, blockIdx.x, lo, hi);
  uint32_t sum = 0;
  for (uint64_t i = lo + threadIdx.x; i < hi; i += kScanBlock) sum += a[i];
  sum = __reduce_add_sync(0xffffffffu, sum);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kScanBlock / 32; ++w) t += s_warp[w];
    partials[blockIdx.x] = t;
  }
}

// 2. partials -> exclusive prefix (one CTA)
static __global__ void __launch_bounds__(kScanBlock) k_scan_partials(uint32_t* __restrict__ partials) {
  griddep_open();
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < kScanChunks; base += kScanBlock) {
    const uint32_t x = partials[base + threadIdx.x];
    const uint32_t incl = block_incl_scan(x, s_warp);
    const uint32_t carry = s_carry;
    partials[base + threadIdx.x] = carry + incl - x;
    __syncthreads();
    if (threadIdx.x == kScanBlock - 1) s_carry = carry + incl;
    __syncthreads();
  }
}

// 3. rescan every chunk with its carry-in, in place
static __global__ void __launch_bounds__(kScanBlock) k_scan_down(uint32_t* __restrict__ a,
                                                                  const uint32_t* __restrict__ m_ptr, uint32_t mult,
                                                                  const uint32_t* __restrict__ partials) {
  griddep_open();
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry;
  const uint64_t m = static_cast<uint64_t>(*m_ptr) * mult;
  uint64_t lo, hi;
  chunk_range(m, blockIdx.x, lo, hi);
  if (threadIdx.x == 0) s_carry = partials[blockIdx.x];
  __syncthreads();
  for (uint64_t base = lo; base < hi; base += kScanBlock) {
    const uint64_t i = base + threadIdx.x;
    const uint32_t x = (i < hi) ? a[i] : 0u;
    const uint32_t incl = block_incl_scan(x, s_warp);
    const uint32_t carry = s_carry;
    if (i < hi) a[i] = carry + incl - x;
    __syncthreads();
    if (threadIdx.x == kScanBlock - 1) s_carry = carry + incl;
    __syncthreads();
  }
}

}  // namespace hs
