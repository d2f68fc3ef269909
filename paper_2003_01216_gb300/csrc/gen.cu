// Device-side twin of paper_2003_01216_gb300/inputs.py: fills device memory
// with the same seeded synthetic keys, bit for bit, so large inputs never
// cross PCIe.  Input generation only: nothing here takes part in the sort.
// Built into its own library (libhsgen.so).
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

// SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

__host__ __device__ __forceinline__ uint64_t stream_base(uint64_t seed, uint64_t stream) {
  return mix64(seed * kGamma + stream);
}

__device__ __forceinline__ uint64_t perm20(uint64_t x) {
  uint64_t y = (x * 0x9E3779B1ull) & 0xFFFFFull;
  return y ^ (y >> 10);
}

// first r with cdf[r] > u (cdf non-decreasing, cdf[m-1] = 1 > u)
__device__ __forceinline__ uint64_t upper_bound(const double* cdf, uint64_t m, double u) {
  uint64_t lo = 0, hi = m;
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1;
    if (cdf[mid] > u) hi = mid; else lo = mid + 1;
  }
  return lo;
}

template <class T>
__global__ void k_fill(int dist, uint64_t seed, uint64_t stream, uint64_t n, uint64_t start, T* out,
                       const double* cdf, uint64_t cdf_n) {
  const uint64_t b = stream_base(seed, stream);
  const uint64_t b2 = stream_base(seed, stream ^ 0xFFFFull);
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint64_t gi = start + i;
    const uint64_t h = mix64(b + (gi + 1) * kGamma);
    uint64_t v = 0;
    switch (dist) {
      case 0: v = h & 0x7FFFFFFFull; break;
      case 1: v = h % 1000000000ull; break;
      case 2: {
        const double u = static_cast<double>(h >> 11) * 0x1.0p-53;
        v = perm20(upper_bound(cdf, cdf_n, u)) << 11;
        break;
      }
      case 3: v = (gi << 31) / (start + n); break;
      case 4: v = ((start + n - 1 - gi) << 31) / (start + n); break;
      case 5: v = 123456789ull; break;
      case 6: v = (h & 15ull) * (1ull << 27) + 12345ull; break;
      case 7: v = h; break;
      case 8: v = mix64(b2 + ((h & ((1ull << 24) - 1)) + 1) * kGamma); break;
      case 9: v = h & 0xFFFFFFFFull; break;
      case 10: v = h & 0xFFFFFFFFull; break;
      case 11: v = h % 1000ull; break;
      default: v = 0; break;
    }
    out[i] = static_cast<T>(v);
  }
}

__global__ void k_iota(uint32_t* out, uint64_t n) {
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
    out[i] = static_cast<uint32_t>(i);
}

}  // namespace

extern "C" {

// Fill out[0..n) with keys i = start .. start + n - 1 of distribution `dist`
// (codes of inputs.DIST; "sorted"/"reverse" take n + start as the length).
// key_bytes: 4 or 8.  cdf: device table for "zipf" (else NULL).
int hsg_fill(int dist, uint64_t seed, uint64_t stream, uint64_t n, uint64_t start, void* out, int key_bytes,
             const double* cdf, uint64_t cdf_n, void* cuda_stream) {
  if (n == 0) return 0;
  if (!out || (key_bytes != 4 && key_bytes != 8) || (dist == 2 && !cdf)) return 1;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int grid = 152 * 8;
  if (key_bytes == 4)
    k_fill<uint32_t><<<grid, 256, 0, st>>>(dist, seed, stream, n, start, static_cast<uint32_t*>(out), cdf, cdf_n);
  else
    k_fill<uint64_t><<<grid, 256, 0, st>>>(dist, seed, stream, n, start, static_cast<uint64_t*>(out), cdf, cdf_n);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// out[i] = i (the stability-witness values of a key-value workload).
int hsg_iota(uint32_t* out, uint64_t n, void* cuda_stream) {
  if (n == 0) return 0;
  if (!out) return 1;
  k_iota<<<152 * 8, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(out, n);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // extern "C"
