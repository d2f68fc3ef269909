// Instantiates the sort for uint64_t keys (one translation unit per key type so
// the library's kernels compile in parallel).
#include "driver.cuh"

namespace hs {
hs_status run_sort_u64(void* keys, uint32_t* vals, size_t n, size_t nseg, const uint64_t* offs, const hs_opts& o,
                      char* ws, uint32_t* err, cudaStream_t st) {
  return run_sort<uint64_t>(keys, vals, n, nseg, offs, o, ws, err, st);
}
}  // namespace hs
