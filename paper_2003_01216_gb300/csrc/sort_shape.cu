// Instantiates the sort for one (key type, tile shape) pair, chosen by the
// build with -DHS_SHAPE_KEY=<type> -DHS_SHAPE_IPT=<items per thread>
// -DHS_SHAPE_FN=<entry name>: one object per pair, so the library's kernels
// compile in parallel.
#include "driver.cuh"

#if !defined(HS_SHAPE_KEY) || !defined(HS_SHAPE_IPT) || !defined(HS_SHAPE_FN)
#error "sort_shape.cu is compiled once per shape with HS_SHAPE_KEY, HS_SHAPE_IPT and HS_SHAPE_FN defined"
#endif

namespace hs {
hs_status HS_SHAPE_FN(void* keys, uint32_t* vals, size_t n, size_t nseg, const uint64_t* offs, const hs_opts& o,
                      char* ws, uint32_t* err, cudaStream_t st, const void* src, int* host_done) {
  return run_sort_ipt<HS_SHAPE_KEY, HS_SHAPE_IPT>(keys, vals, n, nseg, offs, o, ws, err, st, src, host_done);
}
}  // namespace hs
