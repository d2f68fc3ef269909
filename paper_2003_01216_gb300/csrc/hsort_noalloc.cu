// hs_sort_keys_noalloc: the keys-only sort with its scratch memory in a
// fixed device array that the library itself holds, for callers that cannot
// allocate device memory.  Such callers include code that runs where
// cudaMalloc is unavailable or forbidden (inside a CUDA-graph capture that
// may not contain allocations, a real-time loop that must never block on the
// allocator, a plugin whose host framework owns every device allocation), and
// code that must not change the device's memory footprint after start-up.
//
// The scratch array below lives in this library's module: every GPU that
// loads the library holds its 16 MiB until the process exits.  It is a
// host-side stand-in in host code, so host code never passes its name to a
// kernel; the device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and passed on.
#include <cstdio>
#include <mutex>

#include "driver.cuh"

namespace hs {

// Largest input accepted: 2^20 keys of any key type, with either partition.
constexpr size_t kNoAllocMaxKeys = size_t(1) << 20;
constexpr size_t kNoAllocBytes = size_t(16) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

void set_error_message(const char* msg);

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_na_mu;
void* g_na_ptr[kMaxDevices] = {};  // device -> device address of g_noalloc_scratch (set up once)

hs_status scratch_ptr(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return HS_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return HS_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (g_na_ptr[dev]) {
    *out = g_na_ptr[dev];
    return HS_OK;
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // with `dev` current
  if (e != cudaSuccess || p == nullptr) {
    set_cuda_error(e);
    return HS_ERR_CUDA;
  }
  g_na_ptr[dev] = p;
  *out = p;
  return HS_OK;
}
}  // namespace

}  // namespace hs

using namespace hs;

extern "C" hs_status hs_sort_keys_noalloc(hs_dtype dtype, void* d_keys, size_t n, int partition, void* stream) {
  if (dtype != HS_INT32 && dtype != HS_UINT32 && dtype != HS_UINT64) return HS_ERR_INVALID;
  if (partition == 0) partition = 10;
  if (partition != 1 && partition != 10 && partition != 256) return HS_ERR_INVALID;
  if (n > kNoAllocMaxKeys) {
    char msg[128];
    std::snprintf(msg, sizeof(msg), "hs_sort_keys_noalloc: n = %zu exceeds the maximum of %zu keys", n,
                  kNoAllocMaxKeys);
    set_error_message(msg);
    return HS_ERR_INVALID;
  }
  if (n > 0 && !d_keys) return HS_ERR_INVALID;
  if (n == 0) return HS_OK;
  if (timing_on()) {
    // timing records create CUDA events; this entry point creates nothing
    set_error_message("hs_sort_keys_noalloc: turn per-kernel timing off (hs_timing_enable(0)) first");
    return HS_ERR_INVALID;
  }
  void* scratch = nullptr;
  HS_TRY(scratch_ptr(&scratch));
  const size_t need = workspace_bytes(dtype == HS_UINT64 ? 8 : 4, n, false, 1, partition);
  if (need > kNoAllocBytes) {
    set_error_message("hs_sort_keys_noalloc: scratch array too small for this call");
    return HS_ERR_INVALID;
  }
  hs_opts o{};
  o.partition = partition;
  o.d_workspace = scratch;
  o.workspace_bytes = kNoAllocBytes;
  return hs_sort_keys(dtype, d_keys, n, &o, stream);
}
