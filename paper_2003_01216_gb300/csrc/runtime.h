// Host runtime shared by the translation units of the library: a launch
// wrapper that checks every launch and, when timing is on, records a CUDA
// event pair around it on the launching stream; the per-kernel timing table;
// the cumulative count of kernel launches.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

#include "hsort.h"

namespace hs {

bool timing_on();
void timing_add(const char* name, cudaEvent_t a, cudaEvent_t b);
cudaEvent_t event_get();
void set_cuda_error(cudaError_t e);
void count_launch();

#define HS_TRY(x)                  \
  do {                             \
    hs_status _s = (x);            \
    if (_s != HS_OK) return _s;    \
  } while (0)

class Launcher {
 public:
  explicit Launcher(cudaStream_t s) : st_(s) {}
  void begin(const char* name) {
    name_ = name;
    t0_ = nullptr;
    if (timing_on()) {
      t0_ = event_get();
      cudaEventRecord(t0_, st_);
    }
  }
  // after a kernel launch
  hs_status end(bool kernel = true) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return HS_ERR_CUDA;
    }
    if (kernel) count_launch();
    if (t0_) {
      cudaEvent_t t1 = event_get();
      cudaEventRecord(t1, st_);
      timing_add(name_, t0_, t1);
    }
    return HS_OK;
  }
  // One kernel launch.  When the previous operation this launcher put on the
  // stream was a kernel (and no timing events sit between them), the launch
  // is a programmatic dependent launch: the launch is processed while the
  // previous kernel runs and its CTAs start as soon as that kernel completes;
  // every kernel of the library opens with griddepcontrol.wait, which returns
  // once the previous kernel has completed and its writes are visible.  No
  // kernel releases its dependents early: CTAs of the next kernel parked on
  // the SMs while a long persistent kernel runs cost more than they save.
  template <class... KArgs, class... Args>
  hs_status kernel(const char* name, void (*f)(KArgs...), dim3 grid, dim3 block, size_t smem, Args&&... args) {
    begin(name);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st_;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = (prev_kernel_ && !t0_) ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(&cfg, f, std::forward<Args>(args)...);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return HS_ERR_CUDA;
    }
    prev_kernel_ = true;
    return end();
  }
  hs_status memset(const char* name, void* p, int v, size_t bytes) {
    if (!bytes) return HS_OK;
    prev_kernel_ = false;
    begin(name);
    cudaError_t e = cudaMemsetAsync(p, v, bytes, st_);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return HS_ERR_CUDA;
    }
    return end(false);
  }
  hs_status copy(const char* name, void* dst, const void* src, size_t bytes,
                 cudaMemcpyKind kind = cudaMemcpyDeviceToDevice) {
    if (!bytes) return HS_OK;
    prev_kernel_ = false;
    begin(name);
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, st_);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return HS_ERR_CUDA;
    }
    return end(false);
  }

 private:
  cudaStream_t st_;
  const char* name_ = "";
  cudaEvent_t t0_ = nullptr;
  bool prev_kernel_ = false;
};

// Entry points of the per-(key type, tile shape) translation units
// (sort_shape.cu): run_sort_<key>_t<items per thread>.
// `src`: nullptr, or the keys in pinned host memory the device can address
// (hs_sort_keys_host): the sort then reads them from there into `keys`, and
// sets *host_done (when given) to 1 if it also wrote the sorted keys back
// there (else the caller copies `keys` back).
#define HS_SORT_SHAPE_DECL(name)                                                                            \
  hs_status name(void* keys, uint32_t* vals, size_t n, size_t nseg, const uint64_t* offs, const hs_opts& o, \
                 char* ws, uint32_t* err, cudaStream_t st, const void* src, int* host_done)
HS_SORT_SHAPE_DECL(run_sort_i32_t11);
HS_SORT_SHAPE_DECL(run_sort_i32_t15);
HS_SORT_SHAPE_DECL(run_sort_i32_t23);
HS_SORT_SHAPE_DECL(run_sort_i32_t31);
HS_SORT_SHAPE_DECL(run_sort_u32_t11);
HS_SORT_SHAPE_DECL(run_sort_u32_t15);
HS_SORT_SHAPE_DECL(run_sort_u32_t23);
HS_SORT_SHAPE_DECL(run_sort_u32_t31);
HS_SORT_SHAPE_DECL(run_sort_u64_t11);
HS_SORT_SHAPE_DECL(run_sort_u64_t15);
size_t workspace_bytes(size_t key_bytes, size_t n, bool has_vals, size_t nseg, int nb);

}  // namespace hs
