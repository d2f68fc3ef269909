// The C ABI of include/hsort.h: argument checks, work-space management per
// (device, stream), dispatch to the per-key-type drivers, the device error
// word, CUDA-event timing and the launch counter.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "driver.cuh"

namespace hs {

// The device error word: one per device (every device that loads the library
// holds its own copy).  Kernels set bits with atomicOr; hs_stream_error reads
// and clears it.
__device__ uint32_t g_err_word;

namespace {

std::mutex g_mu;

struct Buf {
  char* ptr = nullptr;
  size_t bytes = 0;
};
std::map<std::pair<int, cudaStream_t>, Buf> g_ws;       // work space per (device, stream)
std::map<std::pair<int, cudaStream_t>, Buf> g_stage;    // host-call staging per (device, stream)
std::map<int, uint32_t*> g_err_ptr;                      // device address of g_err_word per device

thread_local std::string t_last_error;

std::atomic<bool> g_timing{false};
struct TimeRec {
  const char* name;
  cudaEvent_t a, b;
};
std::vector<TimeRec> g_times;
std::vector<cudaEvent_t> g_event_pool;
std::atomic<unsigned long long> g_launches{0};

// CUDA graphs of whole calls, keyed by every argument that shapes the launch
// sequence (pointers included: a graph replays with the addresses it saw).
struct GraphKey {
  int dev;
  cudaStream_t st;
  int dtype;
  void* keys;
  uint32_t* vals;
  const uint64_t* offs;
  size_t n, nseg;
  int partition, stop_after, debug, fan_in, tile, merge;
  uint64_t* pkt_out;
  void* ws;
  size_t ws_bytes;
  const void* src;
  bool operator<(const GraphKey& o) const {
    return std::tie(dev, st, dtype, keys, vals, offs, n, nseg, partition, stop_after, debug, fan_in, tile, merge, pkt_out, ws,
                    ws_bytes, src) < std::tie(o.dev, o.st, o.dtype, o.keys, o.vals, o.offs, o.n, o.nseg, o.partition,
                                              o.stop_after, o.debug, o.fan_in, o.tile, o.merge, o.pkt_out, o.ws,
                                              o.ws_bytes, o.src);
  }
};
struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  unsigned long long kernels = 0;
  unsigned long long stamp = 0;
  int host_done = 0;  // the captured kernels write the sorted keys back to host memory
};
constexpr size_t kMaxGraphs = 64;
std::map<GraphKey, GraphEntry> g_graphs;
unsigned long long g_graph_clock = 0;

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

hs_status err_ptr(uint32_t** out) {
  const int dev = current_device();
  auto it = g_err_ptr.find(dev);
  if (it != g_err_ptr.end()) {
    *out = it->second;
    return HS_OK;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_err_word);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return HS_ERR_CUDA;
  }
  g_err_ptr[dev] = static_cast<uint32_t*>(p);
  *out = static_cast<uint32_t*>(p);
  return HS_OK;
}

hs_status grow(std::map<std::pair<int, cudaStream_t>, Buf>& m, cudaStream_t st, size_t need, char** out) {
  auto& b = m[{current_device(), st}];
  if (b.bytes < need) {
    if (b.ptr) {
      cudaError_t e = cudaFree(b.ptr);  // synchronises the device
      b.ptr = nullptr;
      b.bytes = 0;
      if (e != cudaSuccess) {
        set_cuda_error(e);
        return HS_ERR_CUDA;
      }
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_cuda_error(e);
      return HS_ERR_NOMEM;
    }
    b.ptr = static_cast<char*>(p);
    b.bytes = need;
  }
  *out = b.ptr;
  return HS_OK;
}

size_t key_bytes(hs_dtype dt) { return dt == HS_UINT64 ? 8 : 4; }

// Tuning table: merge fan-in per (key type, values, partition, size bucket).
struct TuneKey {
  int dtype, has_vals, partition, log2n;
  bool operator<(const TuneKey& o) const {
    return std::tie(dtype, has_vals, partition, log2n) < std::tie(o.dtype, o.has_vals, o.partition, o.log2n);
  }
};
// value: the fan-in and the tile of the shape (0 = the built-in rule's)
struct TuneVal {
  int fan_in = 0, tile = 0, merge = 0;
};
std::map<TuneKey, TuneVal> g_tune;
std::mutex g_tune_mu;

int size_bucket(size_t n) {
  int b = 0;
  while (b < 63 && (static_cast<size_t>(1) << b) < n) ++b;
  return b;
}
// The shape a call with fan_in == 0 / tile == 0 uses: the tuning table's
// entry for its (key type, values, partition, size bucket), else the built-in
// rule from one GB300: four-way passes while passes are short (launch- and
// latency-bound), two-way passes above 2^21 keys; the default tile.
void tuned_shape(int dtype, bool has_vals, int partition, size_t n, int* fan_in, int* tile, int* merge = nullptr) {
  TuneVal v;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(TuneKey{dtype, has_vals ? 1 : 0, partition, size_bucket(n)});
    if (it != g_tune.end()) v = it->second;
  }
  if (fan_in) *fan_in = v.fan_in ? v.fan_in : (n <= (static_cast<size_t>(1) << 21) ? 4 : 2);
  if (tile) *tile = v.tile ? v.tile : sort_tile_for(dtype == HS_UINT64 ? 8 : 4, has_vals);
  // two-way passes in one persistent launch once passes are long; below, the
  // queue's pass-to-pass hand-over costs more than a launch per pass
  // (measured on one GB300: 64-bit keys from 2^25 keys on, 4-byte keys above
  // 2^26; key-value pairs up to 2^27, the largest size measured, never)
  const bool queue = !has_vals && n > (static_cast<size_t>(1) << (dtype == HS_UINT64 ? 24 : 26));
  if (merge) *merge = v.merge ? v.merge : (queue ? kMergeQueue : kMergePerPass);
}
int tuned_fan_in(int dtype, bool has_vals, int partition, size_t n) {
  int f = 0;
  tuned_shape(dtype, has_vals, partition, n, &f, nullptr);
  return f;
}

// The per-(key type, tile shape) entry points of sort_shape.cu.
hs_status run_shape(hs_dtype dt, int tile, void* keys, uint32_t* vals, size_t n, size_t nseg, const uint64_t* offs,
                    const hs_opts& o, char* ws, uint32_t* err, cudaStream_t st, const void* src, int* host_done) {
  const int ipt = tile / kBlock;
  switch (dt) {
    case HS_INT32:
      switch (ipt) {
        case 11: return run_sort_i32_t11(keys, vals, n, nseg, offs, o, ws, err, st, src, host_done);
        case 15: return run_sort_i32_t15(keys, vals, n, nseg, offs, o, ws, err, st, src, host_done);
        case 23: return run_sort_i32_t23(keys, vals, n, nseg, offs, o, ws, err, st, src, host_done);
        case 31: return run_sort_i32_t31(keys, vals, n, nseg, offs, o, ws, err, st, src, host_done);
      }
      break;
    case HS_UINT32:
      switch (ipt) {
        case 11: return run_sort_u32_t11(keys, vals, n, nseg, offs, o, ws, err, st, src, host_done);
        case 15: return run_sort_u32_t15(keys, vals, n, nseg, offs, o, ws, err, st, src, host_done);
        case 23: return run_sort_u32_t23(keys, vals, n, nseg, offs, o, ws, err, st, src, host_done);
        case 31: return run_sort_u32_t31(keys, vals, n, nseg, offs, o, ws, err, st, src, host_done);
      }
      break;
    default:
      switch (ipt) {
        case 11: return run_sort_u64_t11(keys, vals, n, nseg, offs, o, ws, err, st, src, host_done);
        case 15: return run_sort_u64_t15(keys, vals, n, nseg, offs, o, ws, err, st, src, host_done);
      }
      break;
  }
  return HS_ERR_UNSUPPORTED;
}

hs_status check_opts(const hs_opts* opts, hs_opts* o) {
  hs_opts d{};
  if (opts) d = *opts;
  if (d.partition == 0) d.partition = 10;
  if (d.partition != 1 && d.partition != 10 && d.partition != 256) return HS_ERR_INVALID;
  if (d.tile != 0 && !tile_built(4, false, d.tile) && !tile_built(4, true, d.tile)) return HS_ERR_UNSUPPORTED;
  if (d.fan_in != 0 && d.fan_in != 2 && d.fan_in != 4) return HS_ERR_UNSUPPORTED;
  if (d.stop_after < 0 || d.stop_after > 2 + kMaxPasses) return HS_ERR_INVALID;
  if (d.merge != 0 && d.merge != kMergeQueue && d.merge != kMergePerPass) return HS_ERR_UNSUPPORTED;
  *o = d;
  return HS_OK;
}

// src: nullptr, or the keys in pinned host memory the device can address
// (hs_sort_keys_host); `keys` is then the device array they are sorted in,
// and *host_done (when given) tells whether the sorted keys were also written
// back to src by the call's kernels.
hs_status dispatch(hs_dtype dt, void* keys, uint32_t* vals, size_t n, size_t nseg, const uint64_t* offs,
                   const hs_opts* opts, void* stream, const void* src = nullptr, int* host_done = nullptr) {
  if (host_done) *host_done = 0;
  if (dt != HS_INT32 && dt != HS_UINT32 && dt != HS_UINT64) return HS_ERR_INVALID;
  hs_opts o;
  HS_TRY(check_opts(opts, &o));
  if (n >= (1ull << 32) || nseg >= (1ull << 24)) return HS_ERR_INVALID;
  if (n > 0 && !keys) return HS_ERR_INVALID;
  // element alignment (the kernels load whole elements)
  if ((reinterpret_cast<uintptr_t>(keys) % key_bytes(dt)) || (reinterpret_cast<uintptr_t>(vals) & 3u) ||
      (reinterpret_cast<uintptr_t>(offs) & 7u))
    return HS_ERR_INVALID;
  if (o.tile != 0 && !tile_built(key_bytes(dt), vals != nullptr, o.tile)) return HS_ERR_UNSUPPORTED;
  {
    int f = 0, t = 0, m = 0;
    tuned_shape(static_cast<int>(dt), vals != nullptr, o.partition, n, &f, &t, &m);
    if (o.fan_in == 0) o.fan_in = f;
    if (o.tile == 0) o.tile = t;
    if (o.merge == 0) o.merge = m;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n == 0 && !offs) {
    if (o.d_packet_offsets_out) {
      cudaError_t e = cudaMemsetAsync(o.d_packet_offsets_out, 0, (o.partition + 1) * 8, st);
      if (e != cudaSuccess) {
        set_cuda_error(e);
        return HS_ERR_CUDA;
      }
    }
    return HS_OK;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  uint32_t* err = nullptr;
  HS_TRY(err_ptr(&err));
  const size_t need = workspace_bytes(key_bytes(dt), n, vals != nullptr, nseg, o.partition);
  char* ws = nullptr;
  if (o.d_workspace) {
    if (o.workspace_bytes < need || (reinterpret_cast<uintptr_t>(o.d_workspace) & 255u)) return HS_ERR_INVALID;
    ws = static_cast<char*>(o.d_workspace);
  } else {
    HS_TRY(grow(g_ws, st, need, &ws));
  }
  auto run = [&]() -> hs_status {
    switch (dt) {
      default: return run_shape(dt, o.tile, keys, vals, n, nseg, offs, o, ws, err, st, src, host_done);
    }
  };
  if (!o.graph || st == nullptr || timing_on()) return run();
  const GraphKey key{current_device(), st, static_cast<int>(dt), keys, vals, offs, n, nseg, o.partition,
                     o.stop_after, o.debug_flags, o.fan_in, o.tile, o.merge, o.d_packet_offsets_out, ws,
                     o.d_workspace ? o.workspace_bytes : need, src};
  auto it = g_graphs.find(key);
  if (it == g_graphs.end()) {
    if (g_graphs.size() >= kMaxGraphs) {  // evict the least recently used graph
      auto old = g_graphs.begin();
      for (auto j = g_graphs.begin(); j != g_graphs.end(); ++j)
        if (j->second.stamp < old->second.stamp) old = j;
      cudaGraphExecDestroy(old->second.exec);
      g_graphs.erase(old);
    }
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return HS_ERR_CUDA;
    }
    const unsigned long long l0 = g_launches.load();
    hs_status rs = run();
    const unsigned long long kernels = g_launches.load() - l0;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(st, &graph);
    if (rs != HS_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) set_cuda_error(e);
      return rs != HS_OK ? rs : HS_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return HS_ERR_CUDA;
    }
    g_launches.fetch_sub(kernels);  // captured, not launched: counted when replayed
    it = g_graphs.emplace(key, GraphEntry{exec, kernels, 0, host_done ? *host_done : 0}).first;
  }
  if (host_done) *host_done = it->second.host_done;
  it->second.stamp = ++g_graph_clock;
  cudaError_t e = cudaGraphLaunch(it->second.exec, st);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return HS_ERR_CUDA;
  }
  g_launches.fetch_add(it->second.kernels);
  return HS_OK;
}

}  // namespace

bool timing_on() { return g_timing.load(std::memory_order_relaxed); }

cudaEvent_t event_get() {
  // called with g_mu held (from inside a sort call)
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void timing_add(const char* name, cudaEvent_t a, cudaEvent_t b) { g_times.push_back({name, a, b}); }

void set_cuda_error(cudaError_t e) { t_last_error = cudaGetErrorString(e); }

void set_error_message(const char* msg) { t_last_error = msg; }

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

size_t workspace_bytes(size_t kb, size_t n, bool has_vals, size_t nseg, int nb) {
  return make_layout(kb, n, has_vals, nseg, nb).total;
}

}  // namespace hs

using namespace hs;

extern "C" {

hs_status hs_sort_keys(hs_dtype dtype, void* d_keys, size_t n, const hs_opts* opts, void* stream) {
  return dispatch(dtype, d_keys, nullptr, n, 1, nullptr, opts, stream);
}

hs_status hs_sort_pairs(hs_dtype dtype, void* d_keys, uint32_t* d_vals, size_t n, int stable, const hs_opts* opts,
                        void* stream) {
  (void)stable;  // the result is always the stable order
  if (n > 0 && !d_vals) return HS_ERR_INVALID;
  return dispatch(dtype, d_keys, d_vals, n, 1, nullptr, opts, stream);
}

hs_status hs_sort_batch(hs_dtype dtype, void* d_keys, uint32_t* d_vals, const uint64_t* d_offsets, size_t nseg,
                        size_t n, const hs_opts* opts, void* stream) {
  if (nseg == 0) return n == 0 ? HS_OK : HS_ERR_INVALID;
  if (!d_offsets) return HS_ERR_INVALID;
  return dispatch(dtype, d_keys, d_vals, n, nseg, d_offsets, opts, stream);
}

hs_status hs_sort_keys_host(hs_dtype dtype, void* h_keys, size_t n, const hs_opts* opts, void* stream) {
  if (dtype != HS_INT32 && dtype != HS_UINT32 && dtype != HS_UINT64) return HS_ERR_INVALID;
  if (n == 0) return HS_OK;
  if (!h_keys || n >= (1ull << 32) || (reinterpret_cast<uintptr_t>(h_keys) % key_bytes(dtype))) return HS_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = n * key_bytes(dtype);
  char* d = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    HS_TRY(grow(g_stage, st, bytes, &d));
  }
  // Pinned host memory that the device can address is read by the sort's
  // first pass itself (the histogram copies the keys in while it counts
  // them); other host memory is copied in first.
  const void* src = nullptr;
  cudaPointerAttributes pa{};
  const cudaError_t ea = cudaPointerGetAttributes(&pa, h_keys);
  if (ea == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer != nullptr)
    src = pa.devicePointer;  // an address of that memory the current device can load from
  else if (ea != cudaSuccess)
    cudaGetLastError();  // the query's own error (older runtimes reject unregistered pointers): not the caller's
  cudaError_t e = cudaSuccess;
  if (!src) {
    e = cudaMemcpyAsync(d, h_keys, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return HS_ERR_CUDA;
    }
  }
  int host_done = 0;
  hs_status s = dispatch(dtype, d, nullptr, n, 1, nullptr, opts, stream, src, &host_done);
  if (s != HS_OK) return s;
  // the kernels wrote the result back themselves (merge passes in one
  // persistent launch), or it is copied back now
  if (!host_done) e = cudaMemcpyAsync(h_keys, d, bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return HS_ERR_CUDA;
  }
  return HS_OK;
}

hs_status hs_workspace_size(hs_dtype dtype, size_t n, int has_vals, size_t nseg, const hs_opts* opts, size_t* bytes) {
  if (!bytes || (dtype != HS_INT32 && dtype != HS_UINT32 && dtype != HS_UINT64)) return HS_ERR_INVALID;
  hs_opts o;
  HS_TRY(check_opts(opts, &o));
  if (nseg == 0) nseg = 1;
  *bytes = workspace_bytes(key_bytes(dtype), n, has_vals != 0, nseg, o.partition);
  return HS_OK;
}

hs_status hs_workspace_reserve(size_t bytes, void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  char* p = nullptr;
  return grow(g_ws, static_cast<cudaStream_t>(stream), bytes, &p);
}

hs_status hs_workspace_release(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  const int dev = current_device();
  for (auto* m : {&g_ws, &g_stage}) {
    for (auto it = m->begin(); it != m->end();) {
      if (it->first.first == dev) {
        if (it->second.ptr) cudaFree(it->second.ptr);
        it = m->erase(it);
      } else {
        ++it;
      }
    }
  }
  return HS_OK;
}

hs_status hs_tune_set(hs_dtype dtype, int has_vals, int partition, int log2n, int fan_in) {
  if (dtype != HS_INT32 && dtype != HS_UINT32 && dtype != HS_UINT64) return HS_ERR_INVALID;
  if (partition != 1 && partition != 10 && partition != 256) return HS_ERR_INVALID;
  if (log2n < 0 || log2n > 32 || (fan_in != 2 && fan_in != 4)) return HS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[TuneKey{static_cast<int>(dtype), has_vals ? 1 : 0, partition, log2n}].fan_in = fan_in;
  return HS_OK;
}

hs_status hs_tune_set_shape(hs_dtype dtype, int has_vals, int partition, int log2n, int fan_in, int tile,
                            int merge) {
  if (dtype != HS_INT32 && dtype != HS_UINT32 && dtype != HS_UINT64) return HS_ERR_INVALID;
  if (partition != 1 && partition != 10 && partition != 256) return HS_ERR_INVALID;
  if (log2n < 0 || log2n > 32 || (fan_in != 0 && fan_in != 2 && fan_in != 4)) return HS_ERR_INVALID;
  if (tile != 0 && !tile_built(key_bytes(dtype), has_vals != 0, tile)) return HS_ERR_INVALID;
  if (merge != 0 && merge != kMergeQueue && merge != kMergePerPass) return HS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  TuneVal& v = g_tune[TuneKey{static_cast<int>(dtype), has_vals ? 1 : 0, partition, log2n}];
  v.fan_in = fan_in;
  v.tile = tile;
  v.merge = merge;
  return HS_OK;
}

hs_status hs_tune_get_shape(hs_dtype dtype, int has_vals, int partition, size_t n, int* fan_in, int* tile,
                            int* merge) {
  if (!fan_in || !tile || !merge || (dtype != HS_INT32 && dtype != HS_UINT32 && dtype != HS_UINT64))
    return HS_ERR_INVALID;
  if (partition == 0) partition = 10;
  if (partition != 1 && partition != 10 && partition != 256) return HS_ERR_INVALID;
  tuned_shape(static_cast<int>(dtype), has_vals != 0, partition, n, fan_in, tile, merge);
  return HS_OK;
}

hs_status hs_tiles(hs_dtype dtype, int has_vals, int* tiles, int max, int* count) {
  if (!count || (dtype != HS_INT32 && dtype != HS_UINT32 && dtype != HS_UINT64) || (max > 0 && !tiles))
    return HS_ERR_INVALID;
  int c = 0;
  for (int ipt : kTileIpts) {
    if (!tile_built(key_bytes(dtype), has_vals != 0, kBlock * ipt)) continue;
    if (c < max) tiles[c] = kBlock * ipt;
    ++c;
  }
  *count = c;
  return HS_OK;
}

hs_status hs_tune_get(hs_dtype dtype, int has_vals, int partition, size_t n, int* fan_in) {
  if (!fan_in || (dtype != HS_INT32 && dtype != HS_UINT32 && dtype != HS_UINT64)) return HS_ERR_INVALID;
  if (partition == 0) partition = 10;
  if (partition != 1 && partition != 10 && partition != 256) return HS_ERR_INVALID;
  *fan_in = tuned_fan_in(static_cast<int>(dtype), has_vals != 0, partition, n);
  return HS_OK;
}

hs_status hs_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  return HS_OK;
}

hs_status hs_graph_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& kv : g_graphs) cudaGraphExecDestroy(kv.second.exec);
  g_graphs.clear();
  return HS_OK;
}

hs_status hs_stream_error(void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return HS_ERR_CUDA;
  }
  uint32_t* p = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    HS_TRY(err_ptr(&p));
  }
  uint32_t w = 0;
  e = cudaMemcpy(&w, p, 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(p, 0, 4);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return HS_ERR_CUDA;
  }
  if (w & kErrTimeout) return HS_ERR_TIMEOUT;
  if (w & kErrBadOffsets) return HS_ERR_INVALID;
  if (w & kErrBounds) return HS_ERR_DEVICE;
  return HS_OK;
}

hs_status hs_plan_describe(hs_dtype dtype, size_t n, int has_vals, size_t nseg, const hs_opts* opts, hs_plan* out) {
  if (!out || (dtype != HS_INT32 && dtype != HS_UINT32 && dtype != HS_UINT64)) return HS_ERR_INVALID;
  hs_opts o;
  HS_TRY(check_opts(opts, &o));
  if (o.tile != 0 && !tile_built(key_bytes(dtype), has_vals != 0, o.tile)) return HS_ERR_UNSUPPORTED;
  {
    int f = 0, t = 0, m = 0;
    tuned_shape(static_cast<int>(dtype), has_vals != 0, o.partition, n, &f, &t, &m);
    if (o.fan_in == 0) o.fan_in = f;
    if (o.tile == 0) o.tile = t;
    if (o.merge == 0) o.merge = m;
  }
  out->tile = o.tile;
  out->part_tile = kTile;
  out->fan_in = o.fan_in;
  out->merge_passes = (n == 0) ? 0 : worst_passes(n, static_cast<size_t>(out->tile), o.fan_in);
  // seg_plan, hist (x2 for int32), finalize, fold, 3 scan kernels, pkt, scan_units, scatter,
  // tilesort, 2 per merge pass; without the packet step: seg_plan, pkt, scan_units, tilesort.
  // Small calls run finalize .. scan_units (or pkt, scan_units) as one kernel.
  const Layout L = make_layout(key_bytes(dtype), n, has_vals != 0, nseg ? nseg : 1, o.partition);
  const bool small = static_cast<uint64_t>(L.max_blocks) * o.partition <= kPlanSmallEntries &&
                     static_cast<uint64_t>(L.npk) <= kPlanSmallEntries;
  const int plan_kernels = small ? 1 : (o.partition == 1 ? 2 : 7);
  int l = (o.partition == 1) ? 1 + plan_kernels : 1 + (dtype == HS_INT32 ? 2 : 1) + plan_kernels + 1;
  // one short array (at most a tile) skips the packet-step kernels: the tile
  // sort launch sorts it whole
  if (o.stop_after == 0 && (nseg ? nseg : 1) == 1 && n <= static_cast<size_t>(out->tile)) l = 1 + plan_kernels;
  if (o.stop_after != 1) l += 1;
  // fan-in 2: every merge pass in one persistent launch; fan-in 4 (and the
  // per-pass ablation, debug flag 4): two launches per pass
  const bool sched = o.fan_in == 2 && o.merge == kMergeQueue;
  auto merge_launches = [&](int p) { return p == 0 ? 0 : (sched ? 1 : 2 * p); };
  if (o.stop_after == 0) l += merge_launches(out->merge_passes);
  if (o.stop_after >= 3) l += merge_launches(std::min(out->merge_passes, o.stop_after - 2)) + 1;
  out->launches = (n == 0) ? 0 : l;
  return HS_OK;
}

hs_status hs_timing_enable(int on) {
  g_timing.store(on != 0);
  return HS_OK;
}

hs_status hs_timing_read_launches(hs_kernel_time* out, int max, int* count) {
  if ((!out && max > 0) || max < 0) return HS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return HS_ERR_CUDA;
  }
  int c = 0;
  for (auto& r : g_times) {
    if (c < max) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, r.a, r.b);
      hs_kernel_time k{};
      std::snprintf(k.name, sizeof(k.name), "%s", r.name);
      k.launches = 1;
      k.total_ms = ms;
      out[c++] = k;
    }
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_times.clear();
  if (count) *count = c;
  return HS_OK;
}

hs_status hs_timing_read(hs_kernel_time* out, int max, int* count) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return HS_ERR_CUDA;
  }
  std::vector<hs_kernel_time> agg;
  for (auto& r : g_times) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    size_t i = 0;
    for (; i < agg.size(); ++i)
      if (std::strcmp(agg[i].name, r.name) == 0) break;
    if (i == agg.size()) {
      hs_kernel_time k{};
      std::snprintf(k.name, sizeof(k.name), "%s", r.name);
      agg.push_back(k);
    }
    agg[i].launches += 1;
    agg[i].total_ms += ms;
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_times.clear();
  int c = 0;
  for (size_t i = 0; i < agg.size() && c < max; ++i) out[c++] = agg[i];
  if (count) *count = c;
  return HS_OK;
}

unsigned long long hs_kernel_launches(void) { return g_launches.load(); }

const char* hs_status_string(hs_status s) {
  switch (s) {
    case HS_OK: return "ok";
    case HS_ERR_INVALID: return "invalid argument";
    case HS_ERR_NOMEM: return "out of device memory";
    case HS_ERR_CUDA: return "CUDA error";
    case HS_ERR_TIMEOUT: return "bounded device wait expired";
    case HS_ERR_UNSUPPORTED: return "unsupported option";
    case HS_ERR_DEVICE: return "device-side consistency check failed";
  }
  return "unknown status";
}

const char* hs_last_error(void) { return t_last_error.c_str(); }

}  // extern "C"
