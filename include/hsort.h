/*
 * hsort.h -- C ABI of a GPU (sm_103a) implementation of the hybrid sort of
 * Alghamdi & Alaghband, "High Performance Parallel Sort for Shared and
 * Distributed Memory MIMD" (arXiv 2003.01216).
 *
 * The method (Sec. 3.4, with the per-node sort of Sec. 3.2):
 *   1. one MSD-radix step divides the keys into ten packets by their most
 *      significant decimal digit; packets do not overlap in value (Sec. 2.1);
 *   2. every packet is sorted independently: its data is split into parts that
 *      are sorted one by one (quicksort in the paper, Fig. 1(c); here,
 *      sorting networks and merges inside one thread block per tile);
 *   3. the sorted parts are merged bottom-up, pairwise, until each packet is
 *      one sorted run (non-recursive merge, Fig. 1(b), Sec. 3.2);
 *   4. each sorted packet lands at its place in the original array (Sec. 3.4).
 *
 * Conventions for every call:
 *   - Device pointers are CUDA device (or managed) memory of the current
 *     device.  The caller owns every buffer it passes.  Sorts are IN PLACE and
 *     ascending.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Every sort call is asynchronous on `stream`: it only enqueues
 *     work and never synchronises the host (except hs_sort_keys_host).
 *   - Keys and key images: packets are cut on an order-preserving unsigned
 *     image u of each key: u = key for uint32/uint64 keys and for int32 arrays
 *     without negative keys; u = key XOR 2^31 for int32 arrays holding a
 *     negative key.  D = number of decimal digits of the largest u and
 *     packet(u) = floor(u / 10^(D-1)).  The 256-bucket ablation uses
 *     bucket(u) = u >> max(0, B - 8), B = bit length of the largest u.
 *   - Sizes: n < 2^32 elements per call (and per batch).
 *   - Host-detectable errors return at once and enqueue nothing.  Errors found
 *     on the device (a bounded wait that expired, malformed batch offsets) set
 *     bits of an error word held once per device; hs_stream_error() reads and
 *     clears it.  Calls running on several streams of one device share that
 *     word, so an error can be reported to whichever stream asks first.
 *   - Work space: unless opts->d_workspace is given, the library keeps one
 *     device work buffer per (device, stream), grown on demand with cudaMalloc
 *     and reused; growth synchronises the device.  Calls on the same stream
 *     share it (they are ordered); calls on different streams never share it.
 *   - Thread safety: calls may come from several host threads; the library's
 *     tables are guarded by a mutex.
 */
#ifndef HSORT_H
#define HSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HS_OK = 0,
  HS_ERR_INVALID = 1,     /* bad argument (null pointer with n > 0, bad dtype, n too large, ...) */
  HS_ERR_NOMEM = 2,       /* device work space could not be allocated */
  HS_ERR_CUDA = 3,        /* a CUDA launch or runtime call failed */
  HS_ERR_TIMEOUT = 4,     /* a bounded device-side wait expired (reported by hs_stream_error) */
  HS_ERR_UNSUPPORTED = 5, /* option not built (e.g. a tile shape that has no kernel) */
  HS_ERR_DEVICE = 6       /* device-side consistency check failed (reported by hs_stream_error) */
} hs_status;

typedef enum { HS_INT32 = 0, HS_UINT32 = 1, HS_UINT64 = 2 } hs_dtype;

/* Optional knobs.  A NULL hs_opts*, or any zero field, means "default". */
typedef struct {
  int partition;        /* 10 (default): MSD decimal packets (Sec. 3.4); 256: top-8-bit ablation;
                           1: no MSD step, the whole array is one packet (the shared-memory
                           hybrid of Sec. 3.2 alone; ablation) */
  int tile;             /* keys per tile of the per-packet sort (= 256 threads x items per thread;
                           also the outputs of one merge block).  Built tiles (hs_tiles): 3840,
                           5888 and 7936 for 4-byte keys without values; 2816 and 3840 otherwise.
                           0 = tuned: the tuning table's entry (hs_tune_set_shape), else 7936
                           for 4-byte keys without values and 3840 otherwise.  A tile not built
                           for the call's key type returns HS_ERR_UNSUPPORTED */
  int fan_in;           /* runs merged per merge pass (Fig. 1(b) merges two): 2, or 4 (every
                           pass merges groups of four adjacent runs, so half the passes over
                           memory; same result bit for bit), or 0 = tuned: the entry of the
                           tuning table (hs_tune_set) for this key type, values, partition
                           and size bucket, else 4 up to 2^21 keys and 2 above.  Other values
                           return HS_ERR_UNSUPPORTED */
  int stop_after;       /* testing: 0 = whole sort; 1 = stop after the packet step
                           (array holds the stable packet layout); 2 = stop after the
                           tile sort (every tile of every packet sorted on its own);
                           2 + r (r = 1 .. 64) = stop after merge pass r (inside every
                           packet, each group of fan_in^r tiles sorted on its own, pairs
                           stably; packets needing fewer passes fully sorted).  Other
                           values: HS_ERR_INVALID */
  uint64_t* d_packet_offsets_out; /* optional device array of partition*nseg + 1 uint64:
                           packet p of segment s spans [off[s*partition + p], off[s*partition+p+1])
                           as absolute element positions */
  void* d_workspace;    /* optional caller-owned device work space (see hs_workspace_size),
                           256-byte aligned (else HS_ERR_INVALID); when set, the library
                           allocates nothing for this call */
  size_t workspace_bytes;
  int debug_flags;      /* testing only: bit 0 = one bulk copy of the tile sort announces 16
                           bytes that never arrive and the wait limit is shortened, so a
                           bounded wait expires; bit 1 = in the persistent merge launch, the
                           first merge block never publishes its completion and the wait limit
                           is shortened, so the blocks that read its run give up; bit 2 = as
                           bit 0, for a bulk copy of the packet step's scatter (ten packets).
                           Each reports HS_ERR_TIMEOUT (the keys are then unspecified) */
  int graph;            /* 1 = capture this call's whole launch sequence in a CUDA graph the
                           first time these exact arguments (pointers, sizes, options, stream)
                           are seen, and replay the instantiated graph on later calls.  Needs a
                           created stream (the legacy default stream cannot be captured) and
                           per-kernel timing off; otherwise the call runs without a graph.  The
                           library keeps up to 64 graphs; hs_graph_cache_clear frees them. */
  int merge;            /* how two-way merge passes are launched (the result is the same):
                           1 = every pass in one persistent launch, a work queue of
                           (packet, pass, merge block) items each started as soon as the runs
                           it reads are complete; 2 = one co-rank and one merge launch per
                           pass; 0 = tuned: the tuning table's entry, else 1 above 2^24 keys
                           (64-bit keys without values) or 2^26 keys (4-byte keys without
                           values), 2 otherwise.  Other values: HS_ERR_UNSUPPORTED */
} hs_opts;

/*
 * hs_sort_keys -- sort n keys in place, ascending (Sec. 3.4: MSD step, then
 * per-packet sort and bottom-up merge; the whole array is one "original
 * array" of the master node).
 *   dtype   HS_INT32 / HS_UINT32 / HS_UINT64 (4, 4, 8 bytes per key)
 *   d_keys  device pointer to n keys, aligned to the key size (4 or 8 bytes;
 *           else HS_ERR_INVALID), no other alignment needed
 *   n       element count; 0 is a no-op returning HS_OK
 * Returns HS_OK once the work is enqueued, HS_ERR_INVALID, HS_ERR_NOMEM or
 * HS_ERR_CUDA.
 */
hs_status hs_sort_keys(hs_dtype dtype, void* d_keys, size_t n, const hs_opts* opts, void* stream);

/*
 * hs_sort_pairs -- sort n (key, value) pairs in place by key.  The order is
 * stable: equal keys keep their input order (merge sort's stability, Sec. 2.1;
 * ties broken by input index).  `stable` = 0 is accepted and returns the same
 * stable order.  d_vals: device pointer to n uint32 values (4-byte aligned, else
 * HS_ERR_INVALID), moved with their keys.
 */
hs_status hs_sort_pairs(hs_dtype dtype, void* d_keys, uint32_t* d_vals, size_t n, int stable,
                        const hs_opts* opts, void* stream);

/*
 * hs_sort_batch -- segmented sort: nseg independent arrays stored back to
 * back in d_keys; segment s is [d_offsets[s], d_offsets[s+1]).  Each segment
 * goes through the whole method on its own (its own D and packets).
 *   d_offsets  device array of nseg + 1 uint64 (8-byte aligned, else HS_ERR_INVALID),
 *              non-decreasing, d_offsets[0] = 0,
 *              d_offsets[nseg] = n (checked on the device: a violation sets
 *              the error word so hs_stream_error returns HS_ERR_INVALID, and no
 *              key moves)
 *   d_vals     optional (NULL = keys only); when given, pairs sort stably
 *   n          total element count (the host cannot read d_offsets without a sync)
 */
hs_status hs_sort_batch(hs_dtype dtype, void* d_keys, uint32_t* d_vals, const uint64_t* d_offsets,
                        size_t nseg, size_t n, const hs_opts* opts, void* stream);

/*
 * hs_sort_keys_host -- the same sort for keys in HOST memory: the n keys go
 * to a library-owned device staging buffer, are sorted there and are copied
 * back; `stream` is synchronised before returning.  Pinned host memory that
 * the device can address (cudaHostAlloc / cudaMallocHost, or registered with
 * cudaHostRegister and mapped; with unified addressing every pinned block is)
 * is read by the sort's first pass itself: the histogram kernel loads the
 * keys from host memory and writes them to the staging buffer while it
 * counts them, so the copy in and the histogram are one pass (a call without
 * a histogram -- partition 1, or n of at most one tile -- copies them in
 * first); and when the call's merge passes run in one persistent launch
 * (hs_opts.merge), the last merge pass of every packet writes its blocks
 * straight into the host array (packet by packet, so that one packet's
 * writes over the host link overlap the next packets' device passes) and
 * the packets that need no merge pass are copied there by a small kernel,
 * so no separate copy out follows.  Pageable
 * memory is copied in and out with cudaMemcpyAsync.  Same result either way.
 */
hs_status hs_sort_keys_host(hs_dtype dtype, void* h_keys, size_t n, const hs_opts* opts, void* stream);

/*
 * hs_sort_keys_noalloc -- hs_sort_keys for callers that cannot allocate device
 * memory (the paper has no counterpart: this is an interface for such callers,
 * e.g. code inside a stream capture that must hold no allocation, or a host
 * framework that owns every device allocation).  The scratch lives in a
 * fixed 16 MiB device array inside this library; every GPU that loads the
 * library holds it until the process exits.  No cudaMalloc, cudaFree or other
 * allocating call is made.
 *   dtype, d_keys, n, stream  as hs_sort_keys (sorted in place)
 *   partition  10, 256 or 1 (0 = 10)
 * Limits and rules:
 *   - n <= 1,048,576 keys, else HS_ERR_INVALID (hs_last_error says why);
 *   - per-kernel timing (hs_timing_enable) must be off, else HS_ERR_INVALID;
 *   - the first call on a device sets up that device (looks up the device
 *     address of the scratch array with that device current); make that first
 *     call before any stream capture;
 *   - every call shares the one scratch array, which keeps the previous call's
 *     contents (the sort clears what it needs): calls whose work overlaps on
 *     the GPU (different streams, or different host threads) race and must be
 *     ordered by the caller.
 */
hs_status hs_sort_keys_noalloc(hs_dtype dtype, void* d_keys, size_t n, int partition, void* stream);

/* Work space needed by one call (bytes).  nseg = 1 and d_offsets unused for
 * the plain sorts; has_vals = 1 for pairs. */
hs_status hs_workspace_size(hs_dtype dtype, size_t n, int has_vals, size_t nseg,
                            const hs_opts* opts, size_t* bytes);

/* Grow the library's work space for `stream` on the current device to at
 * least `bytes` now (outside any timed or captured region). */
hs_status hs_workspace_reserve(size_t bytes, void* stream);

/* Free every work space the library holds on the current device
 * (synchronises the device). */
hs_status hs_workspace_release(void);

/* Synchronise `stream`, read and clear the device error word.  Returns HS_OK,
 * HS_ERR_TIMEOUT, HS_ERR_INVALID (bad batch offsets) or HS_ERR_DEVICE. */
hs_status hs_stream_error(void* stream);

/* Static description of the plan a call would run (no device work). */
typedef struct {
  int tile;            /* keys per tile of the per-packet sort (= outputs per merge block) */
  int part_tile;       /* keys per block of the packet step (3840) */
  int merge_passes;    /* merge passes enqueued (worst case for n; passes no packet needs exit at once) */
  int launches;        /* kernel launches enqueued by one call */
  int fan_in;          /* runs merged per merge pass */
} hs_plan;
hs_status hs_plan_describe(hs_dtype dtype, size_t n, int has_vals, size_t nseg, const hs_opts* opts,
                           hs_plan* out);

/* Per-kernel timing with CUDA events recorded on the launching stream around
 * every launch (off by default; costs one event pair per launch). */
typedef struct {
  char name[32];
  int launches;
  double total_ms;
} hs_kernel_time;
hs_status hs_timing_enable(int on);
/* Synchronises the device, returns up to `max` entries, clears the record. */
hs_status hs_timing_read(hs_kernel_time* out, int max, int* count);
/* The same record launch by launch, in launch order (launches = 1, total_ms =
 * that launch's time): up to `max` entries, *count = how many were written;
 * clears the record. */
hs_status hs_timing_read_launches(hs_kernel_time* out, int max, int* count);

/* Destroy every cached CUDA graph (see hs_opts.graph). */
hs_status hs_graph_cache_clear(void);

/* Tuning table (process-wide, thread-safe): the merge fan-in that calls with
 * opts->fan_in == 0 use, per (key type, has values, partition, size bucket);
 * bucket = ceil(log2(n)) (0..32).  Filled by a tuner that times the candidates
 * on this GPU (the Python package's tune module) or by the caller.
 * hs_tune_set: fan_in 2 or 4 (else HS_ERR_INVALID); partition 1, 10 or 256.
 * hs_tune_get: the fan-in a call with fan_in == 0 would use for n keys
 * (table entry, else the built-in rule).  hs_tune_clear: empties the table. */
hs_status hs_tune_set(hs_dtype dtype, int has_vals, int partition, int log2n, int fan_in);
hs_status hs_tune_get(hs_dtype dtype, int has_vals, int partition, size_t n, int* fan_in);
hs_status hs_tune_clear(void);

/* Tuning table, whole shape: the merge fan-in (2, 4, or 0 = the built-in rule),
 * the tile (a built tile of the key type, or 0 = the default tile) and the
 * merge launch style (1, 2, or 0 = the built-in rule; see hs_opts.merge) that
 * calls with opts->fan_in / tile / merge == 0 use for this (key type, has
 * values, partition, size bucket = ceil(log2(n))).  The shape changes only how
 * the work is cut (tile sort, merge blocks, passes), never the result, which is
 * the sorted order of Sec. 3.4 bit for bit.  Invalid values: HS_ERR_INVALID.
 * hs_tune_get_shape: the shape a call for n keys would use. */
hs_status hs_tune_set_shape(hs_dtype dtype, int has_vals, int partition, int log2n, int fan_in, int tile,
                            int merge);
hs_status hs_tune_get_shape(hs_dtype dtype, int has_vals, int partition, size_t n, int* fan_in, int* tile,
                            int* merge);

/* The tiles built for a key type (and values): writes up to `max` of them to
 * `tiles` (ascending) and their number to *count. */
hs_status hs_tiles(hs_dtype dtype, int has_vals, int* tiles, int max, int* count);

/* Cumulative number of kernel launches this library has enqueued in this
 * process (memsets and copies not counted; a graph replay counts the kernels
 * in the graph). */
unsigned long long hs_kernel_launches(void);

const char* hs_status_string(hs_status s);
/* Text of the last CUDA error seen by the library in this thread ("" if none). */
const char* hs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HSORT_H */
