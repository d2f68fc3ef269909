// Host side of one sort call: work-space layout and the launch sequence.
// Included by one translation unit per (key type, tile shape): sort_shape.cu
// compiled once per pair, so they compile in parallel.
#pragma once
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "hsort.h"
#include "common.cuh"
#include "partition.cuh"
#include "blockmerge.cuh"
#include "merge.cuh"
#include "merge4.cuh"
#include "tilesort.cuh"
#include "sched.cuh"
#include "runtime.h"

namespace hs {

// Fixed shapes of this build.
constexpr int kBlock = 256;     // threads per CTA of every heavy kernel
constexpr int kIpt = 15;        // items per thread of the packet step (odd: conflict-free blocked access)
constexpr int kTile = kBlock * kIpt;  // keys per packet-step block

// Tile shapes (items per thread of the tile sort and the merge passes; a
// tile is kBlock x IPT keys), all odd so blocked shared-memory access is free
// of bank conflicts.  Built: 15, 23 and 31 for 4-byte keys without values;
// 11 and 15 otherwise (where 31 items and their companions would not fit in
// registers).  Default (no tuning-table entry, hs_opts.tile = 0): 31 for
// 4-byte keys without values (twice the work per co-rank search and per
// block of 15, one merge pass fewer), 15 otherwise.
template <class K, bool HAS_V>
constexpr int sort_ipt() {
  return (sizeof(K) == 4 && !HAS_V) ? 31 : 15;
}
template <class K, bool HAS_V, int IPT>
constexpr bool ipt_built() {
  return (sizeof(K) == 4 && !HAS_V) ? (IPT == 15 || IPT == 23 || IPT == 31) : (IPT == 11 || IPT == 15);
}
constexpr int kTileIpts[] = {11, 15, 23, 31};
inline bool tile_built(size_t key_bytes, bool has_vals, int tile) {
  const bool wide = key_bytes == 4 && !has_vals;
  return wide ? (tile == kBlock * 15 || tile == kBlock * 23 || tile == kBlock * 31)
              : (tile == kBlock * 11 || tile == kBlock * 15);
}
inline int sort_tile_for(size_t key_bytes, bool has_vals) {
  return kBlock * ((key_bytes == 4 && !has_vals) ? 31 : 15);
}
// the smallest built tile: work-space tables are sized for it, so one work
// space serves every tile shape of its key type
inline int min_tile_for(size_t key_bytes, bool has_vals) {
  return kBlock * ((key_bytes == 4 && !has_vals) ? 15 : 11);
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

constexpr int kMaxPasses = 64;
constexpr int kMergeQueue = 1;    // hs_opts.merge: every two-way pass in one persistent launch
constexpr int kMergePerPass = 2;  // hs_opts.merge: a co-rank and a merge launch per pass
// Lanes per co-rank search: more lanes per search when a pass has few merge
// blocks (its co-rank kernel is then bound by the latency of the search
// chain), one thread per merge block when it has many.
inline int corank_group(size_t units) { return units <= 4096 ? 16 : (units <= 16384 ? 4 : 1); }
constexpr int kMerge4Spt = 2;  // fan-in-4 merge: chunk slots per tile (average chunk = tile / slots)  // pass-control words (n < 2^32 needs at most 32 passes)

// Worst-case merge passes for a packet of up to n keys, sorted in tiles of
// `tile`, merged `fan_in` runs at a time.
inline int worst_passes(size_t n, size_t tile, int fan_in = 2) {
  size_t tiles = (n + tile - 1) / tile;
  int p = 0;
  while ((static_cast<size_t>(1) << p) < tiles) ++p;
  return fan_in == 4 ? (p + 1) / 2 : p;
}

struct Layout {
  size_t keys_w, vals_w, seg_off, blk_prefix, cls_raw, cnt_raw, flat, scan_part, seg_neg, seg_cmax, seg_class,
      seg_flip, pkt_off, unit_prefix, recs, list, any_neg, pass_ctl, zero, zero_bytes, small_before, small_list,
      small_cnt, sched, sched_bytes, total;
  uint32_t max_blocks, max_units, npk;
};

inline Layout make_layout(size_t key_bytes, size_t n, bool has_vals, size_t nseg, int nb) {
  const size_t stile = min_tile_for(key_bytes, has_vals);
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  L.max_blocks = static_cast<uint32_t>((n + kTile - 1) / kTile + nseg);
  L.npk = static_cast<uint32_t>(nseg * nb);
  L.max_units = static_cast<uint32_t>((n + stile - 1) / stile + L.npk);
  L.keys_w = take(n * key_bytes + 16);
  L.vals_w = take(has_vals ? n * 4 + 16 : 0);
  L.seg_off = take((nseg + 1) * 8);
  L.blk_prefix = take((nseg + 1) * 4);
  L.cls_raw = take(static_cast<size_t>(L.max_blocks) * 4);
  L.cnt_raw = take(static_cast<size_t>(L.max_blocks) * nb * 4);
  L.flat = take(static_cast<size_t>(L.max_blocks) * nb * 4);
  L.scan_part = take(kScanChunks * 4);
  // seg_neg, seg_cmax, any_neg and pass_ctl are adjacent: one memset zeroes them
  L.zero = take(nseg * 4 + nseg * 2 * 4 + 4 + kMaxPasses * 4);
  L.seg_neg = L.zero;
  L.seg_cmax = L.zero + nseg * 4;
  L.any_neg = L.seg_cmax + nseg * 2 * 4;
  L.pass_ctl = L.any_neg + 4;
  L.zero_bytes = nseg * 4 + nseg * 2 * 4 + 4 + kMaxPasses * 4;
  L.seg_class = take(nseg * 4);
  L.seg_flip = take(nseg * 4);
  L.pkt_off = take((L.npk + 1) * 8);
  L.unit_prefix = take((L.npk + 1) * 4);
  const size_t slots = static_cast<size_t>(L.max_units) * kMerge4Spt + 1;  // fan-in-4 chunk slots
  L.recs = take(std::max((static_cast<size_t>(L.max_units) + 1) * sizeof(MergeRec), slots * sizeof(Rec4)));
  L.list = take(slots * 4);
  L.small_before = take((nseg + 1) * 4);
  L.small_list = take(nseg * 4);
  L.small_cnt = take(4);
  // merge scheduler: the ticket counter (256 bytes) and one completion
  // counter per (pass, unit) for passes 0 .. worst case
  L.sched_bytes = 256 + static_cast<size_t>(worst_passes(n, stile) + 1) * L.max_units * 4;
  L.sched = take(L.sched_bytes);
  L.total = off;
  return L;
}

inline Tables make_tables(char* base, const Layout& L, uint32_t* err, int fan_log2) {
  Tables t;
  t.fan_log2 = fan_log2;
  t.seg_off = reinterpret_cast<uint64_t*>(base + L.seg_off);
  t.blk_prefix = reinterpret_cast<uint32_t*>(base + L.blk_prefix);
  t.cls_raw = reinterpret_cast<uint32_t*>(base + L.cls_raw);
  t.cnt_raw = reinterpret_cast<uint32_t*>(base + L.cnt_raw);
  t.flat = reinterpret_cast<uint32_t*>(base + L.flat);
  t.scan_part = reinterpret_cast<uint32_t*>(base + L.scan_part);
  t.seg_neg = reinterpret_cast<uint32_t*>(base + L.seg_neg);
  t.seg_cmax = reinterpret_cast<uint32_t*>(base + L.seg_cmax);
  t.seg_class = reinterpret_cast<uint32_t*>(base + L.seg_class);
  t.seg_flip = reinterpret_cast<uint32_t*>(base + L.seg_flip);
  t.pkt_off = reinterpret_cast<uint64_t*>(base + L.pkt_off);
  t.unit_prefix = reinterpret_cast<uint32_t*>(base + L.unit_prefix);
  t.any_neg = reinterpret_cast<uint32_t*>(base + L.any_neg);
  t.pass_ctl = reinterpret_cast<uint32_t*>(base + L.pass_ctl);
  t.small_before = reinterpret_cast<uint32_t*>(base + L.small_before);
  t.small_list = reinterpret_cast<uint32_t*>(base + L.small_list);
  t.small_cnt = reinterpret_cast<uint32_t*>(base + L.small_cnt);
  t.err = err;
  return t;
}

inline int fan_log2_of(int fan_in) { return fan_in == 4 ? 2 : 1; }

template <class K, bool HAS_V, int NB>
inline size_t scatter_smem() {
  constexpr int NW = kBlock / kWarp;
  size_t b = 0;
  b += kTile * sizeof(K);
  b += HAS_V ? kTile * 4 : 0;
  b += NW * (NB + 1) * 4;
  b += ((NB + 2) & ~1) * 4;
  b += ((NB + 1) & ~1) * 4;
  b += ((NB + 1) & ~1) * 4;
  b += kTile * 2;
  return b;
}
template <class K>
inline size_t hist_smem() {  // two stages of keys
  return 2 * ((region_elems(kTile) * sizeof(K) + 127) & ~size_t(127));
}
template <class K, bool HAS_V, int IPT>
inline size_t sort_smem() {  // one region of keys (and values)
  return merge_stage_bytes<K, HAS_V>(kBlock * IPT);
}
// Fan-in-4 merge shape: threads per CTA and CTAs per SM.
constexpr int kMerge4Block = 256;
constexpr int kMerge4MinBlocks = 3;
template <class K, bool HAS_V, int IPT>
constexpr int merge4_cmax() {
  return chunk_max<kBlock * IPT, kMerge4Spt>();
}
template <class K, bool HAS_V, int IPT>
inline size_t merge4_smem_for() {  // two stages of the largest chunk and T
  return merge4_smem<K, HAS_V, merge4_cmax<K, HAS_V, IPT>()>();
}
template <class K, bool HAS_V, int IPT>
inline size_t merge_smem() {  // two input stages (+ two output buffers when they fit)
  constexpr int T = kBlock * IPT;
  return merge_buffers<K, HAS_V, T>() * merge_stage_bytes<K, HAS_V>(T);
}

// Launch shapes are cached per device: kernel attributes (shared-memory size,
// carveout) are set per device, and the occupancy query is per device.
constexpr int kMaxDevices = 64;
struct PerDevice {
  int v[kMaxDevices] = {};
  int& operator()() {
    int d = 0;
    cudaGetDevice(&d);
    static int spare;  // devices beyond the table: recomputed on every call
    if (d < 0 || d >= kMaxDevices) return spare = 0;
    return v[d];
  }
};

// A persistent grid never larger than the work a call can have (every
// persistent kernel loops over its work, so any grid size is correct; CTAs
// that would find nothing to do are not launched).
inline int capped(int grid, uint64_t need) {
  return static_cast<int>(std::max<uint64_t>(1, std::min<uint64_t>(static_cast<uint64_t>(grid), need)));
}

template <class Kern>
inline int persistent_grid(Kern kern, int block, size_t smem) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // (opt in whenever dynamic shared memory is used: static plus dynamic above
  // 48 KB needs it even when the dynamic part alone is below)
  if (smem > 0) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, smem);
  if (occ < 1) occ = 1;
  return sms * occ;
}

template <class K, int T, int G>
hs_status launch_corank(Launcher& lc, K* keys, K* kw, MergeRec* recs, uint32_t npk, int r, const Tables& tb,
                        uint64_t max_units) {
  static PerDevice grid_cache;
  int& grid = grid_cache();
  auto ck = k_corank<K, T, G>;
  if (!grid) grid = persistent_grid(ck, 256, 0);
  const uint64_t lanes = max_units * (G == 1 ? 1 : 2 * G);  // lanes per merge block
  return lc.kernel("corank", ck, capped(grid, (lanes + 255) / 256), 256, 0, keys, kw, recs, npk, r, tb);
}

// Fan-in-4 sample ranking: one warp per sample (eight lanes per run) up to
// this many tiles, one thread per sample above.
constexpr size_t kBound4WarpTiles = 1024;
template <class K, int T, int LG>
hs_status launch_bound4(Launcher& lc, K* keys, K* kw, Rec4* recs, uint32_t* list, uint32_t npk, int r,
                        const Tables& tb, uint64_t max_units) {
  static PerDevice grid_cache;
  int& grid = grid_cache();
  auto ck = k_bound4<K, T, kMerge4Spt, LG>;
  if (!grid) grid = persistent_grid(ck, 256, 0);
  const uint64_t lanes = max_units * kMerge4Spt * kSamplesPerChunk * (LG == 1 ? 1 : 32);  // per sample slot
  return lc.kernel("bound4", ck, capped(grid, (lanes + 255) / 256), 256, 0, keys, kw, recs, list, npk, r, tb);
}

// One sort call.  keys/vals: the caller's arrays (U).  offs: batch offsets
// (device) or nullptr for one segment.  ws: work space of at least
// make_layout(...).total bytes.  src: nullptr, or the keys in pinned host
// memory the device can address (one segment, no values): the histogram
// reads them from there and writes them into `keys` in the same pass (a
// call without a histogram copies them in first).
// host_done (may be nullptr): set to 1 when the sorted keys were also
// written back to `src` by the kernels (the merge queue writes every packet's
// last pass there, and the packets with no merge pass are copied there);
// otherwise 0 and the caller copies `keys` back.
template <class K, bool HAS_V, int NB, int IPT>
hs_status run_sort_nb(K* keys, uint32_t* vals, size_t n, size_t nseg, const uint64_t* offs, const hs_opts& o,
                      char* ws, uint32_t* err, cudaStream_t st, const K* src, int* host_done) {
  if (host_done) *host_done = 0;
  const Layout L = make_layout(sizeof(K), n, HAS_V, nseg, NB);
  const int fan = o.fan_in == 4 ? 4 : 2;
  Tables tb = make_tables(ws, L, err, fan_log2_of(fan));
  K* kw = reinterpret_cast<K*>(ws + L.keys_w);
  uint32_t* vw = HAS_V ? reinterpret_cast<uint32_t*>(ws + L.vals_w) : nullptr;
  const uint32_t nseg32 = static_cast<uint32_t>(nseg);
  Launcher lc(st);

  // zero the per-segment flags and maxima and the pass control (one region)
  HS_TRY(lc.memset("zero_tables", ws + L.zero, 0, L.zero_bytes));
  // the merge scheduler's ticket and completion counters
  const bool use_sched = fan == 2 && o.merge != kMergePerPass && o.stop_after != 1 && o.stop_after != 2 &&
                         worst_passes(n, (kBlock * IPT)) > 0;
  if (use_sched) HS_TRY(lc.memset("zero_sched", ws + L.sched, 0, L.sched_bytes));
  const bool small = static_cast<uint64_t>(L.max_blocks) * NB <= kPlanSmallEntries &&
                     static_cast<uint64_t>(L.npk) <= kPlanSmallEntries;

  // Short segments (at most one tile) are sorted whole by one CTA of the tile
  // sort launch; not when a testing stop point asks for the packet layout or
  // the tile sort's state.
  const uint32_t small_max = o.stop_after == 0 ? static_cast<uint32_t>((kBlock * IPT)) : 0u;
  // one segment known on the host to be short: no packet-step kernels at all
  const bool all_short = nseg == 1 && n <= small_max;
  HS_TRY(lc.kernel("seg_plan", k_seg_plan, 1, 1024, 0, offs, nseg32, n, kTile, small_max, tb));
  // keys in host memory and no histogram to read them: copy them in
  const bool hist_reads_src = src != nullptr && NB != 1 && !all_short;
  if (src && !hist_reads_src) HS_TRY(lc.copy("copy_in", keys, src, n * sizeof(K), cudaMemcpyHostToDevice));

  if constexpr (NB == 1) {
    // no MSD step (ablation): every segment is one packet; the tile sort
    // reads the caller's array directly
    if (small) {
      HS_TRY(lc.kernel("plan_small", (k_plan_small<1>), 1, kPlanThreads, 0, nseg32, (kBlock * IPT), tb));
    } else {
      HS_TRY(lc.kernel("pkt", k_pkt_whole, (nseg32 + 255) / 256, 256, 0, nseg32, (kBlock * IPT), tb));
      HS_TRY(lc.kernel("scan_units", k_scan_units, 1, 1024, 0, L.npk, tb));
    }
  } else {
    if (!all_short) {
      static PerDevice grid_cache, sgrid_cache;
      int& grid = grid_cache();
      int& sgrid = sgrid_cache();
      const size_t smem = hist_smem<K>();
      auto kern = k_hist<K, NB, kBlock, kIpt>;
      auto skern = k_hist<K, NB, kBlock, kIpt, true>;  // reads the keys from host memory
      if (!grid) grid = persistent_grid(kern, kBlock, smem);
      if (hist_reads_src && !sgrid) sgrid = persistent_grid(skern, kBlock, 0);
      for (int img = 0; img < (std::is_same<K, int32_t>::value ? 2 : 1); ++img) {
        if (img == 0 && hist_reads_src)
          HS_TRY(lc.kernel("hist_copy_in", skern, capped(sgrid, L.max_blocks), kBlock, 0, keys, src, nseg32, kTile,
                           img, tb));
        else
          HS_TRY(lc.kernel(img ? "hist_flip" : "hist", kern, capped(grid, L.max_blocks), kBlock, smem, keys,
                           static_cast<const K*>(nullptr), nseg32, kTile, img, tb));
      }
    }
    if (small) {
      HS_TRY(lc.kernel("plan_small", (k_plan_small<NB>), 1, kPlanThreads, 0, nseg32, (kBlock * IPT), tb));
    } else {
    HS_TRY(lc.kernel("finalize", (k_finalize<NB>), (nseg32 + 255) / 256, 256, 0, nseg32, tb));
    {
      static PerDevice grid_cache;
      int& grid = grid_cache();
      if (!grid) grid = persistent_grid(k_fold<NB>, 256, 0);
      HS_TRY(lc.kernel("fold", (k_fold<NB>), grid, 256, 0, nseg32, tb));
    }
    // exclusive scan of the (segment, packet, block) counts: absolute positions
    const uint32_t* m_ptr = tb.blk_prefix + nseg;  // total blocks (device)
    HS_TRY(lc.kernel("scan_reduce", k_scan_reduce, kScanChunks, kScanBlock, 0, tb.flat, m_ptr, NB,
                     tb.scan_part));
    HS_TRY(lc.kernel("scan_partials", k_scan_partials, 1, kScanBlock, 0, tb.scan_part));
    HS_TRY(lc.kernel("scan_down", k_scan_down, kScanChunks, kScanBlock, 0, tb.flat, m_ptr, NB, tb.scan_part));
    {
      static PerDevice grid_cache;
      int& grid = grid_cache();
      if (!grid) grid = persistent_grid(k_pkt<NB>, 256, 0);
      HS_TRY(lc.kernel("pkt", (k_pkt<NB>), grid, 256, 0, nseg32, (kBlock * IPT), tb));
    }
    HS_TRY(lc.kernel("scan_units", k_scan_units, 1, 1024, 0, L.npk, tb));
    }

    if (all_short) {
      // nothing to scatter: the one segment is sorted whole by the tile sort launch
    } else if constexpr (NB <= 16) {
      // persistent: bulk copies in and out, ranks from one scan of packed counts
      static PerDevice grid_cache;
      int& grid = grid_cache();
      const size_t smem = ScatterSmallLayout<K, HAS_V, kBlock, kIpt>::bytes;
      auto kern = k_scatter_small<K, HAS_V, NB, kBlock, kIpt>;
      if (!grid) {
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        grid = persistent_grid(kern, kBlock, smem);
      }
      const bool stuck = (o.debug_flags & 4) != 0;
      const uint64_t limit_ns = stuck ? 2000000ull : 2000000000ull;  // 2 ms when injected, else 2 s
      HS_TRY(lc.kernel("scatter", kern, capped(grid, L.max_blocks), kBlock, smem, keys, vals, kw, vw, nseg32, kTile,
                       stuck ? 1 : 0, limit_ns, tb));
    } else {
      const size_t smem = scatter_smem<K, HAS_V, NB>();
      auto kern = k_scatter<K, HAS_V, NB, kBlock, kIpt>;
      static PerDevice attr_cache;
      int& attr = attr_cache();
      if (!attr) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        attr = 1;
      }
      HS_TRY(lc.kernel("scatter", kern, L.max_blocks, kBlock, smem, keys, vals, kw, vw, nseg32, kTile, tb));
    }
  }
  if (o.stop_after == 1) {
    if (NB != 1) {  // with one packet the packet layout is the input itself
      HS_TRY(lc.copy("copy_back", keys, kw, n * sizeof(K)));
      if (HAS_V) HS_TRY(lc.copy("copy_back_v", vals, vw, n * 4));
    }
  } else {
    {
      static PerDevice grid_cache;
      int& grid = grid_cache();
      const size_t smem = sort_smem<K, HAS_V, IPT>();
      auto kern = k_tilesort<K, HAS_V, NB, kBlock, IPT>;
      if (!grid) grid = persistent_grid(kern, kBlock, smem);
      const bool stuck = (o.debug_flags & 1) != 0;
      const uint64_t limit_ns = stuck ? 2000000ull : 2000000000ull;  // 2 ms when injected, else 2 s
      const K* ts_k = (NB == 1) ? keys : kw;
      const uint32_t* ts_v = (NB == 1) ? vals : vw;
      // work items: the tiles of the packets, then the short segments
      const uint64_t items = static_cast<uint64_t>(L.max_units) + (small_max ? nseg : 0);
      HS_TRY(lc.kernel("tilesort", kern, capped(grid, items), kBlock, smem, ts_k, ts_v, keys, vals, kw, vw, L.npk,
                       o.stop_after == 2 ? 1 : 0, stuck ? 1 : 0, limit_ns, tb));
    }
    if (o.stop_after == 2) {
      HS_TRY(lc.copy("copy_back", keys, kw, n * sizeof(K)));
      if (HAS_V) HS_TRY(lc.copy("copy_back_v", vals, vw, n * 4));
    } else if (fan == 4) {
      constexpr int T = (kBlock * IPT);
      static PerDevice mgrid_cache;
      int& mgrid = mgrid_cache();
      const size_t smem = merge4_smem_for<K, HAS_V, IPT>();
      auto mk = k_merge4<K, HAS_V, kMerge4Block, kMerge4MinBlocks, merge4_cmax<K, HAS_V, IPT>()>;
      if (!mgrid) mgrid = persistent_grid(mk, kMerge4Block, smem);
      Rec4* recs = reinterpret_cast<Rec4*>(ws + L.recs);
      uint32_t* list = reinterpret_cast<uint32_t*>(ws + L.list);
      const int P = o.stop_after >= 3 ? std::min(worst_passes(n, T, 4), o.stop_after - 2) : worst_passes(n, T, 4);
      const bool warp_per_sample = (n + T - 1) / T <= kBound4WarpTiles;
      for (int r = 1; r <= P; ++r) {
        if (warp_per_sample) HS_TRY((launch_bound4<K, T, 8>(lc, keys, kw, recs, list, L.npk, r, tb, L.max_units)));
        else HS_TRY((launch_bound4<K, T, 1>(lc, keys, kw, recs, list, L.npk, r, tb, L.max_units)));
        HS_TRY(lc.kernel("merge4", mk, capped(mgrid, static_cast<uint64_t>(L.max_units) * kMerge4Spt), kMerge4Block,
                         smem, keys, vals, kw, vw, recs, list, r, tb));
      }
    } else if (o.merge != kMergePerPass) {
      // every merge pass in one persistent launch (dependency-driven queue)
      static PerDevice sgrid_cache, hgrid_cache;
      int& sgrid = sgrid_cache();
      int& hgrid = hgrid_cache();
      const size_t smem = 2 * merge_stage_bytes<K, HAS_V>(kBlock * IPT);  // two stages
      auto sk = k_merge_sched<K, HAS_V, kBlock, IPT>;
      auto hk = k_merge_sched<K, HAS_V, kBlock, IPT, !HAS_V>;  // last passes to host memory (keys only)
      if (!sgrid) sgrid = persistent_grid(sk, kBlock + 32, smem);
      const bool drop = (o.debug_flags & 2) != 0;
      SchedArgs sa;
      sa.ticket = reinterpret_cast<uint32_t*>(ws + L.sched);
      sa.done = reinterpret_cast<uint32_t*>(ws + L.sched + 256);
      sa.pass_limit = o.stop_after >= 3 ? o.stop_after - 2 : kMaxPasses;
      sa.debug_drop = drop ? 1 : 0;
      sa.limit_ns = drop ? 2000000ull : 2000000000ull;  // 2 ms when a completion is dropped, else 2 s
      // keys from host memory: every packet's last pass writes straight back
      // to the caller's host array (no copy out after the sort)
      const bool to_host = !HAS_V && src != nullptr && nseg == 1 && o.stop_after == 0;
      sa.host_out = to_host ? const_cast<K*>(src) : nullptr;
      if (worst_passes(n, (kBlock * IPT)) > 0) {
        if (to_host) {
          if (!hgrid) hgrid = persistent_grid(hk, kBlock + 32, smem);
          HS_TRY(lc.kernel("merge_sched", hk, capped(hgrid, L.max_units), kBlock + 32, smem, keys, vals, kw, vw,
                           L.npk, tb, sa));
        } else {
          HS_TRY(lc.kernel("merge_sched", sk, capped(sgrid, L.max_units), kBlock + 32, smem, keys, vals, kw, vw,
                           L.npk, tb, sa));
        }
        if (to_host) {
          HS_TRY(lc.kernel("copy_unmerged", k_copy_unmerged<K>, L.npk, 256, 0, static_cast<const K*>(keys),
                           const_cast<K*>(src), L.npk, tb));
          if (host_done) *host_done = 1;
        }
      }
    } else {
      // per-pass launches: a co-rank kernel, then a merge kernel
      static PerDevice mgrid_cache;
      int& mgrid = mgrid_cache();
      const size_t smem = merge_smem<K, HAS_V, IPT>();
      auto mk = k_merge<K, HAS_V, kBlock, IPT>;
      constexpr int T = (kBlock * IPT);
      if (!mgrid) mgrid = persistent_grid(mk, kBlock, smem);
      MergeRec* recs = reinterpret_cast<MergeRec*>(ws + L.recs);
      const int P = o.stop_after >= 3 ? std::min(worst_passes(n, T), o.stop_after - 2) : worst_passes(n, T);
      const int G = corank_group((n + T - 1) / T);
      for (int r = 1; r <= P; ++r) {
        if (G == 16) HS_TRY((launch_corank<K, T, 16>(lc, keys, kw, recs, L.npk, r, tb, L.max_units)));
        else if (G == 4) HS_TRY((launch_corank<K, T, 4>(lc, keys, kw, recs, L.npk, r, tb, L.max_units)));
        else HS_TRY((launch_corank<K, T, 1>(lc, keys, kw, recs, L.npk, r, tb, L.max_units)));
        HS_TRY(lc.kernel("merge", mk, capped(mgrid, L.max_units), kBlock, smem, keys, vals, kw, vw, recs, r, tb));
      }
    }
    if (o.stop_after >= 3) {  // testing: the state after merge pass r, gathered into the caller's array
      auto kcb = k_copy_back_pass<K, HAS_V, (kBlock * IPT)>;
      HS_TRY(lc.kernel("copy_back_pass", kcb, 2 * 152, 256, 0, keys, vals, kw, vw, L.npk, o.stop_after - 2,
                       tb));
    }
  }
  if (o.d_packet_offsets_out)
    HS_TRY(lc.copy("copy_offsets", o.d_packet_offsets_out, tb.pkt_off, (static_cast<size_t>(L.npk) + 1) * 8));
  return HS_OK;
}

// One sort call with the tile shape IPT (hs_opts.tile resolved by the
// caller): values or not, then the partition variant.  Instantiated in one
// translation unit per (key type, IPT) (sort_shape.cu).
template <class K, bool HAS_V, int IPT>
hs_status run_sort_part(K* k, uint32_t* vals, size_t n, size_t nseg, const uint64_t* offs, const hs_opts& o,
                        char* ws, uint32_t* err, cudaStream_t st, const K* src, int* host_done) {
  if (o.partition == 1) return run_sort_nb<K, HAS_V, 1, IPT>(k, vals, n, nseg, offs, o, ws, err, st, src, host_done);
  if (o.partition == 256)
    return run_sort_nb<K, HAS_V, 256, IPT>(k, vals, n, nseg, offs, o, ws, err, st, src, host_done);
  return run_sort_nb<K, HAS_V, 10, IPT>(k, vals, n, nseg, offs, o, ws, err, st, src, host_done);
}

template <class K, int IPT>
hs_status run_sort_ipt(void* keys, uint32_t* vals, size_t n, size_t nseg, const uint64_t* offs, const hs_opts& o,
                       char* ws, uint32_t* err, cudaStream_t st, const void* src, int* host_done) {
  K* k = static_cast<K*>(keys);
  const K* ks = static_cast<const K*>(src);
  if (host_done) *host_done = 0;
  if (src && (vals || nseg != 1)) return HS_ERR_INVALID;  // host keys: one array, keys only
  if (vals) {
    if constexpr (ipt_built<K, true, IPT>())
      return run_sort_part<K, true, IPT>(k, vals, n, nseg, offs, o, ws, err, st, nullptr, nullptr);
    else return HS_ERR_UNSUPPORTED;
  } else {
    if constexpr (ipt_built<K, false, IPT>())
      return run_sort_part<K, false, IPT>(k, vals, n, nseg, offs, o, ws, err, st, ks, host_done);
    else return HS_ERR_UNSUPPORTED;
  }
}

}  // namespace hs
