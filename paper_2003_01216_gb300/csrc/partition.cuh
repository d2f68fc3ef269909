// Packet step (Sec. 2.1, Sec. 3.4): one MSD-radix pass that moves every key
// into one of ten packets (or 256 buckets for the ablation) by the leading
// digit of its image, keeping input order inside each packet.
//
// Kernels, in launch order:
//   k_seg_plan    segment table and packet-step block prefix (one CTA)
//   k_hist        one read of the keys: per block its class and its packet
//                 counts under that class; per segment the largest class
//   k_finalize    per segment: the final class and image
//   k_fold        per block: its counts under the segment's class, laid out
//                 in (segment, packet, block) order
//   k_scan_*      exclusive scan of that array: because the sorted output
//                 holds segment after segment and, inside one, packet after
//                 packet in block order, the prefix IS every block's absolute
//                 first position in every packet
//   k_pkt         packet offsets and tiles per packet
//   k_scan_units  exclusive scan of the tiles per packet (one CTA)
//   (small calls run k_finalize .. k_scan_units as one CTA: k_plan_small)
//   k_scatter_small / k_scatter
//                 stable scatter into packets (one read + one write of the
//                 keys and values; no block waits on another): persistent with
//                 bulk copies for up to 16 packets, one CTA per block for 256
//
// The class trick: the packet of a key depends on the class (digit count D,
// or bit length B) of the LARGEST key image of its array, which no block
// knows before the whole array has been read.  k_hist therefore counts every
// block under its own block-local class c_b.  A block whose class is below
// the array's class C holds only keys smaller than every threshold of C
// (decimal: all its keys fall in packet 0; binary: its local bucket t becomes
// t >> (shift(C) - shift(c_b))), so k_fold turns every block's counts into
// counts under C exactly, without a second read of the keys.
#pragma once
#include "async.cuh"
#include "common.cuh"
#include "scan.cuh"
#include "blockmerge.cuh"

namespace hs {

// ---------------------------------------------------------------------------
// k_seg_plan: segment table.  Plain sorts pass offs == nullptr (one segment
// [0, n)).  Batches pass the caller's offsets, which are validated here; if
// they are malformed every segment is treated as empty (no key moves) and the
// error word gets kErrBadOffsets.
//
// Short segments (1 .. small_max keys; small_max = 0 turns this off) skip the
// packet step, the tile sort of packets and the merges: one CTA of the tile
// sort launch sorts each of them whole and writes its packet offsets (see
// k_tilesort).  They get no packet-step blocks, so the (segment, packet,
// block) scan counts only the other segments' keys; small_before[s] (keys of
// short segments before s) turns its positions back into absolute ones, and
// small_list holds the short segments in order (small_cnt of them).
// ---------------------------------------------------------------------------
// Block-wide exclusive scan of three counters at once (all threads call it);
// returns the exclusive prefixes and writes the block totals to tot.
__device__ __forceinline__ void block_scan3(uint32_t (&v)[3], uint32_t (&excl)[3], uint32_t (&tot)[3],
                                            uint32_t (*s_warp)[32]) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  uint32_t inc[3] = {v[0], v[1], v[2]};
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, inc[q], o);
      if (lane >= o) inc[q] += x;
    }
  }
  if (lane == 31) {
#pragma unroll
    for (int q = 0; q < 3; ++q) s_warp[q][wid] = inc[q];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      uint32_t w = (lane < nw) ? s_warp[q][lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += x;
      }
      s_warp[q][lane] = w;  // inclusive over warps
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    excl[q] = inc[q] - v[q] + (wid ? s_warp[q][wid - 1] : 0u);
    tot[q] = s_warp[q][31];
  }
  __syncthreads();  // s_warp is reused by the next call
}

static __global__ void k_seg_plan(const uint64_t* __restrict__ offs, uint32_t nseg, uint64_t n, uint32_t part_tile,
                                  uint32_t small_max, Tables tb) {
  griddep_open();
  __shared__ uint32_t s_bad;
  __shared__ uint32_t s_warp[3][32];
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  if (offs) {
    for (uint32_t s = tid; s < nseg; s += nt)
      if (offs[s + 1] < offs[s]) s_bad = 1;
    if (tid == 0 && (offs[0] != 0 || offs[nseg] != n)) s_bad = 1;
  }
  __syncthreads();
  const bool bad = s_bad != 0;
  if (bad && tid == 0) atomicOr(tb.err, kErrBadOffsets);
  uint32_t carry[3] = {0, 0, 0};  // blocks, short-segment keys, short segments
  for (uint32_t base = 0; base <= nseg; base += nt) {
    const uint32_t s = base + tid;
    if (s <= nseg) {
      const uint64_t so = offs ? offs[s] : (s == 0 ? 0 : n);
      tb.seg_off[s] = bad ? 0 : so;
    }
    uint32_t v[3] = {0, 0, 0};
    if (s < nseg && !bad) {
      const uint64_t lo = offs ? offs[s] : 0;
      const uint64_t hi = offs ? offs[s + 1] : n;
      const uint64_t len = hi - lo;
      if (len > 0 && len <= small_max) {
        v[1] = static_cast<uint32_t>(len);
        v[2] = 1;
      } else {
        v[0] = static_cast<uint32_t>((len + part_tile - 1) / part_tile);
      }
    }
    uint32_t ex[3], tot[3];
    block_scan3(v, ex, tot, s_warp);
    if (s <= nseg) {
      tb.blk_prefix[s] = carry[0] + ex[0];
      tb.small_before[s] = carry[1] + ex[1];
    }
    if (v[2]) tb.small_list[carry[2] + ex[2]] = s;
#pragma unroll
    for (int q = 0; q < 3; ++q) carry[q] += tot[q];
  }
  if (tid == 0) *tb.small_cnt = carry[2];
}

// A segment that skips the packet step: keys, but no packet-step blocks.
__device__ __forceinline__ bool seg_is_small(const Tables& tb, uint32_t s) {
  return tb.seg_off[s + 1] > tb.seg_off[s] && tb.blk_prefix[s + 1] == tb.blk_prefix[s];
}

// Locate the segment of packet-step block b (blk_prefix is non-decreasing).
__device__ __forceinline__ uint32_t find_seg(const uint32_t* __restrict__ pre, uint32_t nseg, uint32_t b) {
  uint32_t lo = 0, hi = nseg;  // answer in [0, nseg): last s with pre[s] <= b
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (pre[mid] <= b) lo = mid; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// k_hist: each CTA walks a contiguous range of packet-step blocks.  For every
// block it reduces the largest key image, takes the block's class c_b and
// counts its keys per packet under c_b; it writes c_b and the NB counts of
// the block, and keeps the largest class of the current segment, flushed
// (atomicMax) when the segment changes and at the end.
//   img = 0: identity image (and every segment's "has a negative key" flag);
//            the keys of block b+1 arrive by bulk copy into the other of two
//            shared-memory stages while block b is counted.  FROM_SRC (keys
//            in pinned host memory that the device can address, at `src`):
//            each block is read from src by plain loads and written to
//            `keys` on the way: the copy into the device and the count are
//            one pass.
//   img = 1: sign-flipped image, only for blocks of segments flagged by the
//            img = 0 pass (plain loads; the kernel returns at once when no
//            segment holds a negative key)
// ---------------------------------------------------------------------------
// Decimal digit count of a 32-bit image (1..10), by comparisons with
// immediate powers of ten.
__device__ __forceinline__ int dec_class32(uint32_t v) {
  return 1 + (v >= 10u) + (v >= 100u) + (v >= 1000u) + (v >= 10000u) + (v >= 100000u) + (v >= 1000000u) +
         (v >= 10000000u) + (v >= 100000000u) + (v >= 1000000000u);
}

// The keys of one block: images into u[] (and the block maximum into m);
// FULL: every item of the block exists (no bounds tests).
template <class K, int BLOCK, int IPT, bool FULL>
__device__ __forceinline__ void hist_load(const K* keysrc, uint32_t cnt, bool flip, K* copy_to,
                                          typename KT<K>::U (&u)[IPT], typename KT<K>::U& m) {
  using U = typename KT<K>::U;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const uint32_t i = wid * kWarp * IPT + j * kWarp + lane;
    u[j] = U(0);
    if (FULL || i < cnt) {
      const K x = keysrc[i];
      if (copy_to) copy_to[i] = x;  // keys read from host memory also go to the device array
      u[j] = KT<K>::image(x, flip);
    }
    m = max(m, u[j]);
  }
}

// Ten packets: packed per-thread counters, 4 bits per packet (a thread holds
// at most IPT <= 15 keys), packets 0..7 in `lo`, 8..9 in `hi`.
template <class U, int IPT, bool FULL>
__device__ __forceinline__ void hist_count10(const U (&u)[IPT], uint32_t cnt, const DigitRule& rule, uint32_t& lo,
                                             uint32_t& hi) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const uint32_t i = wid * kWarp * IPT + j * kWarp + lane;
    const uint32_t p = packet_of<10>(u[j], rule);
    const uint32_t inc = (FULL || i < cnt) ? (1u << (4 * (p & 7))) : 0u;
    if (p < 8) lo += inc; else hi += inc;
  }
}

template <class K, int NB, int BLOCK, int IPT>
__device__ __forceinline__ void hist_count_block(const K* keysrc, uint32_t cnt, bool flip, int img,
                                                 uint32_t* s_cnt, typename KT<K>::U* s_max, uint32_t& s_neg,
                                                 int& cls_out, K* copy_to = nullptr) {
  using U = typename KT<K>::U;
  constexpr int NW = BLOCK / kWarp;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int q = tid; q < NB; q += BLOCK) s_cnt[q] = 0;
  U u[IPT];
  U m = 0;
  const bool full = cnt == static_cast<uint32_t>(BLOCK * IPT);
  if (full) hist_load<K, BLOCK, IPT, true>(keysrc, cnt, flip, copy_to, u, m);
  else hist_load<K, BLOCK, IPT, false>(keysrc, cnt, flip, copy_to, u, m);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, static_cast<U>(__shfl_xor_sync(0xffffffffu, m, o)));
  if (lane == 0) s_max[wid] = m;
  __syncthreads();
  m = s_max[0];
#pragma unroll
  for (int w = 1; w < NW; ++w) m = max(m, s_max[w]);
  // int32 under the identity image: a negative key is an image with the top bit set
  if (std::is_same<K, int32_t>::value && img == 0 && tid == 0 && (static_cast<uint64_t>(m) >> 31)) s_neg = 1;
  int cls;
  if constexpr (NB == 10) cls = (sizeof(U) == 4) ? dec_class32(static_cast<uint32_t>(m)) : dec_class(m);
  else cls = bin_class(m);
  const DigitRule rule = (NB == 10) ? rule_dec(cls) : make_rule_bin(cls);
  if constexpr (NB == 10) {
    static_assert(IPT <= 15, "4-bit counters");
    uint32_t lo = 0, hi = 0;
    if (full) hist_count10<U, IPT, true>(u, cnt, rule, lo, hi);
    else hist_count10<U, IPT, false>(u, cnt, rule, lo, hi);
    // warp sums, two packets per reduction (16-bit fields: a warp counts at
    // most 32 x 15 keys), then lane q adds packet q's sum to the block count
    uint32_t mine = 0;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const uint32_t w0 = ((k < 4 ? lo : hi) >> (8 * (k & 3))) & 15u;
      const uint32_t w1 = ((k < 4 ? lo : hi) >> (8 * (k & 3) + 4)) & 15u;
      const uint32_t r = __reduce_add_sync(0xffffffffu, w0 | (w1 << 16));
      if ((lane >> 1) == k) mine = (r >> (16 * (lane & 1))) & 0xffffu;
    }
    if (lane < 10 && mine) atomicAdd(&s_cnt[lane], mine);
  } else {
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const uint32_t i = wid * kWarp * IPT + j * kWarp + lane;
      const uint32_t q = (full || i < cnt) ? packet_of<NB>(u[j], rule) : NB;
      const uint32_t peers = __match_any_sync(0xffffffffu, q);
      if (q < NB && lane == __ffs(peers) - 1) atomicAdd(&s_cnt[q], __popc(peers));
    }
  }
  cls_out = cls;
  __syncthreads();
}

template <class K, int NB, int BLOCK, int IPT, bool FROM_SRC = false>
__global__ void __launch_bounds__(BLOCK) k_hist(K* keys, const K* __restrict__ src, uint32_t nseg, uint32_t part_tile,
                                                 int img, Tables tb) {
  griddep_open();
  using U = typename KT<K>::U;
  constexpr int NW = BLOCK / kWarp;
  constexpr int TILE = BLOCK * IPT;
  extern __shared__ __align__(128) unsigned char s_raw[];  // img 0: two stages of (TILE + 8) keys
  __shared__ uint32_t s_cnt[NB];
  __shared__ U s_max[NW];
  __shared__ uint32_t s_neg, s_cmax;
  __shared__ __align__(8) uint64_t s_bar[2];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  if (img == 1 && *tb.any_neg == 0) return;
  const uint32_t total = tb.blk_prefix[nseg];
  const uint32_t per = (total + gridDim.x - 1) / gridDim.x;
  const uint32_t b0 = min(total, blockIdx.x * per), b1 = min(total, b0 + per);
  if (b0 >= b1) return;
  if (tid == 0) {
    s_neg = 0;
    s_cmax = 0;
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
  }
  mbar_fence_init();
  __syncthreads();

  uint32_t seg = find_seg(tb.blk_prefix, nseg, b0);
  auto flush = [&](uint32_t sg) {
    __syncthreads();
    if (tid == 0) {
      if (s_neg) {
        atomicOr(&tb.seg_neg[sg], 1u);
        atomicOr(tb.any_neg, 1u);
      }
      if (s_cmax) atomicMax(&tb.seg_cmax[sg * 2 + img], s_cmax);
      s_neg = 0;
      s_cmax = 0;
    }
    __syncthreads();
  };
  // where block bb's keys live (segment found by advancing from `sg`)
  auto block_span = [&](uint32_t bb, uint32_t sg, uint64_t& beg, uint32_t& cnt) {
    while (bb >= tb.blk_prefix[sg + 1]) ++sg;
    beg = tb.seg_off[sg] + static_cast<uint64_t>(bb - tb.blk_prefix[sg]) * part_tile;
    cnt = static_cast<uint32_t>(min64(part_tile, tb.seg_off[sg + 1] - beg));
  };
  constexpr size_t STAGE = ((region_elems(TILE) * sizeof(K) + 127) & ~size_t(127));
  auto issue = [&](uint32_t bb, int st) {  // the last warp (warp 0 leads the block reductions)
    uint64_t beg;
    uint32_t cnt;
    block_span(bb, seg, beg, cnt);
    if (lane == 0) fence_proxy_async();  // generic reads of this stage happened before the last barrier
    __syncwarp();
    K* region = reinterpret_cast<K*>(s_raw + st * STAGE);
    const PendingBulk<K> pk = load_window_singles(region, phase_of(keys + beg), keys + beg, cnt, lane);
    cp_async_mbar_arrive(&s_bar[st]);
    __syncwarp();
    if (lane == 0) {
      mbar_arrive_expect_tx(&s_bar[st], pk.bytes);
      if (pk.bytes) bulk_g2s(pk.sdst, pk.gsrc, pk.bytes, &s_bar[st]);
    }
  };

  // keys in host memory (src): plain loads, no bulk copies
  const bool from_src = FROM_SRC && img == 0;
  if (img == 0 && !from_src && wid == NW - 1) issue(b0, 0);
  uint32_t par0 = 0, par1 = 0;
  int st = 0;
  for (uint32_t b = b0; b < b1; ++b) {
    while (b >= tb.blk_prefix[seg + 1]) {
      flush(seg);
      ++seg;
    }
    const uint64_t beg = tb.seg_off[seg] + static_cast<uint64_t>(b - tb.blk_prefix[seg]) * part_tile;
    const uint32_t cnt = static_cast<uint32_t>(min64(part_tile, tb.seg_off[seg + 1] - beg));
    int cls = 0;
    if constexpr (FROM_SRC) {
      if (img == 0) {
        hist_count_block<K, NB, BLOCK, IPT>(src + beg, cnt, false, 0, s_cnt, s_max, s_neg, cls, keys + beg);
      } else {
        if (!tb.seg_neg[seg]) continue;  // block-uniform
        hist_count_block<K, NB, BLOCK, IPT>(keys + beg, cnt, true, 1, s_cnt, s_max, s_neg, cls);
      }
    } else if (img == 0) {
      if (wid == NW - 1 && b + 1 < b1) issue(b + 1, st ^ 1);
      const uint32_t ph = st ? par1 : par0;
      const bool ok = mbar_wait_bounded(&s_bar[st], ph, tb.err, 2000000000ull);
      if (st) par1 ^= 1; else par0 ^= 1;
      if (__syncthreads_or(!ok)) {
        // copies may still be landing in this stage, and in the other one
        // when the next block's copy was issued: bounded waits, then leave
        mbar_wait_bounded(&s_bar[st], ph, tb.err, 2000000000ull);
        if (b + 1 < b1) mbar_wait_bounded(&s_bar[st ^ 1], st ? par0 : par1, tb.err, 2000000000ull);
        return;
      }
      const K* region = reinterpret_cast<const K*>(s_raw + st * STAGE) + phase_of(keys + beg);
      hist_count_block<K, NB, BLOCK, IPT>(region, cnt, false, 0, s_cnt, s_max, s_neg, cls);
      st ^= 1;
    } else {
      if (!tb.seg_neg[seg]) continue;  // block-uniform
      hist_count_block<K, NB, BLOCK, IPT>(keys + beg, cnt, true, 1, s_cnt, s_max, s_neg, cls);
    }
    for (int q = tid; q < NB; q += BLOCK) tb.cnt_raw[static_cast<size_t>(b) * NB + q] = s_cnt[q];
    if (tid == 0) {
      tb.cls_raw[b] = static_cast<uint32_t>(cls);
      s_cmax = max(s_cmax, static_cast<uint32_t>(cls));
    }
    __syncthreads();  // s_cnt reuse; the stage just read may be refilled
  }
  flush(seg);
}

// ---------------------------------------------------------------------------
// k_finalize: one thread per segment: the image (flipped when the segment
// holds a negative int32 key) and the segment class C.
// ---------------------------------------------------------------------------
template <int NB>
__global__ void k_finalize(uint32_t nseg, Tables tb) {
  griddep_open();
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  const uint32_t neg = tb.seg_neg[s];
  const bool empty = tb.blk_prefix[s + 1] == tb.blk_prefix[s];
  const uint32_t C = tb.seg_cmax[s * 2 + (neg ? 1 : 0)];
  tb.seg_class[s] = empty ? (NB == 10 ? 1u : 0u) : C;
  tb.seg_flip[s] = neg;
}

// ---------------------------------------------------------------------------
// k_fold: block b's count for packet p under its segment's class C, written
// at (segment s, packet p, block b): index blk_prefix[s]*NB + p*nb_s + (b - first block).
// ---------------------------------------------------------------------------
template <int NB>
__global__ void k_fold(uint32_t nseg, Tables tb) {
  griddep_open();
  const uint32_t total = tb.blk_prefix[nseg];
  const uint64_t m = static_cast<uint64_t>(total) * NB;
  for (uint64_t idx = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; idx < m;
       idx += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint32_t b = static_cast<uint32_t>(idx / NB), p = static_cast<uint32_t>(idx % NB);
    const uint32_t s = find_seg(tb.blk_prefix, nseg, b);
    const uint32_t first = tb.blk_prefix[s], nb_s = tb.blk_prefix[s + 1] - first;
    const uint32_t C = tb.seg_class[s], cb = tb.cls_raw[b];
    const uint32_t* raw = tb.cnt_raw + static_cast<size_t>(b) * NB;
    uint32_t v = 0;
    if constexpr (NB == 10) {
      if (cb == C) {
        v = raw[p];
      } else if (p == 0) {  // every key of the block is below 10^(C-1): packet 0
#pragma unroll
        for (int t = 0; t < 10; ++t) v += raw[t];
      }
    } else {
      const uint32_t d = (C > 8 ? C - 8 : 0) - (cb > 8 ? cb - 8 : 0);
      const uint32_t lo = p << d, hi = min(static_cast<uint32_t>(NB), (p + 1) << d);
      for (uint32_t t = lo; t < hi; ++t) v += raw[t];
    }
    tb.flat[static_cast<size_t>(first) * NB + static_cast<size_t>(p) * nb_s + (b - first)] = v;
  }
}

// ---------------------------------------------------------------------------
// k_pkt: per (segment, packet): the packet's absolute start and its tiles.
// ---------------------------------------------------------------------------
template <int NB>
__global__ void k_pkt(uint32_t nseg, uint32_t tile, Tables tb) {
  griddep_open();
  const uint64_t m = static_cast<uint64_t>(nseg) * NB;
  for (uint64_t idx = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; idx < m;
       idx += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint32_t s = static_cast<uint32_t>(idx / NB), p = static_cast<uint32_t>(idx % NB);
    const uint32_t first = tb.blk_prefix[s], nb_s = tb.blk_prefix[s + 1] - first;
    const uint64_t sb = tb.small_before[s];
    // a segment without blocks (empty or short) has no tiles here
    const uint64_t start = nb_s ? sb + tb.flat[static_cast<size_t>(first) * NB + static_cast<size_t>(p) * nb_s]
                                : tb.seg_off[s];
    const uint64_t end = !nb_s ? tb.seg_off[s]
                               : (p + 1 < NB) ? sb + tb.flat[static_cast<size_t>(first) * NB + static_cast<size_t>(p + 1) * nb_s]
                                              : tb.seg_off[s + 1];
    tb.pkt_off[idx] = start;
    const uint32_t tiles = static_cast<uint32_t>((end - start + tile - 1) / tile);
    tb.unit_prefix[idx] = tiles;
    // merge passes this packet needs; the largest is kept for the merge passes
    const uint32_t passes = static_cast<uint32_t>(passes_of(tiles, tb.fan_log2));
    const uint32_t wmax = __reduce_max_sync(__activemask(), passes);
    if (wmax && passes == wmax) atomicMax(&tb.pass_ctl[0], wmax);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) tb.pkt_off[m] = tb.seg_off[nseg];
}

// ---------------------------------------------------------------------------
// k_pkt_whole: no MSD step (ablation): every segment is one packet.
// ---------------------------------------------------------------------------
static __global__ void k_pkt_whole(uint32_t nseg, uint32_t tile, Tables tb) {
  griddep_open();
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x) {
    const uint64_t start = tb.seg_off[s], end = seg_is_small(tb, s) ? start : tb.seg_off[s + 1];
    tb.pkt_off[s] = start;
    const uint32_t tiles = static_cast<uint32_t>((end - start + tile - 1) / tile);
    tb.unit_prefix[s] = tiles;
    const uint32_t passes = static_cast<uint32_t>(passes_of(tiles, tb.fan_log2));
    if (passes) atomicMax(&tb.pass_ctl[0], passes);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) tb.pkt_off[nseg] = tb.seg_off[nseg];
}

// ---------------------------------------------------------------------------
// k_scan_units: in-place exclusive scan of unit_prefix[0..m), total to [m].
// ---------------------------------------------------------------------------
static __global__ void k_scan_units(uint32_t m, Tables tb) {
  griddep_open();
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < m; base += nt) {
    const uint32_t i = base + tid;
    const uint32_t x0 = (i < m) ? tb.unit_prefix[i] : 0;
    uint32_t v = x0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t x = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += x;
    }
    if (lane == 31) s_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
      uint32_t w = (lane < (nt >> 5)) ? s_warp[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t x = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += x;
      }
      s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t incl = v + (wid ? s_warp[wid - 1] : 0);
    const uint32_t carry = s_carry;
    if (i < m) tb.unit_prefix[i] = carry + incl - x0;
    __syncthreads();
    if (tid == nt - 1) s_carry = carry + incl;
    __syncthreads();
  }
  if (tid == 0) tb.unit_prefix[m] = s_carry;
}

// ---------------------------------------------------------------------------
// In-place exclusive scan of a[0, m) by the calling CTA alone (any multiple
// of 32 threads up to 1024); the total goes to *total.  All threads call it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cta_exclusive_scan(uint32_t* a, uint32_t m, uint32_t* total, uint32_t* s_warp,
                                                   uint32_t* s_carry) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) *s_carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < m; base += nt) {
    const uint32_t i = base + tid;
    const uint32_t x0 = (i < m) ? a[i] : 0u;
    uint32_t v = x0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += x;
    }
    if (lane == 31) s_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
      uint32_t w = (lane < (nt >> 5)) ? s_warp[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += x;
      }
      s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t incl = v + (wid ? s_warp[wid - 1] : 0u);
    const uint32_t carry = *s_carry;
    if (i < m) a[i] = carry + incl - x0;
    __syncthreads();
    if (tid == nt - 1) *s_carry = carry + incl;
    __syncthreads();
  }
  if (tid == 0) *total = *s_carry;
}

// ---------------------------------------------------------------------------
// k_plan_small: for small calls (at most kPlanSmallEntries block x packet and
// segment x packet entries) the steps between the histogram and the scatter
// -- k_finalize, k_fold, the three-kernel scan, k_pkt and k_scan_units -- in
// one CTA, one launch instead of seven.  Same results, same tables.  With
// NB == 1 (no MSD step) it is k_pkt_whole and k_scan_units.
// ---------------------------------------------------------------------------
constexpr uint32_t kPlanSmallEntries = 1u << 16;

// Count of packet p of block b under class C when the block's own class cb
// differs from C (see k_fold).
template <int NB>
__device__ __forceinline__ uint32_t fold_other(const Tables& tb, uint32_t b, uint32_t p, uint32_t cb, uint32_t C) {
  const uint32_t* raw = tb.cnt_raw + static_cast<size_t>(b) * NB;
  uint32_t v = 0;
  if constexpr (NB == 10) {
    if (p == 0) {  // every key of the block is below 10^(C-1): packet 0
#pragma unroll
      for (int t = 0; t < 10; ++t) v += raw[t];
    }
  } else {
    const uint32_t d = (C > 8 ? C - 8 : 0) - (cb > 8 ? cb - 8 : 0);
    const uint32_t l = p << d, h = min(static_cast<uint32_t>(NB), (p + 1) << d);
    for (uint32_t t = l; t < h; ++t) v += raw[t];
  }
  return v;
}

// Entry e of the (segment, packet, block) array: its block b, packet p and
// the segment's class C.  Segment s owns entries
// [blk_prefix[s] * NB, blk_prefix[s + 1] * NB), packet-major inside it.
template <int NB>
__device__ __forceinline__ void folded_pos(const Tables& tb, uint32_t nseg, uint32_t e, uint32_t& b, uint32_t& p,
                                           uint32_t& C) {
  uint32_t lo = 0, hi = nseg;  // last s with blk_prefix[s] * NB <= e
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (tb.blk_prefix[mid] * NB <= e) lo = mid; else hi = mid;
  }
  const uint32_t first = tb.blk_prefix[lo], nb_s = tb.blk_prefix[lo + 1] - first;
  const uint32_t rel = e - first * NB;
  p = rel / nb_s;
  b = first + (rel - p * nb_s);
  C = tb.seg_class[lo];
}

constexpr int kPlanThreads = 1024;
constexpr int kPer = 8;                          // entries per thread per chunk
constexpr int kChunk = kPlanThreads * kPer;
__device__ __forceinline__ uint32_t chunk_pad(uint32_t i) { return i + (i >> 5); }

template <int NB>
__global__ void __launch_bounds__(kPlanThreads) k_plan_small(uint32_t nseg, uint32_t tile, Tables tb) {
  griddep_open();
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_chunk[kChunk + kChunk / 32];  // one pad word per 32: conflict-free raking
  __shared__ uint32_t s_carry;
  const uint32_t tid = threadIdx.x, nt = blockDim.x;
  const uint32_t m = nseg * NB;
  if constexpr (NB == 1) {
    for (uint32_t s = tid; s < nseg; s += nt) {
      const uint64_t start = tb.seg_off[s], end = seg_is_small(tb, s) ? start : tb.seg_off[s + 1];
      tb.pkt_off[s] = start;
      const uint32_t tiles = static_cast<uint32_t>((end - start + tile - 1) / tile);
      tb.unit_prefix[s] = tiles;
      const uint32_t passes = static_cast<uint32_t>(passes_of(tiles, tb.fan_log2));
      if (passes) atomicMax(&tb.pass_ctl[0], passes);
    }
    if (tid == 0) tb.pkt_off[nseg] = tb.seg_off[nseg];
  } else {
    // finalize: segment class and image
    for (uint32_t s = tid; s < nseg; s += nt) {
      const uint32_t neg = tb.seg_neg[s];
      const bool empty = tb.blk_prefix[s + 1] == tb.blk_prefix[s];
      const uint32_t C = tb.seg_cmax[s * 2 + (neg ? 1 : 0)];
      tb.seg_class[s] = empty ? (NB == 10 ? 1u : 0u) : C;
      tb.seg_flip[s] = neg;
    }
    __syncthreads();
    // fold + exclusive scan in chunks of kChunk entries: every thread loads and
    // folds kPer entries strided by the CTA size (coalesced, all loads in flight
    // at once) into shared memory, then scans kPer contiguous ones (raking),
    // and the chunk leaves coalesced with the running carry
    const uint32_t total = tb.blk_prefix[nseg];
    const uint32_t E = total * NB;
    const uint32_t C0 = tb.seg_class[0];
    const uint32_t lane = tid & 31, wid = tid >> 5;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < E; base += kChunk) {
      uint32_t cb[kPer], direct[kPer], bb[kPer], pp[kPer], cc[kPer];
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const uint32_t e = base + k * kPlanThreads + tid;
        uint32_t b = 0, p = 0, C = C0;
        if (e < E) {
          if (nseg == 1) {
            p = e / total;
            b = e - p * total;
          } else {
            folded_pos<NB>(tb, nseg, e, b, p, C);
          }
        }
        bb[k] = b;
        pp[k] = p;
        cc[k] = C;
        cb[k] = (e < E) ? tb.cls_raw[b] : C;
        direct[k] = (e < E) ? tb.cnt_raw[static_cast<size_t>(b) * NB + p] : 0u;
      }
#pragma unroll
      for (int k = 0; k < kPer; ++k)
        s_chunk[chunk_pad(k * kPlanThreads + tid)] =
            (cb[k] == cc[k]) ? direct[k] : fold_other<NB>(tb, bb[k], pp[k], cb[k], cc[k]);
      __syncthreads();
      uint32_t x[kPer];
      uint32_t sum = 0;
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        x[k] = s_chunk[chunk_pad(tid * kPer + k)];
        sum += x[k];
      }
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= static_cast<uint32_t>(o)) incl += y;
      }
      if (lane == 31) s_warp[wid] = incl;
      __syncthreads();
      if (wid == 0) {
        uint32_t w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
          if (lane >= static_cast<uint32_t>(o)) w += y;
        }
        s_warp[lane] = w;  // inclusive over warps
      }
      __syncthreads();
      uint32_t run = carry + incl - sum + (wid ? s_warp[wid - 1] : 0u);
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        s_chunk[chunk_pad(tid * kPer + k)] = run;
        run += x[k];
      }
      const uint32_t chunk_total = s_warp[31];
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const uint32_t e = base + k * kPlanThreads + tid;
        if (e < E) tb.flat[e] = s_chunk[chunk_pad(k * kPlanThreads + tid)];
      }
      carry += chunk_total;
      __syncthreads();  // s_chunk and s_warp are reused by the next chunk
    }
    // packet starts and tiles
    for (uint32_t idx = tid; idx < m; idx += nt) {
      const uint32_t s = idx / NB, p = idx % NB;
      const uint32_t first = tb.blk_prefix[s], nb_s = tb.blk_prefix[s + 1] - first;
      const uint64_t sb = tb.small_before[s];
      const uint64_t start = nb_s ? sb + tb.flat[static_cast<size_t>(first) * NB + static_cast<size_t>(p) * nb_s]
                                  : tb.seg_off[s];
      const uint64_t end = !nb_s ? tb.seg_off[s]
                                 : (p + 1 < NB)
                                       ? sb + tb.flat[static_cast<size_t>(first) * NB + static_cast<size_t>(p + 1) * nb_s]
                                       : tb.seg_off[s + 1];
      tb.pkt_off[idx] = start;
      const uint32_t tiles = static_cast<uint32_t>((end - start + tile - 1) / tile);
      tb.unit_prefix[idx] = tiles;
      const uint32_t passes = static_cast<uint32_t>(passes_of(tiles, tb.fan_log2));
      if (passes) atomicMax(&tb.pass_ctl[0], passes);
    }
    if (tid == 0) tb.pkt_off[m] = tb.seg_off[nseg];
  }
  __syncthreads();
  // first tile of every packet
  cta_exclusive_scan(tb.unit_prefix, m, tb.unit_prefix + m, s_warp, &s_carry);
}

// ---------------------------------------------------------------------------
// k_scatter: stable move into packets, one CTA per packet-step block.  Each
// warp ranks its keys in input order (warp-striped items, a match over packet
// ids); warps are ordered by position; the block's absolute first position
// in every packet comes from the scan.  Keys are staged in shared memory
// grouped by packet and written out as contiguous runs.  Every write is
// checked against its packet's end (kErrBounds on violation, write skipped).
// ---------------------------------------------------------------------------
template <class K, bool HAS_V, int NB, int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK, 2) k_scatter(const K* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                                                    K* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                                                    uint32_t nseg, uint32_t part_tile, Tables tb) {
  griddep_open();
  constexpr int NW = BLOCK / kWarp;
  constexpr int TILE = BLOCK * IPT;
  constexpr int NBX = NB + 1;  // + a dummy packet for lanes past the end
  extern __shared__ __align__(128) unsigned char s_raw[];
  K* s_keys = reinterpret_cast<K*>(s_raw);                               // TILE
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + TILE);        // TILE (pairs)
  uint32_t* s_wc = s_vals + (HAS_V ? TILE : 0);                         // NW * NBX warp counts
  uint32_t* s_bs = s_wc + NW * NBX;                                     // NB + 1 block packet starts
  uint32_t* s_gb = s_bs + ((NB + 2) & ~1);                              // NB absolute bases, then deltas
  uint32_t* s_pe = s_gb + ((NB + 1) & ~1);                              // NB packet ends (absolute)
  uint16_t* s_pk = reinterpret_cast<uint16_t*>(s_pe + ((NB + 1) & ~1)); // TILE packet ids

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t b = blockIdx.x;
  const uint32_t total = tb.blk_prefix[nseg];
  if (b >= total) return;
  for (int i = tid; i < NW * NBX; i += BLOCK) s_wc[i] = 0;
  const uint32_t seg = find_seg(tb.blk_prefix, nseg, b);
  const uint32_t first = tb.blk_prefix[seg], nb_s = tb.blk_prefix[seg + 1] - first;
  const uint64_t beg = tb.seg_off[seg] + static_cast<uint64_t>(b - first) * part_tile;
  const uint32_t cnt = static_cast<uint32_t>(min64(part_tile, tb.seg_off[seg + 1] - beg));
  const bool flip = tb.seg_flip[seg] != 0;
  const int cls = static_cast<int>(tb.seg_class[seg]);
  const DigitRule rule = (NB == 10) ? rule_dec(cls) : make_rule_bin(cls);
  // absolute first position of this block's keys in every packet
  for (int p = tid; p < NB; p += BLOCK) {
    s_gb[p] = tb.small_before[seg] + tb.flat[static_cast<size_t>(first) * NB + static_cast<size_t>(p) * nb_s + (b - first)];
    s_pe[p] = static_cast<uint32_t>(tb.pkt_off[static_cast<size_t>(seg) * NB + p + 1]);
  }
  __syncthreads();

  // load (warp-striped) and compute packets; rank and packet share a register
  K k[IPT];
  uint32_t v[IPT];
  uint32_t rq[IPT];  // packet in bits 0..15, warp rank in bits 16..31
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const uint32_t i = wid * kWarp * IPT + j * kWarp + lane;
    if (i < cnt) {
      k[j] = keys_in[beg + i];
      if constexpr (HAS_V) v[j] = vals_in[beg + i];
      rq[j] = packet_of<NB>(KT<K>::image(k[j], flip), rule);
    } else {
      rq[j] = NB;
    }
  }
  // warp ranking in input order; every item's peers first (independent
  // matches overlap), then the running per-warp counts
  uint32_t* wc = s_wc + wid * NBX;
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t pm[IPT];
#pragma unroll
  for (int j = 0; j < IPT; ++j) pm[j] = __match_any_sync(0xffffffffu, rq[j]);
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const uint32_t q = rq[j];
    const uint32_t peers = pm[j];
    const uint32_t base = wc[q];
    rq[j] = q | ((base + __popc(peers & lt_mask)) << 16);
    __syncwarp();
    if (lane == __ffs(peers) - 1) wc[q] = base + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per packet: warp prefixes (in place in s_wc) and block totals
  for (int p = tid; p < NB; p += BLOCK) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const uint32_t c = s_wc[w * NBX + p];
      s_wc[w * NBX + p] = run;
      run += c;
    }
    s_bs[p] = run;
  }
  __syncthreads();
  {  // block packet starts: exclusive scan of the totals (one packet per thread)
    static_assert(NB <= BLOCK && BLOCK == kScanBlock, "one packet per thread");
    __shared__ uint32_t s_warp[32];
    const uint32_t c = (tid < NB) ? s_bs[tid] : 0u;
    const uint32_t incl = block_incl_scan(c, s_warp);
    if (tid < NB) s_bs[tid] = incl - c;
    if (tid == NB - 1) s_bs[NB] = incl;
  }
  __syncthreads();
  // staged element e of packet p goes to e + (first position - block start) of p
  for (int p = tid; p < NB; p += BLOCK) s_gb[p] -= s_bs[p];
  // stage grouped by packet, in input order inside each packet
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const uint32_t q = rq[j] & 0xffffu;
    if (q < NB) {
      const uint32_t pos = s_bs[q] + s_wc[wid * NBX + q] + (rq[j] >> 16);
      s_keys[pos] = k[j];
      if constexpr (HAS_V) s_vals[pos] = v[j];
      s_pk[pos] = static_cast<uint16_t>(q);
    }
  }
  __syncthreads();
  for (uint32_t e = tid; e < cnt; e += BLOCK) {
    const uint32_t p = s_pk[e];
    const uint32_t dst = s_gb[p] + e;  // positions < n < 2^32
    if (dst >= s_pe[p]) {
      atomicOr(tb.err, kErrBounds);
      continue;
    }
    keys_out[dst] = s_keys[e];
    if constexpr (HAS_V) vals_out[dst] = s_vals[e];
  }
}

// ---------------------------------------------------------------------------
// k_scatter_small: the stable move for up to 16 packets (the ten decimal
// packets), persistent CTAs over blocks blockIdx.x, +gridDim.x, ...
//   * a block's keys (and values) arrive by bulk copy in one of the CTA's
//     input stages; thread t takes items t*IPT .. t*IPT+IPT-1 (so input order
//     is thread order, then item order).  With two stages the next block's
//     copy is issued as soon as this block's has landed (into the stage the
//     previous block was read from); with one (64-bit keys with values, where
//     a second stage would halve the CTAs per SM) once every thread holds its
//     items;
//   * each thread counts its items per packet in 4-bit fields (its local rank
//     of every item falls out on the way), and one block-wide scan of those
//     counts, two packets per 32-bit word, gives every thread its first rank
//     in every packet: stable ranks without a per-item warp vote;
//   * every packet's run is staged in shared memory at the 16-byte phase of
//     its destination and leaves as one bulk store (unaligned ends by plain
//     stores); a run that would pass its packet's end sets kErrBounds and is
//     not written.
// The output buffers must be 16-byte aligned (the work space is 256-byte
// aligned).
// ---------------------------------------------------------------------------
template <class K, bool HAS_V, int BLOCK, int IPT>
struct ScatterSmallLayout {
  static constexpr int TILE = BLOCK * IPT;
  static constexpr int STAGES = (sizeof(K) == 8 && HAS_V) ? 1 : 2;
  static constexpr size_t SK = (region_elems(TILE) * sizeof(K) + 127) & ~size_t(127);
  static constexpr size_t SV = HAS_V ? ((region_elems(TILE) * 4 + 127) & ~size_t(127)) : 0;
  static constexpr int OUTE = TILE + 8 * 16;  // runs padded to their phase: at most 7 extra per run
  static constexpr size_t OK = (OUTE * sizeof(K) + 127) & ~size_t(127);
  static constexpr size_t OV = HAS_V ? ((OUTE * 4 + 127) & ~size_t(127)) : 0;
  static constexpr size_t PREF = BLOCK * 16 * 2;  // u16 first staging position per thread and packet
  static constexpr size_t bytes = STAGES * (SK + SV) + OK + OV + PREF;
};

// Register budget: four CTAs per SM for 4-byte keys without values (64
// registers; its shared memory, ~54 KB, fits four times under the largest
// carveout, which the launch requests), two otherwise.
template <class K, bool HAS_V, int NB, int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK, (HAS_V || sizeof(K) == 8) ? 2 : 4) k_scatter_small(const K* __restrict__ keys_in,
                                                            const uint32_t* __restrict__ vals_in,
                                                            K* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                                                            uint32_t nseg, uint32_t part_tile, int debug_stuck,
                                                            uint64_t limit_ns, Tables tb) {
  griddep_open();
  static_assert(NB <= 16 && IPT <= 15, "4-bit local counts; 16-bit block counts");
  using LY = ScatterSmallLayout<K, HAS_V, BLOCK, IPT>;
  constexpr int NW = BLOCK / kWarp;
  constexpr int NWORD = (NB + 1) / 2;
  constexpr int ST = LY::STAGES;
  extern __shared__ __align__(128) unsigned char s_raw[];
  auto s_in = [&](int st) { return reinterpret_cast<K*>(s_raw + st * LY::SK); };
  auto s_inv = [&](int st) { return reinterpret_cast<uint32_t*>(s_raw + ST * LY::SK + st * LY::SV); };
  K* s_out = reinterpret_cast<K*>(s_raw + ST * (LY::SK + LY::SV));
  uint32_t* s_outv = reinterpret_cast<uint32_t*>(s_raw + ST * (LY::SK + LY::SV) + LY::OK);
  uint16_t* s_pref = reinterpret_cast<uint16_t*>(s_raw + ST * (LY::SK + LY::SV) + LY::OK + LY::OV);
  __shared__ uint32_t s_wsum[NW][NWORD];
  __shared__ uint32_t s_blk[NWORD];
  __shared__ uint32_t s_run[NB], s_tot[NB], s_dst[NB], s_pe[NB];
  __shared__ __align__(8) uint64_t s_bar[2];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  const uint32_t total = tb.blk_prefix[nseg];
  const uint32_t G = gridDim.x;
  uint32_t b = blockIdx.x;
  if (b >= total) return;
  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
  }
  mbar_fence_init();
  __syncthreads();

  auto geom = [&](uint32_t bb, uint32_t& sg, uint64_t& beg, uint32_t& cnt) {
    sg = find_seg(tb.blk_prefix, nseg, bb);
    beg = tb.seg_off[sg] + static_cast<uint64_t>(bb - tb.blk_prefix[sg]) * part_tile;
    cnt = static_cast<uint32_t>(min64(part_tile, tb.seg_off[sg + 1] - beg));
  };
  auto issue = [&](uint32_t bb, int st) {  // one warp (the last)
    uint32_t sg, c;
    uint64_t bg;
    geom(bb, sg, bg, c);
    if (lane == 0) fence_proxy_async();  // the generic reads of the stage happened before the last barrier
    __syncwarp();
    const PendingBulk<K> pk = load_window_singles(s_in(st), phase_of(keys_in + bg), keys_in + bg, c, lane);
    PendingBulk<uint32_t> pv{nullptr, nullptr, 0};
    if constexpr (HAS_V) pv = load_window_singles(s_inv(st), phase_of(vals_in + bg), vals_in + bg, c, lane);
    cp_async_mbar_arrive(&s_bar[st]);
    __syncwarp();
    if (lane == 0) {
      // testing hook: CTA 0 announces 16 bytes that never arrive for its
      // first block, so its bounded wait expires
      const uint32_t extra = (debug_stuck && blockIdx.x == 0 && bb == blockIdx.x) ? 16u : 0u;
      mbar_arrive_expect_tx(&s_bar[st], pk.bytes + pv.bytes + extra);
      if (pk.bytes) bulk_g2s(pk.sdst, pk.gsrc, pk.bytes, &s_bar[st]);
      if (HAS_V && pv.bytes) bulk_g2s(pv.sdst, pv.gsrc, pv.bytes, &s_bar[st]);
    }
  };
  // absolute first position and packet end of every packet of block bb (threads < NB)
  auto load_dst = [&](uint32_t bb, uint32_t& d, uint32_t& e) {
    const uint32_t sg = find_seg(tb.blk_prefix, nseg, bb);
    const uint32_t first = tb.blk_prefix[sg], nb_s = tb.blk_prefix[sg + 1] - first;
    d = tb.small_before[sg] + tb.flat[static_cast<size_t>(first) * NB + static_cast<size_t>(tid) * nb_s + (bb - first)];
    e = static_cast<uint32_t>(tb.pkt_off[static_cast<size_t>(sg) * NB + tid + 1]);
  };

  constexpr int kIssueWarp = NW - 1;  // warp 0 computes the run offsets
  if (wid == kIssueWarp) issue(b, 0);
  uint32_t nd = 0, npe = 0;
  if (tid < NB) load_dst(b, nd, npe);
  uint32_t par0 = 0, par1 = 0;
  int st = 0;
  bool failed = false;
  for (; b < total; b += G) {
    uint32_t seg, cnt;
    uint64_t beg;
    geom(b, seg, beg, cnt);
    const bool ok = mbar_wait_bounded(&s_bar[st], st ? par1 : par0, tb.err, limit_ns);
    if (st) par1 ^= 1; else par0 ^= 1;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    // after the barrier: every warp has finished the previous block's stores,
    // which read s_dst and s_pe, and its reads of the other stage
    if constexpr (ST == 2) {
      if (wid == kIssueWarp && b + G < total) issue(b + G, st ^ 1);  // refill the other stage now
    }
    if (tid < NB) {
      s_dst[tid] = nd;
      s_pe[tid] = npe;
      if (b + G < total) load_dst(b + G, nd, npe);
    }
    const bool flip = tb.seg_flip[seg] != 0;
    const DigitRule rule = (NB == 10) ? rule_dec(static_cast<int>(tb.seg_class[seg]))
                                      : make_rule_bin(static_cast<int>(tb.seg_class[seg]));
    const K* rk = s_in(st) + phase_of(keys_in + beg);
    const uint32_t* rv = HAS_V ? s_inv(st) + phase_of(vals_in + beg) : nullptr;
    K k[IPT];
    uint32_t v[IPT];
    uint32_t pr[IPT];  // packet in bits 0..7 (NB = none), local rank from bit 8
    uint32_t lo = 0, hi = 0;
    auto take = [&](int j) {
      const uint32_t i = tid * IPT + j;
      k[j] = rk[i];
      if constexpr (HAS_V) v[j] = rv[i];
      const uint32_t p = packet_of<NB>(KT<K>::image(k[j], flip), rule);
      const uint32_t sh = 4 * (p & 7);
      const uint32_t lr = (((p < 8) ? lo : hi) >> sh) & 15u;
      if (p < 8) lo += 1u << sh; else hi += 1u << sh;
      pr[j] = p | (lr << 8);
    };
    if (cnt == static_cast<uint32_t>(LY::TILE)) {  // full block: no bounds tests
#pragma unroll
      for (int j = 0; j < IPT; ++j) take(j);
    } else {
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        if (tid * IPT + j < cnt) take(j);
        else pr[j] = NB;
      }
    }
    if constexpr (ST == 1) {
      __syncthreads();  // every item is in registers: the stage may be refilled
      if (wid == kIssueWarp && b + G < total) issue(b + G, 0);
    }
    // local counts, two packets per word, and their block-wide scan
    uint32_t wv[NWORD], incl[NWORD];
#pragma unroll
    for (int q = 0; q < NWORD; ++q) {
      const uint32_t c0 = (((2 * q < 8) ? lo : hi) >> (4 * ((2 * q) & 7))) & 15u;
      const uint32_t c1 = (2 * q + 1 < NB) ? ((((2 * q + 1 < 8) ? lo : hi) >> (4 * ((2 * q + 1) & 7))) & 15u) : 0u;
      wv[q] = c0 | (c1 << 16);
      uint32_t x = wv[q];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      incl[q] = x;
      if (lane == 31) s_wsum[wid][q] = x;
    }
    if (lane == 0) bulk_wait_read0();  // this warp's stores of the previous block have read the staging buffer
    __syncthreads();
    if (wid == 0) {
      if (lane < NWORD) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const uint32_t t = s_wsum[w][lane];
          s_wsum[w][lane] = run;
          run += t;
        }
        s_blk[lane] = run;
      }
      __syncwarp();
      // staging start of every run: at its destination's 16-byte phase
      uint32_t tot = 0, units = 0;
      if (lane < NB) {
        tot = (s_blk[lane >> 1] >> (16 * (lane & 1))) & 0xffffu;
        units = (tot + 3) / 4 + 1;
      }
      uint32_t x = units;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane < NB) {
        s_run[lane] = 4 * (x - units) + (s_dst[lane] & 3u);
        s_tot[lane] = tot;
      }
    }
    __syncthreads();
    // this thread's first staging position in every packet
#pragma unroll
    for (int p = 0; p < NB; ++p) {
      const uint32_t ex = incl[p >> 1] - wv[p >> 1] + s_wsum[wid][p >> 1];
      s_pref[tid * NB + p] = static_cast<uint16_t>(s_run[p] + ((ex >> (16 * (p & 1))) & 0xffffu));
    }
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const uint32_t p = pr[j] & 0xffu;
      if (p < NB) {
        const uint32_t pos = s_pref[tid * NB + p] + (pr[j] >> 8);
        s_out[pos] = k[j];
        if constexpr (HAS_V) s_outv[pos] = v[j];
      }
    }
    fence_proxy_async();
    __syncthreads();
    // warp w stores the runs of packets w, w + NW, ...
    bool stored = false;
#pragma unroll 1
    for (int p = wid; p < NB; p += NW) {
      const uint32_t t = s_tot[p];
      if (t == 0) continue;
      const uint32_t d = s_dst[p];
      if (d + t > s_pe[p]) {
        if (lane == 0) atomicOr(tb.err, kErrBounds);
        continue;
      }
      store_window(keys_out + d, s_out + s_run[p], t, lane);
      if constexpr (HAS_V) store_window(vals_out + d, s_outv + s_run[p], t, lane);
      stored = true;
    }
    if (stored && lane == 0) bulk_commit();
    if constexpr (ST == 2) st ^= 1;
  }
  // the copy that did not arrive may still be in flight into its stage (the
  // next block's copy is issued only after the barrier that saw the failure):
  // give it a bounded chance to land before the CTA's shared memory is released
  if (failed) mbar_wait_bounded(&s_bar[st], st ? par1 ^ 1u : par0 ^ 1u, tb.err, limit_ns);
  if (lane == 0) bulk_wait0();
}

}  // namespace hs
