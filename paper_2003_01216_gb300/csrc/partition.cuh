// Packet step (Sec. 2.1, Sec. 3.4): one MSD-radix pass that moves every key
// into one of ten packets (or 256 buckets for the ablation) by the leading
// digit of its image, keeping input order inside each packet.
//
// Kernels, in launch order:
//   k_seg_plan   segment table and packet-step block prefix (one CTA)
//   k_hist       per-block class + per-class packet counts (one read of the keys)
//   k_finalize   per segment: final class, folded packet counts, packet offsets,
//                tiles per packet
//   k_scan_units exclusive scan of the tiles per packet (one CTA)
//   k_scatter    stable scatter into packets with a decoupled look-back across
//                blocks (one read + one write of keys and values)
//
// The class trick: the packet of a key depends on the class (digit count D,
// or bit length B) of the LARGEST key image of its array, which no block
// knows before the whole array has been read.  k_hist therefore counts every
// block under its own block-local class c_b and files the counts under c_b.
// A block whose class is below the array's class C holds only keys smaller
// than every threshold of C (decimal: all its keys fall in packet 0; binary:
// its local bucket t becomes t >> (shift(C) - shift(c_b))), so k_finalize can
// fold every row into the counts under C exactly, after one read of the keys.
#pragma once
#include "common.cuh"

namespace hs {

constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagInc = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;

// ---------------------------------------------------------------------------
// k_seg_plan: segment table.  Plain sorts pass offs == nullptr (one segment
// [0, n)).  Batches pass the caller's offsets, which are validated here; if
// they are malformed every segment is treated as empty (no key moves) and the
// error word gets kErrBadOffsets.
// ---------------------------------------------------------------------------
static __global__ void k_seg_plan(const uint64_t* __restrict__ offs, uint32_t nseg, uint64_t n, uint32_t part_tile,
                           Tables tb) {
  __shared__ uint32_t s_bad;
  __shared__ uint32_t s_carry;
  __shared__ uint32_t s_warp[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) {
    s_bad = 0;
    s_carry = 0;
  }
  __syncthreads();
  if (offs) {
    for (uint32_t s = tid; s < nseg; s += nt)
      if (offs[s + 1] < offs[s]) s_bad = 1;
    if (tid == 0 && (offs[0] != 0 || offs[nseg] != n)) s_bad = 1;
  }
  __syncthreads();
  const bool bad = s_bad != 0;
  if (bad && tid == 0) atomicOr(tb.err, kErrBadOffsets);
  for (uint32_t base = 0; base <= nseg; base += nt) {
    uint32_t s = base + tid;
    uint64_t lo = 0, hi = 0;
    if (s <= nseg) {
      uint64_t so = offs ? offs[s] : (s == 0 ? 0 : n);
      tb.seg_off[s] = bad ? 0 : so;
    }
    uint32_t nblk = 0;
    if (s < nseg && !bad) {
      lo = offs ? offs[s] : 0;
      hi = offs ? offs[s + 1] : n;
      nblk = static_cast<uint32_t>((hi - lo + part_tile - 1) / part_tile);
    }
    // block-wide exclusive scan of nblk
    uint32_t v = nblk;
    const int lane = tid & 31, wid = tid >> 5;
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
      s_warp[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    uint32_t incl = v + (wid ? s_warp[wid - 1] : 0);
    uint32_t carry = s_carry;
    if (s <= nseg) tb.blk_prefix[s] = carry + incl - nblk;
    __syncthreads();
    if (tid == nt - 1) s_carry = carry + incl;
    __syncthreads();
  }
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
// block it reduces the largest key image, takes the block's class, and counts
// its keys per packet under that class into a shared-memory table
// acc[class][packet]; the table is flushed into the segment's global
// histogram when the segment changes and at the end.
//   img = 0: identity image (and every segment's "has a negative key" flag)
//   img = 1: sign-flipped image, only for segments flagged by the img = 0 pass
// ---------------------------------------------------------------------------
template <class K, int NB, int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK) k_hist(const K* __restrict__ keys, uint32_t nseg, uint32_t part_tile,
                                                 int img, Tables tb) {
  using U = typename KT<K>::U;
  constexpr int NCLS = (NB == 10) ? kDecClasses : kBinClasses;
  constexpr int NW = BLOCK / kWarp;
  extern __shared__ uint32_t s_acc[];  // [NCLS][NB]
  __shared__ U s_max[NW];
  __shared__ uint32_t s_neg;
  __shared__ unsigned long long s_used[2];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  const uint32_t total = tb.blk_prefix[nseg];
  const uint32_t per = (total + gridDim.x - 1) / gridDim.x;
  const uint32_t b0 = min(total, blockIdx.x * per), b1 = min(total, b0 + per);
  if (b0 >= b1) return;

  for (int i = tid; i < NCLS * NB; i += BLOCK) s_acc[i] = 0;
  if (tid == 0) {
    s_used[0] = s_used[1] = 0;
    s_neg = 0;
  }
  __syncthreads();

  uint32_t seg = find_seg(tb.blk_prefix, nseg, b0);
  auto flush = [&](uint32_t s) {
    __syncthreads();
    uint32_t* g = tb.hist + (static_cast<size_t>(s) * 2 + img) * NCLS * NB;
    for (int c = 0; c < NCLS; ++c) {
      if (!((s_used[c >> 6] >> (c & 63)) & 1ull)) continue;
      for (int q = tid; q < NB; q += BLOCK) {
        uint32_t v = s_acc[c * NB + q];
        if (v) {
          atomicAdd(&g[c * NB + q], v);
          s_acc[c * NB + q] = 0;
        }
      }
    }
    __syncthreads();  // every thread is done reading s_used before it is cleared
    if (tid == 0) {
      if (s_neg) atomicOr(&tb.seg_neg[s], 1u);
      s_used[0] = s_used[1] = 0;
      s_neg = 0;
    }
    __syncthreads();
  };

  for (uint32_t b = b0; b < b1; ++b) {
    while (b >= tb.blk_prefix[seg + 1]) {
      flush(seg);
      ++seg;
    }
    const bool flip = (img == 1);
    if (flip && !tb.seg_neg[seg]) continue;  // block-uniform
    const uint64_t s_lo = tb.seg_off[seg];
    const uint64_t beg = s_lo + static_cast<uint64_t>(b - tb.blk_prefix[seg]) * part_tile;
    const uint32_t cnt = static_cast<uint32_t>(min64(part_tile, tb.seg_off[seg + 1] - beg));
    const K* src = keys + beg;

    U u[IPT];
    bool any_neg = false;
    U m = 0;
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      uint32_t i = wid * kWarp * IPT + j * kWarp + lane;
      if (i < cnt) {
        K k = src[i];
        any_neg |= KT<K>::negative(k);
        u[j] = KT<K>::image(k, flip);
        m = max(m, u[j]);
      } else {
        u[j] = 0;
      }
    }
    // block max of the images
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, static_cast<U>(__shfl_xor_sync(0xffffffffu, m, o)));
    if (lane == 0) s_max[wid] = m;
    if (img == 0 && __any_sync(0xffffffffu, any_neg) && lane == 0) s_neg = 1;
    __syncthreads();
    m = s_max[0];
#pragma unroll
    for (int w = 1; w < NW; ++w) m = max(m, s_max[w]);
    const int cls = (NB == 10) ? dec_class(static_cast<uint64_t>(m)) : bin_class(m);
    const DigitRule rule = (NB == 10) ? make_rule_dec(cls) : make_rule_bin(cls);
    uint32_t* row = s_acc + cls * NB;

    if constexpr (NB == 10) {
      // packed per-thread counters: 6 bits per packet
      unsigned long long pc = 0;
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        uint32_t i = wid * kWarp * IPT + j * kWarp + lane;
        if (i < cnt) pc += 1ull << (6 * packet_of<NB>(u[j], rule));
      }
#pragma unroll
      for (int q = 0; q < 10; ++q) {
        uint32_t c = static_cast<uint32_t>((pc >> (6 * q)) & 63ull);
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0 && c) atomicAdd(&row[q], c);
      }
    } else {
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        uint32_t i = wid * kWarp * IPT + j * kWarp + lane;
        uint32_t q = (i < cnt) ? packet_of<NB>(u[j], rule) : NB;
        uint32_t peers = __match_any_sync(0xffffffffu, q);
        if (q < NB && lane == __ffs(peers) - 1) atomicAdd(&row[q], __popc(peers));
      }
    }
    if (tid == 0) atomicOr(&s_used[cls >> 6], 1ull << (cls & 63));
    __syncthreads();  // s_max reuse
  }
  flush(seg);
}

// ---------------------------------------------------------------------------
// k_finalize: one warp per segment (kFinWarps segments per CTA).  Picks the
// image (flipped when the segment holds a negative int32 key), the segment
// class C = largest class with a non-empty row, folds every row into the
// packet counts under C, and writes packet offsets and tiles per packet.
// ---------------------------------------------------------------------------
constexpr int kFinWarps = 8;

template <int NB>
__global__ void __launch_bounds__(kFinWarps * 32) k_finalize(uint32_t nseg, uint32_t tile, Tables tb) {
  constexpr int NCLS = (NB == 10) ? kDecClasses : kBinClasses;
  __shared__ uint32_t s_cnt[kFinWarps][NB];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint32_t s = blockIdx.x * kFinWarps + wib;
  if (s >= nseg) return;
  uint32_t* cnt = s_cnt[wib];
  for (int q = lane; q < NB; q += 32) cnt[q] = 0;
  __syncwarp();
  const uint32_t neg = tb.seg_neg[s];
  const uint32_t* h = tb.hist + (static_cast<size_t>(s) * 2 + (neg ? 1 : 0)) * NCLS * NB;
  // largest class with a non-empty row
  int C = -1;
  for (int c = NCLS - 1; c >= 0 && C < 0; --c) {
    bool nz = false;
    for (int q = lane; q < NB; q += 32) nz |= h[c * NB + q] != 0;
    if (__any_sync(0xffffffffu, nz)) C = c;
  }
  if (C >= 0) {
    if constexpr (NB == 10) {
      // every key of a row below C falls in packet 0
      uint32_t low = 0;
      for (int c = 0; c < C; ++c)
        if (lane < NB) low += h[c * NB + lane];
      low = __reduce_add_sync(0xffffffffu, low);
      if (lane < NB) cnt[lane] = h[C * NB + lane] + (lane == 0 ? low : 0);
    } else {
      // a row of class c holds buckets under shift(c); under shift(C) its
      // bucket t becomes t >> (shift(C) - shift(c))
      const int shC = C > 8 ? C - 8 : 0;
      for (int c = 0; c <= C; ++c) {
        const int d = shC - (c > 8 ? c - 8 : 0);
        for (int t = lane; t < NB; t += 32) {
          const uint32_t v = h[c * NB + t];
          if (v) atomicAdd(&cnt[t >> d], v);
        }
      }
    }
  }
  __syncwarp();
  uint64_t* po = tb.pkt_off + static_cast<size_t>(s) * NB;
  uint32_t* up = tb.unit_prefix + static_cast<size_t>(s) * NB;
  // exclusive prefix over packets, 32 at a time, in packet order
  uint64_t run = tb.seg_off[s];
  for (int q0 = 0; q0 < NB; q0 += 32) {
    const int q = q0 + lane;
    const uint32_t c = (q < NB) ? cnt[q] : 0;
    uint32_t v = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t x = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += x;
    }
    if (q < NB) {
      po[q] = run + (v - c);
      up[q] = (c + tile - 1) / tile;
    }
    run += __shfl_sync(0xffffffffu, v, 31);
  }
  if (lane == 0) {
    tb.seg_class[s] = C >= 0 ? static_cast<uint32_t>(C) : (NB == 10 ? 1u : 0u);
    tb.seg_flip[s] = neg;
    if (s == nseg - 1) tb.pkt_off[static_cast<size_t>(nseg) * NB] = tb.seg_off[nseg];
  }
}

// ---------------------------------------------------------------------------
// k_scan_units: in-place exclusive scan of unit_prefix[0..m), total to [m].
// ---------------------------------------------------------------------------
static __global__ void k_scan_units(uint32_t m, Tables tb) {
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
// k_scatter: stable move into packets.  Blocks take tickets in launch order
// so every block's predecessor is resident or finished (no deadlock).  Inside
// a block, each warp ranks its keys in input order (warp-striped items, a
// match over packet ids); warps are ordered by position; across blocks of the
// same segment a decoupled look-back over per-(block, packet) status words
// gives each packet's count in earlier blocks.  Keys are staged in shared
// memory grouped by packet and written out as contiguous runs.
//
// Bounded wait: a status word not published within `limit_ns` (globaltimer)
// sets kErrTimeout; the block then publishes a value anyway so its successors
// do not wait, and writes nothing.  Every write is checked against its packet's
// bounds (kErrBounds on violation, write skipped).
// ---------------------------------------------------------------------------
template <class K, bool HAS_V, int NB, int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK) k_scatter(const K* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                                                    K* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                                                    uint32_t nseg, uint32_t part_tile, uint64_t limit_ns,
                                                    int debug_stuck, Tables tb) {
  using U = typename KT<K>::U;
  constexpr int NW = BLOCK / kWarp;
  constexpr int TILE = BLOCK * IPT;
  constexpr int NBX = NB + 1;  // + a dummy packet for lanes past the end
  extern __shared__ __align__(128) unsigned char s_raw[];
  K* s_keys = reinterpret_cast<K*>(s_raw);                                    // TILE
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + TILE);             // TILE (pairs)
  uint32_t* s_wc = s_vals + (HAS_V ? TILE : 0);                              // NW * NBX warp counts
  uint32_t* s_tot = s_wc + NW * NBX;                                         // NB block totals
  uint32_t* s_bs = s_tot + ((NB + 1) & ~1);                                  // NB + 1 block packet starts
  unsigned long long* s_gb = reinterpret_cast<unsigned long long*>(s_bs + ((NB + 2) & ~1));  // NB
  uint16_t* s_pk = reinterpret_cast<uint16_t*>(s_gb + NB);                   // TILE packet ids
  __shared__ uint32_t s_ticket, s_fail;

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) {
    s_ticket = atomicAdd(&tb.counters[0], 1u);
    s_fail = 0;
  }
  for (int i = tid; i < NW * NBX; i += BLOCK) s_wc[i] = 0;
  __syncthreads();
  const uint32_t t = s_ticket;
  const uint32_t total = tb.blk_prefix[nseg];
  if (t >= total) return;
  const uint32_t seg = find_seg(tb.blk_prefix, nseg, t);
  const uint32_t first = tb.blk_prefix[seg];
  const uint64_t beg = tb.seg_off[seg] + static_cast<uint64_t>(t - first) * part_tile;
  const uint32_t cnt = static_cast<uint32_t>(min64(part_tile, tb.seg_off[seg + 1] - beg));
  const bool flip = tb.seg_flip[seg] != 0;
  const int cls = static_cast<int>(tb.seg_class[seg]);
  const DigitRule rule = (NB == 10) ? make_rule_dec(cls) : make_rule_bin(cls);

  // load (warp-striped) and compute packets
  K k[IPT];
  uint32_t v[IPT];
  uint32_t q[IPT];
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const uint32_t i = wid * kWarp * IPT + j * kWarp + lane;
    if (i < cnt) {
      k[j] = keys_in[beg + i];
      if constexpr (HAS_V) v[j] = vals_in[beg + i];
      q[j] = packet_of<NB>(KT<K>::image(k[j], flip), rule);
    } else {
      q[j] = NB;
    }
  }
  // warp ranking in input order
  uint32_t r[IPT];
  uint32_t* wc = s_wc + wid * NBX;
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const uint32_t peers = __match_any_sync(0xffffffffu, q[j]);
    const uint32_t base = wc[q[j]];
    r[j] = base + __popc(peers & lt_mask);
    __syncwarp();
    if (lane == __ffs(peers) - 1) wc[q[j]] = base + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per packet: block total, warp prefixes (in place in s_wc), block starts
  for (int p = tid; p < NB; p += BLOCK) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      uint32_t c = s_wc[w * NBX + p];
      s_wc[w * NBX + p] = run;
      run += c;
    }
    s_tot[p] = run;
  }
  __syncthreads();
  // look-back (thread p for packet p) + exclusive scan of block totals
  if (tid < NB) {
    const int p = tid;
    const uint32_t agg = s_tot[p];
    uint64_t* st = tb.status + static_cast<size_t>(t) * NB;
    const bool stuck = debug_stuck && (t == tb.blk_prefix[0] + 1);
    uint64_t excl = 0;
    if (t == first) {
      st_relaxed(&st[p], kFlagInc | agg);
    } else {
      if (!stuck) st_relaxed(&st[p], kFlagAgg | agg);
      int64_t pred = static_cast<int64_t>(t) - 1;
      uint64_t t0 = 0;
      uint64_t spins = 0;
      while (true) {
        const uint64_t w = ld_relaxed(tb.status + static_cast<size_t>(pred) * NB + p);
        const uint64_t f = w & ~kValMask;
        if (f == 0) {
          // two bounds: elapsed globaltimer time, and (should the timer not
          // advance) an iteration count of at least that many nanoseconds
          ++spins;
          if ((spins & 63) == 0) {
            const uint64_t now = globaltimer_ns();
            if (t0 == 0) t0 = now;
            if (now - t0 > limit_ns || spins > (limit_ns >> 4)) {
              s_fail = 1;
              break;
            }
          }
          __nanosleep(32);
          continue;
        }
        excl += w & kValMask;
        if (f == kFlagInc) break;
        --pred;
      }
      if (!stuck) st_relaxed(&st[p], kFlagInc | (excl + agg));
    }
    s_gb[p] = tb.pkt_off[static_cast<size_t>(seg) * NB + p] + excl;
  }
  if (tid == 0) {  // block packet starts: exclusive scan of the totals (s_tot stays intact)
    uint32_t run = 0;
    for (int p = 0; p < NB; ++p) {
      s_bs[p] = run;
      run += s_tot[p];
    }
    s_bs[NB] = run;
  }
  __syncthreads();
  if (s_fail) {
    if (tid == 0) atomicOr(tb.err, kErrTimeout);
    return;
  }
  // stage grouped by packet, in input order inside each packet
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    if (q[j] < NB) {
      const uint32_t pos = s_bs[q[j]] + s_wc[wid * NBX + q[j]] + r[j];
      s_keys[pos] = k[j];
      if constexpr (HAS_V) s_vals[pos] = v[j];
      s_pk[pos] = static_cast<uint16_t>(q[j]);
    }
  }
  __syncthreads();
  const uint64_t* pend = tb.pkt_off + static_cast<size_t>(seg) * NB + 1;
  for (uint32_t e = tid; e < cnt; e += BLOCK) {
    const uint32_t p = s_pk[e];
    const uint64_t dst = s_gb[p] + (e - s_bs[p]);
    if (dst >= pend[p]) {
      atomicOr(tb.err, kErrBounds);
      continue;
    }
    keys_out[dst] = s_keys[e];
    if constexpr (HAS_V) vals_out[dst] = s_vals[e];
  }
}

}  // namespace hs
