// Bottom-up merge passes at fan-in 4: every pass merges groups of four
// adjacent sorted runs, so a packet of T tiles needs ceil(log4 T) passes
// instead of ceil(log2 T).  Each pass still reads and writes every key once;
// the fan-in halves the number of passes over HBM.  The merge is stable: on
// equal keys the earlier run comes first, which is the order of the runs in
// the packet and therefore input order.
//
// Work split by samples.  Inside a group every run contributes a sample at
// each run-relative position m*S (m >= 1, S = TILE / (SPT * G)).  A sample's output
// position is its own position plus its rank in each other run (elements of
// earlier runs that are <= it, of later runs that are < it), and its index
// among the group's boundaries (the group start, then every sample in output
// order) follows from the same ranks: a run holds floor((rank - 1) / S)
// samples before it.  Every G-th boundary starts a merge chunk.  A chunk then
// takes at most (its samples + 1) * S items from each run, so at most
// (G + 4) * S items and on average G * S = TILE / SPT; the number of chunks of
// a group depends on the run lengths only and never exceeds SPT times the
// group's tiles, so chunk c of a group is recorded at slot SPT * (the group's
// first tile) + c.
//
//   k_bound4  one thread per sample slot: the ranks (three binary searches,
//             interleaved), the boundary index and, for every G-th boundary,
//             the chunk record; active chunks are listed densely.
//   k_merge4  persistent CTAs over the listed chunks: the four windows arrive
//             by bulk copy in one of two stages (the next chunk's while this
//             one is merged); two merge-path levels in shared memory (runs 0
//             and 1, runs 2 and 3 into T; then the two halves of T back into
//             the stage) and one bulk store.
#pragma once
#include "blockmerge.cuh"
#include "merge.cuh"

namespace hs {

struct Rec4 {
  uint64_t base;   // absolute index of the group's first item; bit 63: source buffer is W
  uint32_t run;    // run length of this pass
  uint32_t last;   // 1: the chunk ends at the group's end, else where chunk u + 1 starts
  uint32_t c[4];   // chunk start inside each run
  uint32_t len[4]; // lengths of the group's runs
};
static_assert(sizeof(Rec4) == 48, "record layout");

// Samples per merge chunk, chunk slots per tile, and the resulting sample
// spacing and chunk bound.
constexpr int kSamplesPerChunk = 8;
template <int TILE, int SPT>
__host__ __device__ constexpr int sample_gap() {
  return TILE / (SPT * kSamplesPerChunk);
}
template <int TILE, int SPT>
__host__ __device__ constexpr int chunk_max() {
  return (kSamplesPerChunk + 4) * sample_gap<TILE, SPT>();
}

// Samples of a run of `len` items strictly before run position `x` (x <= len),
// and the boundaries of a group: its start plus every sample.
template <int S>
__device__ __forceinline__ uint32_t samples_before(uint32_t x) {
  return x ? (x - 1) / S : 0u;
}

// Record of the chunk that starts at sample boundary q of a group (every G-th
// boundary): returns false (and sets kErrBounds) for a slot outside the packet,
// which the sample bound rules out.
template <int TILE, int SPT>
__device__ __forceinline__ bool bound4_record(uint32_t q, uint32_t up0, uint32_t ntiles, uint64_t pstart,
                                              uint64_t g0, uint64_t R, bool srcw, const uint32_t (&c)[4],
                                              const uint32_t (&lens)[4], Rec4* recs, uint32_t* err,
                                              uint32_t& u_out) {
  constexpr int G = kSamplesPerChunk;
  constexpr uint32_t S = sample_gap<TILE, SPT>();
  uint32_t nbound = 1;
#pragma unroll
  for (int j = 0; j < 4; ++j) nbound += samples_before<S>(lens[j]);
  const uint32_t chunk = q / G, chunks = (nbound + G - 1) / G;
  u_out = (up0 + static_cast<uint32_t>(g0 / TILE)) * SPT + chunk;
  if (chunk >= chunks || u_out >= (up0 + ntiles) * SPT) {  // cannot happen; never write out of the packet
    atomicOr(err, kErrBounds);
    return false;
  }
  Rec4 rec;
  rec.base = (pstart + g0) | (srcw ? kSrcW : 0ull);
  rec.run = static_cast<uint32_t>(R);
  rec.last = (chunk + 1 == chunks) ? 1u : 0u;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    rec.c[j] = c[j];
    rec.len[j] = lens[j];
  }
  recs[u_out] = rec;
  return true;
}

// k_bound4 with one warp per sample slot: lanes 8j .. 8j+7 find the sample's
// rank in run j together (the sample's own run is skipped); lane 0 writes the
// chunk record and lists it.
template <class K, int TILE, int SPT>
__device__ __forceinline__ void bound4_warp(const K* __restrict__ ku, const K* __restrict__ kw,
                                            Rec4* __restrict__ recs, uint32_t* __restrict__ list, uint32_t npk,
                                            int r, const Tables& tb, uint32_t total, int lane) {
  constexpr int G = kSamplesPerChunk;
  constexpr uint32_t S = sample_gap<TILE, SPT>();
  constexpr uint32_t PER_TILE = SPT * G;
  const int jr = lane >> 3, t = lane & 7;  // run searched by this lane, lane in its group
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t z = warp; z < total; z += nwarps) {  // warp-uniform: one sample slot per warp
    const uint32_t u = z / PER_TILE, sub = z % PER_TILE;
    const uint32_t p = find_pkt(tb.unit_prefix, npk, u);
    const uint32_t up0 = tb.unit_prefix[p], ntiles = tb.unit_prefix[p + 1] - up0;
    const int passes = passes_of(ntiles, 2);
    const uint64_t pstart = tb.pkt_off[p], len = tb.pkt_off[p + 1] - pstart;
    const uint64_t k = static_cast<uint64_t>(u - up0) * TILE + static_cast<uint64_t>(sub) * S;
    if (!(r <= passes && k < len)) continue;
    const uint64_t R = static_cast<uint64_t>(TILE) << (2 * (r - 1));
    const uint64_t g0 = k - k % (4 * R);
    const uint32_t i = static_cast<uint32_t>((k - g0) / R);
    const uint32_t pos = static_cast<uint32_t>((k - g0) % R);
    if (pos == 0 && i != 0) continue;  // neither a sample nor the group start
    uint32_t lens[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t st = g0 + static_cast<uint64_t>(j) * R;
      lens[j] = st >= len ? 0u : static_cast<uint32_t>(min(R, len - st));
    }
    const bool srcw = ((passes - r + 1) & 1) != 0;  // the buffer holding pass r-1
    const K* gb = (srcw ? kw : ku) + pstart + g0;
    uint32_t c[4] = {0, 0, 0, 0};
    uint32_t q = 0;
    if (pos != 0) {
      const K e = gb[static_cast<uint64_t>(i) * R + pos];
      const K* run = gb + static_cast<uint64_t>(jr) * R;
      const bool earlier = static_cast<uint32_t>(jr) < i;
      // items of run jr that come before e in the merged order
      uint32_t len_jr = lens[0];  // lens[jr] without a dynamically indexed array
#pragma unroll
      for (int j = 1; j < 4; ++j) len_jr = (jr == j) ? lens[j] : len_jr;
      const uint32_t hi = (static_cast<uint32_t>(jr) == i) ? 0u : len_jr;
      const uint32_t rank = group_search<8>(0u, hi, t, lane & ~7, [&](uint32_t m) {
        const K x = run[m];
        return earlier ? !(e < x) : (x < e);
      });
      q = pos / S;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t rj = __shfl_sync(0xffffffffu, rank, 8 * j);
        c[j] = (static_cast<uint32_t>(j) == i) ? pos : rj;
        if (static_cast<uint32_t>(j) != i) q += samples_before<S>(c[j]);
      }
    }
    if (lane == 0 && q % G == 0) {
      uint32_t u_out = 0;
      if (bound4_record<TILE, SPT>(q, up0, ntiles, pstart, g0, R, srcw, c, lens, recs, tb.err, u_out))
        list[atomicAdd(&tb.pass_ctl[r], 1u)] = u_out;
    }
  }
}

// LG == 1: one thread per sample slot, its three searches interleaved.
// LG == 8: one warp per sample slot, eight lanes per run (group_search), for
// passes with few samples, which are bound by the latency of the search chain.
template <class K, int TILE, int SPT, int LG>
__global__ void k_bound4(const K* __restrict__ ku, const K* __restrict__ kw, Rec4* __restrict__ recs,
                         uint32_t* __restrict__ list, uint32_t npk, int r, Tables tb) {
  griddep_open();
  constexpr int G = kSamplesPerChunk;
  constexpr uint32_t S = sample_gap<TILE, SPT>();
  constexpr uint32_t PER_TILE = SPT * G;  // sample slots per tile
  static_assert(S * PER_TILE == TILE, "whole chunk slots per tile");
  static_assert(LG == 1 || LG == 8, "a thread or a warp per sample");
  if (static_cast<uint32_t>(r) > tb.pass_ctl[0]) return;  // no packet needs pass r
  const uint32_t total = tb.unit_prefix[npk] * PER_TILE;
  const int lane = threadIdx.x & 31;
  if constexpr (LG == 8) {
    bound4_warp<K, TILE, SPT>(ku, kw, recs, list, npk, r, tb, total, lane);
    return;
  }
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total; base += stride) {
    const uint32_t z = base + lane;
    bool active = false;
    uint32_t u_out = 0;
    if (z < total) {
      const uint32_t u = z / PER_TILE, sub = z % PER_TILE;
      const uint32_t p = find_pkt(tb.unit_prefix, npk, u);
      const uint32_t up0 = tb.unit_prefix[p], ntiles = tb.unit_prefix[p + 1] - up0;
      const int passes = passes_of(ntiles, 2);
      const uint64_t pstart = tb.pkt_off[p], len = tb.pkt_off[p + 1] - pstart;
      const uint64_t k = static_cast<uint64_t>(u - up0) * TILE + static_cast<uint64_t>(sub) * S;
      if (r <= passes && k < len) {
        const uint64_t R = static_cast<uint64_t>(TILE) << (2 * (r - 1));
        const uint64_t g0 = k - k % (4 * R);
        const uint32_t i = static_cast<uint32_t>((k - g0) / R);
        const uint32_t pos = static_cast<uint32_t>((k - g0) % R);
        uint32_t lens[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint64_t st = g0 + static_cast<uint64_t>(j) * R;
          lens[j] = st >= len ? 0u : static_cast<uint32_t>(min(R, len - st));
        }
        if (pos != 0 || i == 0) {  // a sample, or the group start
          const bool srcw = ((passes - r + 1) & 1) != 0;  // the buffer holding pass r-1
          const K* gb = (srcw ? kw : ku) + pstart + g0;
          uint32_t c[4] = {0, 0, 0, 0};
          uint32_t q = 0;
          if (pos != 0) {
            const K e = gb[static_cast<uint64_t>(i) * R + pos];
            uint32_t lo[4], hi[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              lo[j] = 0;
              hi[j] = (static_cast<uint32_t>(j) == i) ? 0u : lens[j];
            }
            // three binary searches, interleaved: items of run j that come
            // before e in the merged order
            while (lo[0] < hi[0] || lo[1] < hi[1] || lo[2] < hi[2] || lo[3] < hi[3]) {
              bool before[4];
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                before[j] = false;
                if (lo[j] < hi[j]) {
                  const uint32_t m = (lo[j] + hi[j]) >> 1;
                  const K x = gb[static_cast<uint64_t>(j) * R + m];
                  before[j] = (static_cast<uint32_t>(j) < i) ? !(e < x) : (x < e);
                }
              }
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                if (lo[j] < hi[j]) {
                  const uint32_t m = (lo[j] + hi[j]) >> 1;
                  if (before[j]) lo[j] = m + 1; else hi[j] = m;
                }
              }
            }
            q = pos / S;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              c[j] = (static_cast<uint32_t>(j) == i) ? pos : lo[j];
              if (static_cast<uint32_t>(j) != i) q += samples_before<S>(c[j]);
            }
          }
          if (q % G == 0)
            active = bound4_record<TILE, SPT>(q, up0, ntiles, pstart, g0, R, srcw, c, lens, recs, tb.err, u_out);
        }
      }
    }
    const uint32_t mask = __ballot_sync(0xffffffffu, active);
    if (mask) {
      uint32_t slot = 0;
      if (lane == __ffs(mask) - 1) slot = atomicAdd(&tb.pass_ctl[r], __popc(mask));
      slot = __shfl_sync(0xffffffffu, slot, __ffs(mask) - 1);
      if (active) list[slot + __popc(mask & ((1u << lane) - 1u))] = u_out;
    }
  }
}

// One chunk as the merge kernel uses it.
struct Chunk4 {
  uint64_t base;  // absolute index of the group's first item (bit 63: source W)
  uint32_t run;
  uint32_t c[4];  // window starts inside the runs
  uint32_t l[4];  // window lengths
};

__device__ __forceinline__ Chunk4 empty_chunk4();

// Chunk at unit u.  A chunk that would not fit the shared buffers or leave
// its runs (which the sample bound rules out) sets kErrBounds and is treated
// as empty, so no copy ever runs outside its buffer.
template <int CMAX>
__device__ __forceinline__ Chunk4 load_chunk4(const Rec4* recs, uint32_t u, uint32_t* err) {
  const Rec4 a = recs[u];
  Chunk4 ch;
  ch.base = a.base;
  ch.run = a.run;
  uint32_t e[4];
  if (a.last) {
#pragma unroll
    for (int j = 0; j < 4; ++j) e[j] = a.len[j];
  } else {
    const uint4 nx = *reinterpret_cast<const uint4*>(&recs[u + 1].c[0]);
    e[0] = nx.x;
    e[1] = nx.y;
    e[2] = nx.z;
    e[3] = nx.w;
  }
  bool bad = false;
  uint32_t cnt = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    ch.c[j] = a.c[j];
    ch.l[j] = e[j] - a.c[j];
    bad |= e[j] < a.c[j] || e[j] > a.len[j] || a.len[j] > a.run;
    cnt += ch.l[j];
  }
  if (bad || cnt > static_cast<uint32_t>(CMAX)) {
    if (threadIdx.x == 0) atomicOr(err, kErrBounds);
    return empty_chunk4();
  }
  return ch;
}

__device__ __forceinline__ Chunk4 empty_chunk4() {
  Chunk4 ch;
  ch.base = 0;
  ch.run = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    ch.c[j] = 0;
    ch.l[j] = 0;
  }
  return ch;
}

// Placement of the four windows of a chunk in one shared region: window j at
// the first index at or after the end of window j - 1 with its own 16-byte
// phase, window 0 at its phase.
template <class T>
__device__ __forceinline__ void place4(const T* src, const Chunk4& ch, uint32_t (&pl)[4]) {
  constexpr uint32_t PER = 16 / sizeof(T);
  uint32_t x = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const T* g = src + static_cast<uint64_t>(j) * ch.run + ch.c[j];
    x += (phase_of(g) - x) & (PER - 1);
    pl[j] = x;
    x += ch.l[j];
  }
}

template <class K, bool HAS_V>
__device__ __forceinline__ void merge4_issue(const Chunk4& ch, K* rk, uint32_t* rv, uint64_t* bar, const K* ku,
                                             const uint32_t* vu, const K* kw, const uint32_t* vw, int lane) {
  const bool srcw = (ch.base & kSrcW) != 0;
  const uint64_t b = ch.base & ~kSrcW;
  const K* ks = (srcw ? kw : ku) + b;
  uint32_t pk[4];
  place4(ks, ch, pk);
  PendingBulk<K> bk[4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
    bk[j] = load_window_singles(rk, pk[j], ks + static_cast<uint64_t>(j) * ch.run + ch.c[j], ch.l[j], lane);
  PendingBulk<uint32_t> bv[4];
  if constexpr (HAS_V) {
    const uint32_t* vs = (srcw ? vw : vu) + b;
    uint32_t pv[4];
    place4(vs, ch, pv);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      bv[j] = load_window_singles(rv, pv[j], vs + static_cast<uint64_t>(j) * ch.run + ch.c[j], ch.l[j], lane);
  }
  cp_async_mbar_arrive(bar);
  __syncwarp();
  if (lane == 0) {
    uint32_t bytes = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) bytes += bk[j].bytes + (HAS_V ? bv[j].bytes : 0u);
    mbar_arrive_expect_tx(bar, bytes);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (bk[j].bytes) bulk_g2s(bk[j].sdst, bk[j].gsrc, bk[j].bytes, bar);
      if constexpr (HAS_V) {
        if (bv[j].bytes) bulk_g2s(bv[j].sdst, bv[j].gsrc, bv[j].bytes, bar);
      }
    }
  }
}

// Outputs [d0, d1) of the stable merge of A[0, la) and B[0, lb) into O[d]
// (and values into Ov[d]).  Reads at most one element past either input,
// which the buffer layout keeps inside shared memory (never selected).
template <class K, bool HAS_V>
__device__ __forceinline__ void merge_span(const K* A, const uint32_t* Av, int la, const K* B, const uint32_t* Bv,
                                           int lb, int d0, int d1, K* O, uint32_t* Ov) {
  if (d0 >= d1) return;
  int i = corank_smem(A, la, B, lb, d0);
  int j = d0 - i;
  K ka = A[i], kb = B[j];
#pragma unroll 4
  for (int d = d0; d < d1; ++d) {
    const bool p = (j >= lb) || ((i < la) && !(kb < ka));
    O[d] = p ? ka : kb;
    if constexpr (HAS_V) Ov[d] = p ? Av[i] : Bv[j];
    i += p ? 1 : 0;
    j += p ? 0 : 1;
    const K nv = p ? A[i] : B[j];
    ka = p ? nv : ka;
    kb = p ? kb : nv;
  }
}

// Shared memory of k_merge4: two stages (keys, then values) and T.
template <class K, bool HAS_V, int CMAX>
__host__ __device__ constexpr size_t merge4_region_bytes() {
  return ((static_cast<size_t>(CMAX) + 16) * sizeof(K) + 127) & ~size_t(127);
}
template <class K, bool HAS_V, int CMAX>
__host__ __device__ constexpr size_t merge4_vregion_bytes() {
  return HAS_V ? ((static_cast<size_t>(CMAX) + 16) * 4 + 127) & ~size_t(127) : 0;
}
template <class K, bool HAS_V, int CMAX>
__host__ __device__ constexpr size_t merge4_buffer_bytes() {
  return merge4_region_bytes<K, HAS_V, CMAX>() + merge4_vregion_bytes<K, HAS_V, CMAX>();
}
template <class K, bool HAS_V, int CMAX>
__host__ __device__ constexpr size_t merge4_smem() {
  return 3 * merge4_buffer_bytes<K, HAS_V, CMAX>();
}

template <class K, bool HAS_V, int BLOCK, int MINB, int CMAX>
__global__ void __launch_bounds__(BLOCK, MINB) k_merge4(K* ku, uint32_t* vu, K* kw, uint32_t* vw,
                                                         const Rec4* __restrict__ recs,
                                                         const uint32_t* __restrict__ list, int r, Tables tb) {
  griddep_open();
  constexpr size_t KB = merge4_region_bytes<K, HAS_V, CMAX>();
  constexpr size_t SB = merge4_buffer_bytes<K, HAS_V, CMAX>();
  extern __shared__ __align__(128) unsigned char s_raw[];
  __shared__ __align__(8) uint64_t s_bar[2];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t total = tb.pass_ctl[r];  // active chunks, listed by k_bound4
  const uint32_t G = gridDim.x;
  uint32_t u = blockIdx.x;
  if (u >= total) return;
  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
  }
  mbar_fence_init();
  __syncthreads();
  K* tk = reinterpret_cast<K*>(s_raw + 2 * SB);
  uint32_t* tv = reinterpret_cast<uint32_t*>(s_raw + 2 * SB + KB);

  Chunk4 cur = load_chunk4<CMAX>(recs, list[u], tb.err);
  Chunk4 nxt = (u + G < total) ? load_chunk4<CMAX>(recs, list[u + G], tb.err) : empty_chunk4();
  if (wid == 0)
    merge4_issue<K, HAS_V>(cur, reinterpret_cast<K*>(s_raw), reinterpret_cast<uint32_t*>(s_raw + KB), &s_bar[0], ku,
                           vu, kw, vw, lane);
  uint32_t par0 = 0, par1 = 0;
  int s = 0;
  bool failed = false;
  for (; u < total; u += G) {
    const Chunk4 nn = (u + 2 * G < total) ? load_chunk4<CMAX>(recs, list[u + 2 * G], tb.err) : empty_chunk4();
    unsigned char* st_cur = s_raw + s * SB;
    unsigned char* st_nxt = s_raw + (s ^ 1) * SB;
    if (wid == 0) {
      if (lane == 0) {
        bulk_wait_read0();  // the store staged in the other stage has read it
        fence_proxy_async();
      }
      __syncwarp();
      merge4_issue<K, HAS_V>(nxt, reinterpret_cast<K*>(st_nxt), reinterpret_cast<uint32_t*>(st_nxt + KB),
                             &s_bar[s ^ 1], ku, vu, kw, vw, lane);
    }
    const bool ok = mbar_wait_bounded(&s_bar[s], s ? par1 : par0, tb.err, kWaitNs);
    if (s) par1 ^= 1; else par0 ^= 1;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    K* rk = reinterpret_cast<K*>(st_cur);
    uint32_t* rv = reinterpret_cast<uint32_t*>(st_cur + KB);
    const bool srcw = (cur.base & kSrcW) != 0;
    const uint64_t gbase = cur.base & ~kSrcW;
    uint32_t pk[4], pv[4] = {0, 0, 0, 0};
    place4((srcw ? kw : ku) + gbase, cur, pk);
    if constexpr (HAS_V) place4((srcw ? vw : vu) + gbase, cur, pv);
    const int l0 = static_cast<int>(cur.l[0]), l1 = static_cast<int>(cur.l[1]);
    const int l2 = static_cast<int>(cur.l[2]), l3 = static_cast<int>(cur.l[3]);
    const int l01 = l0 + l1, cnt = l01 + l2 + l3;
    const int d0 = (tid * cnt) / BLOCK, d1 = ((tid + 1) * cnt) / BLOCK;
    // level 1: runs 0 and 1 into T[0, l01), runs 2 and 3 into T[l01, cnt)
    if (d0 < l01)
      merge_span<K, HAS_V>(rk + pk[0], rv + pv[0], l0, rk + pk[1], rv + pv[1], l1, d0, min(d1, l01), tk, tv);
    if (d1 > l01)
      merge_span<K, HAS_V>(rk + pk[2], rv + pv[2], l2, rk + pk[3], rv + pv[3], l3, max(d0, l01) - l01, d1 - l01,
                           tk + l01, tv + l01);
    __syncthreads();  // T complete; every read of the stage is done
    // level 2: the two halves of T into the stage, at the destination's phase
    K* kd = (srcw ? ku : kw) + gbase + cur.c[0] + cur.c[1] + cur.c[2] + cur.c[3];
    uint32_t* vd = HAS_V ? (srcw ? vu : vw) + gbase + cur.c[0] + cur.c[1] + cur.c[2] + cur.c[3] : nullptr;
    const uint32_t ok_ph = phase_of(kd);
    const uint32_t ov_ph = HAS_V ? phase_of(vd) : 0u;
    merge_span<K, HAS_V>(tk, tv, l01, tk + l01, tv + l01, cnt - l01, d0, d1, rk + ok_ph, rv + ov_ph);
    fence_proxy_async();
    __syncthreads();
    if (wid == 0 && cnt > 0) {
      store_window(kd, rk + ok_ph, static_cast<uint32_t>(cnt), lane);
      if constexpr (HAS_V) store_window(vd, rv + ov_ph, static_cast<uint32_t>(cnt), lane);
      if (lane == 0) bulk_commit();
    }
    cur = nxt;
    nxt = nn;
    s ^= 1;
  }
  if (failed) {
    // copies into the other stage may still be in flight: give them a
    // bounded chance to land before the CTA's shared memory is released
    mbar_wait_bounded(&s_bar[s ^ 1], s ? par0 : par1, tb.err, kWaitNs);
  }
  if (tid == 0) bulk_wait0();
}

}  // namespace hs
