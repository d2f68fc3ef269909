// Per-packet sort (Sec. 3.2, Fig. 1) on the GPU:
//   k_tilesort  every packet is cut into tiles of TILE = BLOCK * IPT keys that
//               start at the packet's first key (the last tile of a packet may
//               be short); one CTA sorts one tile: a sorting network per thread
//               over its IPT keys in registers, then log2(BLOCK) merge-path
//               merges in shared memory.  This replaces the paper's per-thread
//               sequential quicksort of one data part.
//   k_corank    merge pass r, for every merge block (TILE outputs) the split of
//               its first and one-past-last output between the two runs it
//               merges (merge path: binary search along the cross diagonal).
//   k_merge     merge pass r: one CTA writes TILE consecutive outputs of one
//               pair of runs of length TILE * 2^(r-1); runs never cross a packet
//               boundary.  Passes repeat until every packet is one run: the
//               non-recursive, bottom-up merge of Fig. 1(b) and Sec. 3.2, with
//               every CTA merging an equal share instead of one thread per pair
//               of lists.
//
// Data movement: tiles and merge windows are contiguous, so they move with the
// bulk-copy engine (TMA): one lane issues the 16-byte-aligned interior of each
// window as one bulk copy and the at most three unaligned elements at each end
// as tracked cp.async copies; an mbarrier completes when all have landed.
// Results leave the same way (bulk store of the aligned interior).
//
// Shared-memory layout: IPT is odd (15), so thread t's blocked items
// t*IPT .. t*IPT+IPT-1 fall in 32 distinct banks across a warp without padding.
//
// Buffers: the packet step writes the work buffer W.  A packet needing P
// merge passes has its tiles sorted into U (the caller's array) when P is
// even, into W when P is odd, and every pass flips between them, so its last
// pass lands in U; packets finished early take no part in later passes.
//
// Stability: merges take the left run on equal keys.  The tile sort of pairs
// orders each thread's items with odd-even transposition (swaps only strictly
// greater neighbours), so equal keys keep their order from the packet step,
// which keeps input order.
#pragma once
#include <utility>

#include "async.cuh"
#include "common.cuh"

namespace hs {

// last p with pre[p] <= u, p in [0, npk)
__device__ __forceinline__ uint32_t find_pkt(const uint32_t* __restrict__ pre, uint32_t npk, uint32_t u) {
  uint32_t lo = 0, hi = npk;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (pre[mid] <= u) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int ceil_log2(uint32_t x) { return x <= 1 ? 0 : 32 - __clz(x - 1); }

// Shared-memory elements of one window region: TILE items plus room for the
// 16-byte phase of two windows placed back to back (and one read past the end).
__host__ __device__ constexpr int region_elems(int tile) { return tile + 8; }

// Geometry of merge block u in pass r (r >= 1) of its packet.
struct MergeGeom {
  uint64_t pstart;   // packet start (absolute)
  uint64_t a_start;  // first run of the pair, packet-relative
  uint32_t a_len, b_len;
  uint32_t diag0;    // first output of this block inside the pair
  uint32_t cnt;      // outputs of this block
  int passes;        // merge passes the packet needs
};

template <int TILE>
__device__ __forceinline__ bool merge_geom(const Tables& tb, uint32_t npk, uint32_t u, int r, MergeGeom& g) {
  const uint32_t p = find_pkt(tb.unit_prefix, npk, u);
  const uint32_t up0 = tb.unit_prefix[p], ntiles = tb.unit_prefix[p + 1] - up0;
  g.passes = ceil_log2(ntiles);
  if (r > g.passes) return false;
  g.pstart = tb.pkt_off[p];
  const uint64_t len = tb.pkt_off[p + 1] - g.pstart;
  const uint64_t R = static_cast<uint64_t>(TILE) << (r - 1);
  const uint64_t k0 = static_cast<uint64_t>(u - up0) * TILE;
  g.a_start = (k0 / (2 * R)) * (2 * R);
  const uint64_t rest = len - g.a_start;
  g.a_len = static_cast<uint32_t>(min(R, rest));
  g.b_len = static_cast<uint32_t>(rest > R ? min(R, rest - R) : 0);
  g.diag0 = static_cast<uint32_t>(k0 - g.a_start);
  g.cnt = static_cast<uint32_t>(min64(TILE, len - k0));
  return true;
}

// ---------------------------------------------------------------------------
// In-register sorting networks over N items.
// ---------------------------------------------------------------------------
template <class K>
__device__ __forceinline__ void cas_keys(K& a, K& b) {
  const K lo = min(a, b), hi = max(a, b);
  a = lo;
  b = hi;
}

// Batcher's odd-even merge sort network over M = 16 or 32 slots: the
// comparators are listed at compile time and expanded by a fold expression,
// so every register index is a constant.  N <= M keys are sorted; unused
// slots hold the largest key and their comparators fold away.  Keys only:
// not stable, which does not matter for keys alone.
struct Comparator {
  int a, b;
};
template <int M>
struct BatcherList {
  Comparator c[M == 16 ? 63 : 191];
};
template <int M>
constexpr int batcher_count() {
  return M == 16 ? 63 : 191;
}
template <int M>
constexpr BatcherList<M> make_batcher() {
  BatcherList<M> l{};
  int n = 0;
  for (int p = 1; p < M; p <<= 1)
    for (int kk = p; kk >= 1; kk >>= 1)
      for (int j = kk % p; j + kk < M; j += 2 * kk)
        for (int i = 0; i < kk; ++i)
          if ((i + j) / (2 * p) == (i + j + kk) / (2 * p)) l.c[n++] = Comparator{i + j, i + j + kk};
  return l;
}
template <int M>
struct Batcher {
  static constexpr BatcherList<M> list = make_batcher<M>();
};
static_assert(Batcher<16>::list.c[62].b != 0 && Batcher<32>::list.c[190].b != 0, "comparator counts");

template <int M, class K, int... I>
__device__ __forceinline__ void apply_batcher(K (&t)[M], std::integer_sequence<int, I...>) {
  (cas_keys(t[Batcher<M>::list.c[I].a], t[Batcher<M>::list.c[I].b]), ...);
}
template <int N, class K>
__device__ __forceinline__ void network_sort(K (&k)[N]) {
  static_assert(N <= 32, "network over at most 32 keys");
  constexpr int M = N <= 16 ? 16 : 32;
  K t[M];
#pragma unroll
  for (int i = 0; i < M; ++i) t[i] = (i < N) ? k[i] : KT<K>::maxv();
  apply_batcher<M>(t, std::make_integer_sequence<int, batcher_count<M>()>{});
#pragma unroll
  for (int i = 0; i < N; ++i) k[i] = t[i];
}

// Odd-even transposition sort: N rounds of neighbour compare-exchanges that
// swap only when the right key is strictly smaller, so equal keys keep order.
template <int N, class K>
__device__ __forceinline__ void transposition_sort(K (&k)[N], uint32_t (&v)[N]) {
#pragma unroll
  for (int r = 0; r < N; ++r) {
#pragma unroll
    for (int i = r & 1; i + 1 < N; i += 2) {
      const bool sw = k[i + 1] < k[i];
      const K a = k[i], b = k[i + 1];
      const uint32_t va = v[i], vb = v[i + 1];
      k[i] = sw ? b : a;
      k[i + 1] = sw ? a : b;
      v[i] = sw ? vb : va;
      v[i + 1] = sw ? va : vb;
    }
  }
}

// Merge path inside shared memory: number of A items among the first `diag`
// outputs of merging A[0, la) and B[0, lb), A first on equal keys.
template <class K>
__device__ __forceinline__ int corank_smem(const K* sA, int la, const K* sB, int lb, int diag) {
  int lo = diag > lb ? diag - lb : 0;
  int hi = diag < la ? diag : la;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (!(sB[diag - 1 - mid] < sA[mid])) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Serial merge of IPT outputs starting at A[ai], B[bi] (A first on ties).
// Reads one element past the end of either side, which the region layout
// keeps inside shared memory (the value read is never selected).
// src[j]: index of output j, with bit 16 set when it came from B.
template <class K, int IPT, bool FULL, bool TRACK>
__device__ __forceinline__ void serial_merge(const K* sA, int ai, int la, const K* sB, int bi, int lb, int nout,
                                             K (&out)[IPT], int (&src)[IPT]) {
  K ka = sA[ai];
  K kb = sB[bi];
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    if (FULL || j < nout) {
      const bool p = (bi >= lb) || ((ai < la) && !(kb < ka));
      out[j] = p ? ka : kb;
      if (TRACK) src[j] = p ? ai : (bi | 0x10000);
      const int na = ai + (p ? 1 : 0), nb = bi + (p ? 0 : 1);
      const K nv = p ? sA[na] : sB[nb];
      ka = p ? nv : ka;
      kb = p ? kb : nv;
      ai = na;
      bi = nb;
    }
  }
}

// ---------------------------------------------------------------------------
// Window transfers (issued by warp 0 of a CTA).
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ uint32_t phase_of(const T* g) {
  return static_cast<uint32_t>((reinterpret_cast<uintptr_t>(g) & 15u) / sizeof(T));
}

// Shared placement of two windows A (la items at ga) and B (at gb) in one
// region: A at pa (its 16-byte phase), B at the first index >= pa + la with
// B's phase.
template <class T>
__device__ __forceinline__ void place2(const T* ga, uint32_t la, const T* gb, uint32_t& pa, uint32_t& pb) {
  constexpr uint32_t PER = 16 / sizeof(T);
  pa = phase_of(ga);
  pb = pa + la;
  pb += (phase_of(gb) - pb) & (PER - 1);
}

// Load window [g, g + cnt) to region + phase_at.  Called by all 32 lanes of
// one warp: the unaligned head and tail elements go by cp.async now; the
// aligned interior is returned for lane 0 to issue as one bulk copy once
// every lane has registered its cp.async copies on the barrier.
template <class T>
struct PendingBulk {
  T* sdst;
  const T* gsrc;
  uint32_t bytes;
};
template <class T>
__device__ __forceinline__ PendingBulk<T> load_window_singles(T* region, uint32_t phase_at, const T* g, uint32_t cnt,
                                                              int lane) {
  const Window w = plan_window<sizeof(T)>(g, cnt);
  T* s = region + phase_at;
  const uint32_t nsingle = w.head + w.tail;
  for (uint32_t i = lane; i < nsingle; i += 32) {
    const uint32_t e = (i < w.head) ? i : cnt - w.tail + (i - w.head);
    cp_async_elem<sizeof(T)>(s + e, g + e);
  }
  return PendingBulk<T>{s + w.head, g + w.head, w.body_bytes};
}

// Store [s, s + cnt) (shared, placed at the 16-byte phase of g) to global g.
// Called by all lanes of one warp after a proxy fence and a CTA barrier.
template <class T>
__device__ __forceinline__ void store_window(T* g, const T* s, uint32_t cnt, int lane) {
  const Window w = plan_window<sizeof(T)>(g, cnt);
  const uint32_t nsingle = w.head + w.tail;
  for (uint32_t i = lane; i < nsingle; i += 32) {
    const uint32_t e = (i < w.head) ? i : cnt - w.tail + (i - w.head);
    g[e] = s[e];
  }
  if (lane == 0 && w.body_bytes) bulk_s2g(g + w.head, s + w.head, w.body_bytes);
}

constexpr uint64_t kWaitNs = 2000000000ull;  // bounded waits on copies: 2 s

// ---------------------------------------------------------------------------
// k_tilesort
// ---------------------------------------------------------------------------
template <class K, bool HAS_V, int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK) k_tilesort(const K* __restrict__ kw, const uint32_t* __restrict__ vw, K* ku,
                                                     uint32_t* vu, K* kw_out, uint32_t* vw_out, uint32_t npk,
                                                     int force_w, int debug_stuck, uint64_t limit_ns, Tables tb) {
  constexpr int TILE = BLOCK * IPT;
  constexpr int RE = region_elems(TILE);
  extern __shared__ __align__(128) unsigned char s_raw[];
  K* rk = reinterpret_cast<K*>(s_raw);
  uint32_t* rv = reinterpret_cast<uint32_t*>(s_raw + ((RE * sizeof(K) + 127) & ~size_t(127)));
  __shared__ __align__(8) uint64_t s_bar;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t total = tb.unit_prefix[npk];
  if (tid == 0) mbar_init(&s_bar, 1);
  mbar_fence_init();
  __syncthreads();
  uint32_t parity = 0;
  bool failed = false;

  for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {
    const uint32_t p = find_pkt(tb.unit_prefix, npk, u);
    const uint32_t up0 = tb.unit_prefix[p], ntiles = tb.unit_prefix[p + 1] - up0;
    const int passes = ceil_log2(ntiles);
    const bool to_w = force_w || (passes & 1);
    const uint64_t beg = tb.pkt_off[p] + static_cast<uint64_t>(u - up0) * TILE;
    const int cnt = static_cast<int>(min64(TILE, tb.pkt_off[p + 1] - beg));
    const K* gk = kw + beg;
    const uint32_t* gv = HAS_V ? vw + beg : nullptr;
    const uint32_t pk = phase_of(gk);
    const uint32_t pv = HAS_V ? phase_of(gv) : 0u;

    if (wid == 0) {  // the tile's keys (and values) into the region at their phase
      if (lane == 0) {
        bulk_wait_read0();  // the previous tile's bulk store has read the region
        fence_proxy_async();
      }
      __syncwarp();
      const PendingBulk<K> bk = load_window_singles(rk, pk, gk, cnt, lane);
      PendingBulk<uint32_t> bv{nullptr, nullptr, 0};
      if constexpr (HAS_V) bv = load_window_singles(rv, pv, gv, cnt, lane);
      cp_async_mbar_arrive(&s_bar);
      __syncwarp();
      if (lane == 0) {
        // testing hook: CTA 0 announces 16 bytes that never arrive on its
        // first tile, so its bounded wait expires
        const uint32_t extra = (debug_stuck && blockIdx.x == 0 && u == blockIdx.x) ? 16u : 0u;
        mbar_arrive_expect_tx(&s_bar, bk.bytes + bv.bytes + extra);
        if (bk.bytes) bulk_g2s(bk.sdst, bk.gsrc, bk.bytes, &s_bar);
        if (HAS_V && bv.bytes) bulk_g2s(bv.sdst, bv.gsrc, bv.bytes, &s_bar);
      }
    }
    const bool ok = mbar_wait_bounded(&s_bar, parity, tb.err, limit_ns);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    parity ^= 1;

    K k[IPT];
    uint32_t v[IPT];
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const int i = tid * IPT + j;
      k[j] = (i < cnt) ? rk[pk + i] : KT<K>::maxv();
      if constexpr (HAS_V) v[j] = (i < cnt) ? rv[pv + i] : 0u;
    }
    if constexpr (HAS_V) transposition_sort<IPT>(k, v);
    else network_sort<IPT>(k);

    // merge levels: runs of `run` items -> 2 * run, in the region at offset 0
#pragma unroll 1
    for (int run = IPT; run < TILE; run <<= 1) {
      __syncthreads();
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        rk[tid * IPT + j] = k[j];
        if constexpr (HAS_V) rv[tid * IPT + j] = v[j];
      }
      __syncthreads();
      const int tpg = (2 * run) / IPT;
      const int a0 = (tid / tpg) * 2 * run;
      const int diag = (tid % tpg) * IPT;
      const K* sA = rk + a0;
      const K* sB = rk + a0 + run;
      const int i = corank_smem(sA, run, sB, run, diag);
      int src[IPT];
      serial_merge<K, IPT, true, HAS_V>(sA, i, run, sB, diag - i, run, IPT, k, src);
      if constexpr (HAS_V) {
#pragma unroll
        for (int j = 0; j < IPT; ++j) v[j] = (src[j] & 0x10000) ? rv[a0 + run + (src[j] & 0xffff)] : rv[a0 + src[j]];
      }
    }
    // blocked registers -> region at the destination's phase -> bulk store
    K* kd = (to_w ? kw_out : ku) + beg;
    uint32_t* vd = HAS_V ? (to_w ? vw_out : vu) + beg : nullptr;
    const uint32_t ok_ph = phase_of(kd);
    const uint32_t ov_ph = HAS_V ? phase_of(vd) : 0u;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const int i = tid * IPT + j;
      if (i < cnt) {
        rk[ok_ph + i] = k[j];
        if constexpr (HAS_V) rv[ov_ph + i] = v[j];
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (wid == 0) {
      store_window(kd, rk + ok_ph, cnt, lane);
      if constexpr (HAS_V) store_window(vd, rv + ov_ph, cnt, lane);
      if (lane == 0) bulk_commit();
    }
  }
  // a copy may still be in flight into the region: give it a bounded chance
  // to land before the CTA's shared memory is released
  if (failed) mbar_wait_bounded(&s_bar, parity, tb.err, limit_ns);
  if (tid == 0) bulk_wait0();
}

// ---------------------------------------------------------------------------
// Merge pass r, step 1 -- k_corank: for every merge block, the split of its
// first and of its one-past-last output between the two runs it merges (the
// merge path co-ranks), packed into a record the merge kernel reads once.
// ---------------------------------------------------------------------------
struct MergeRec {
  uint64_t a;    // absolute index of the block's first A item; bit 63: source buffer is W
  uint64_t b;    // absolute index of the block's first B item
  uint64_t out;  // absolute index of the block's first output
  uint32_t la;   // A items merged by the block
  uint32_t lb;   // B items merged by the block (la + lb = outputs; 0 = nothing to do)
};
constexpr uint64_t kSrcW = 1ull << 63;

// Number of A items among the first `diag` outputs of merging A[0, la) and
// B[0, lb) with A first on ties, for two diagonals at once (two independent
// binary searches interleaved so their loads overlap).
template <class K>
__device__ __forceinline__ void corank2(const K* __restrict__ A, uint32_t la, const K* __restrict__ B, uint32_t lb,
                                        uint32_t d0, uint32_t d1, uint32_t& r0, uint32_t& r1) {
  uint32_t lo0 = d0 > lb ? d0 - lb : 0, hi0 = min(d0, la);
  uint32_t lo1 = d1 > lb ? d1 - lb : 0, hi1 = min(d1, la);
  while (lo0 < hi0 || lo1 < hi1) {
    const uint32_t m0 = (lo0 + hi0) >> 1, m1 = (lo1 + hi1) >> 1;
    bool g0 = false, g1 = false;
    if (lo0 < hi0) g0 = !(B[d0 - 1 - m0] < A[m0]);
    if (lo1 < hi1) g1 = !(B[d1 - 1 - m1] < A[m1]);
    if (lo0 < hi0) {
      if (g0) lo0 = m0 + 1; else hi0 = m0;
    }
    if (lo1 < hi1) {
      if (g1) lo1 = m1 + 1; else hi1 = m1;
    }
  }
  r0 = lo0;
  r1 = lo1;
}

template <class K, int TILE>
__global__ void k_corank(const K* __restrict__ ku, const K* __restrict__ kw, MergeRec* __restrict__ recs,
                         uint32_t npk, int r, Tables tb) {
  const uint32_t total = tb.unit_prefix[npk];
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x) {
    MergeGeom g;
    MergeRec rec{0, 0, 0, 0, 0};
    if (merge_geom<TILE>(tb, npk, u, r, g)) {
      const bool srcw = ((g.passes - r + 1) & 1) != 0;  // the buffer holding pass r-1
      const K* A = (srcw ? kw : ku) + g.pstart + g.a_start;
      const K* B = A + g.a_len;
      uint32_t i0, i1;
      corank2(A, g.a_len, B, g.b_len, g.diag0, g.diag0 + g.cnt, i0, i1);
      const uint64_t abs_a = g.pstart + g.a_start;
      rec.a = (abs_a + i0) | (srcw ? kSrcW : 0ull);
      rec.b = abs_a + g.a_len + (g.diag0 - i0);
      rec.out = abs_a + g.diag0;
      rec.la = i1 - i0;
      rec.lb = g.cnt - rec.la;
    }
    recs[u] = rec;
  }
}

// ---------------------------------------------------------------------------
// Merge pass r, step 2 -- k_merge: persistent CTAs; each walks merge blocks
// blockIdx.x, +gridDim.x, ...  Two input stages: while block k is merged out
// of one, warp 0 has the bulk-copy engine fill the other with block k+1's A
// and B windows; block k+2's record is fetched one block ahead.  The merged
// block is staged in one of two output buffers and leaves by bulk store; the
// previous block's store has a whole block's time to read the other buffer,
// so the outputs can be staged without waiting for the inputs to be released.
// ---------------------------------------------------------------------------
template <class K, bool HAS_V>
__device__ __forceinline__ void merge_issue(const MergeRec& rec, K* rk, uint32_t* rv, uint64_t* bar, const K* ku,
                                            const uint32_t* vu, const K* kw, const uint32_t* vw, int lane) {
  const bool srcw = (rec.a & kSrcW) != 0;
  const uint64_t a = rec.a & ~kSrcW;
  const K* ks = srcw ? kw : ku;
  uint32_t pa, pb;
  place2(ks + a, rec.la, ks + rec.b, pa, pb);
  const PendingBulk<K> ba = load_window_singles(rk, pa, ks + a, rec.la, lane);
  const PendingBulk<K> bb = load_window_singles(rk, pb, ks + rec.b, rec.lb, lane);
  PendingBulk<uint32_t> va{nullptr, nullptr, 0}, vb{nullptr, nullptr, 0};
  if constexpr (HAS_V) {
    const uint32_t* vs = srcw ? vw : vu;
    uint32_t qa, qb;
    place2(vs + a, rec.la, vs + rec.b, qa, qb);
    va = load_window_singles(rv, qa, vs + a, rec.la, lane);
    vb = load_window_singles(rv, qb, vs + rec.b, rec.lb, lane);
  }
  cp_async_mbar_arrive(bar);
  __syncwarp();
  if (lane == 0) {
    mbar_arrive_expect_tx(bar, ba.bytes + bb.bytes + va.bytes + vb.bytes);
    if (ba.bytes) bulk_g2s(ba.sdst, ba.gsrc, ba.bytes, bar);
    if (bb.bytes) bulk_g2s(bb.sdst, bb.gsrc, bb.bytes, bar);
    if (HAS_V && va.bytes) bulk_g2s(va.sdst, va.gsrc, va.bytes, bar);
    if (HAS_V && vb.bytes) bulk_g2s(vb.sdst, vb.gsrc, vb.bytes, bar);
  }
}

template <class K, bool HAS_V>
__host__ __device__ constexpr size_t merge_stage_bytes(int tile) {
  return ((region_elems(tile) * sizeof(K) + 127) & ~size_t(127)) +
         (HAS_V ? ((region_elems(tile) * 4 + 127) & ~size_t(127)) : 0);
}

// Output staging: when four stage-sized buffers fit in 64 KB, the merged
// block is staged in one of two separate output buffers; otherwise it is
// staged back into the stage it was merged from, which costs one more CTA
// barrier but keeps more CTAs per SM.
template <class K, bool HAS_V, int TILE>
__host__ __device__ constexpr bool separate_out() {
  return 4 * merge_stage_bytes<K, HAS_V>(TILE) <= 64 * 1024;
}
template <class K, bool HAS_V, int TILE>
__host__ __device__ constexpr int merge_buffers() {
  return separate_out<K, HAS_V, TILE>() ? 4 : 2;
}

template <class K, bool HAS_V, int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK, (HAS_V || sizeof(K) == 8) ? 2 : 3) k_merge(K* ku, uint32_t* vu, K* kw, uint32_t* vw,
                                                                 const MergeRec* __restrict__ recs, uint32_t npk,
                                                                 Tables tb) {
  constexpr int TILE = BLOCK * IPT;
  constexpr bool SEP = separate_out<K, HAS_V, TILE>();
  constexpr size_t KB = (region_elems(TILE) * sizeof(K) + 127) & ~size_t(127);
  constexpr size_t SB = merge_stage_bytes<K, HAS_V>(TILE);
  extern __shared__ __align__(128) unsigned char s_raw[];
  __shared__ __align__(8) uint64_t s_bar[2];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t total = tb.unit_prefix[npk];
  const uint32_t G = gridDim.x;
  uint32_t u = blockIdx.x;
  if (u >= total) return;
  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
  }
  mbar_fence_init();
  __syncthreads();

  const MergeRec none{0, 0, 0, 0, 0};
  MergeRec cur = recs[u];
  MergeRec nxt = (u + G < total) ? recs[u + G] : none;
  if (wid == 0)
    merge_issue<K, HAS_V>(cur, reinterpret_cast<K*>(s_raw), reinterpret_cast<uint32_t*>(s_raw + KB), &s_bar[0], ku,
                          vu, kw, vw, lane);
  uint32_t par0 = 0, par1 = 0;
  int s = 0;
  bool failed = false;
  for (; u < total; u += G) {
    const MergeRec nn = (u + 2 * G < total) ? recs[u + 2 * G] : none;
    unsigned char* st_cur = s_raw + s * SB;
    unsigned char* st_nxt = s_raw + (s ^ 1) * SB;
    if (wid == 0) {
      if constexpr (!SEP) {
        if (lane == 0) {
          bulk_wait_read0();  // the store staged in the other stage has read it
          fence_proxy_async();
        }
        __syncwarp();
      }
      merge_issue<K, HAS_V>(nxt, reinterpret_cast<K*>(st_nxt), reinterpret_cast<uint32_t*>(st_nxt + KB),
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
    const bool srcw = (cur.a & kSrcW) != 0;
    const uint64_t a = cur.a & ~kSrcW;
    const K* ks = srcw ? kw : ku;
    uint32_t pa, pb;
    place2(ks + a, cur.la, ks + cur.b, pa, pb);
    const int la = static_cast<int>(cur.la), lb = static_cast<int>(cur.lb), cnt = la + lb;
    const K* sA = rk + pa;
    const K* sB = rk + pb;
    K k[IPT];
    int src[IPT];
    const int d = tid * IPT;
    if (d < cnt) {
      const int i = corank_smem(sA, la, sB, lb, d);
      if (cnt == TILE) serial_merge<K, IPT, true, HAS_V>(sA, i, la, sB, d - i, lb, IPT, k, src);
      else serial_merge<K, IPT, false, HAS_V>(sA, i, la, sB, d - i, lb, min(IPT, cnt - d), k, src);
    }
    uint32_t v[IPT];
    if constexpr (HAS_V) {
      const uint32_t* vsrc = srcw ? vw : vu;
      uint32_t qa, qb;
      place2(vsrc + a, cur.la, vsrc + cur.b, qa, qb);
#pragma unroll
      for (int j = 0; j < IPT; ++j)
        if (d + j < cnt) v[j] = (src[j] & 0x10000) ? rv[qb + (src[j] & 0xffff)] : rv[qa + src[j]];
    }
    unsigned char* ob = SEP ? s_raw + (2 + s) * SB : st_cur;
    if constexpr (!SEP) __syncthreads();  // every read of the stage is done: stage the outputs in it
    K* okb = reinterpret_cast<K*>(ob);
    uint32_t* ovb = reinterpret_cast<uint32_t*>(ob + KB);
    K* kd = (srcw ? ku : kw) + cur.out;
    uint32_t* vd = HAS_V ? (srcw ? vu : vw) + cur.out : nullptr;
    const uint32_t ok_ph = phase_of(kd);
    const uint32_t ov_ph = HAS_V ? phase_of(vd) : 0u;
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      if (d + j < cnt) {
        okb[ok_ph + d + j] = k[j];
        if constexpr (HAS_V) ovb[ov_ph + d + j] = v[j];
      }
    }
    fence_proxy_async();
    if (SEP && tid == 0) bulk_wait_read0();  // the previous block's store has read the other output buffer
    __syncthreads();
    if (wid == 0 && cnt > 0) {
      store_window(kd, okb + ok_ph, cnt, lane);
      if constexpr (HAS_V) store_window(vd, ovb + ov_ph, cnt, lane);
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
