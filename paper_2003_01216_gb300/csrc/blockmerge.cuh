// Shared pieces of the per-packet sort (Sec. 3.2, Fig. 1) on the GPU:
//   k_tilesort  every packet is cut into tiles of TILE = BLOCK * IPT keys that
//               start at the packet's first key (the last tile of a packet may
//               be short); one CTA sorts one tile: a sorting network per thread
//               over its IPT keys in registers, then log2(BLOCK) merge-path
//               merges in shared memory.  This replaces the paper's per-thread
//               sequential quicksort of one data part.
//   k_corank    merge pass r, for every merge block (TILE outputs) the split of
//               its first and one-past-last output between the two runs it
//               merges (merge path: a search along the cross diagonal, binary
//               per thread, or by a group of lanes when the pass has few
//               merge blocks).
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
// Search by a group of G lanes (G a power of two, at most 16; lanes
// [gbase, gbase + G) of the warp, j = this lane's index in the group): the
// first position in [lo, hi) whose predicate `taken` is false, hi if none,
// for a predicate that is true on a prefix of the interval.  Every step the
// G lanes probe G evenly spaced points at once, so the interval shrinks
// (G + 1)-fold per dependent load instead of 2-fold; once it holds at most G
// points all of them are probed.  Every lane of the warp calls it (the loop
// is warp-uniform); a group with an empty interval probes nothing.
// ---------------------------------------------------------------------------
template <int G, class Taken>
__device__ __forceinline__ uint32_t group_search(uint32_t lo, uint32_t hi, int j, int gbase, Taken taken) {
  static_assert(G >= 2 && G <= 16 && (G & (G - 1)) == 0, "group of 2, 4, 8 or 16 lanes");
  while (__any_sync(0xffffffffu, lo < hi)) {
    const uint32_t n = hi - lo;
    bool t = false;
    if (n > 0) {
      const uint32_t m = (n <= static_cast<uint32_t>(G))
                             ? lo + j
                             : lo + static_cast<uint32_t>((static_cast<uint64_t>(j + 1) * n) / (G + 1));
      if (m < hi) t = taken(m);
    }
    const uint32_t k = __popc((__ballot_sync(0xffffffffu, t) >> gbase) & ((1u << G) - 1u));
    if (n > 0) {
      if (n <= static_cast<uint32_t>(G)) {  // every point of the interval probed
        lo += k;
        hi = lo;
      } else {  // the taken probes are a prefix: keep the gap after the last one
        const uint32_t nlo = k ? lo + static_cast<uint32_t>((static_cast<uint64_t>(k) * n) / (G + 1)) + 1u : lo;
        const uint32_t nhi =
            (k < static_cast<uint32_t>(G)) ? lo + static_cast<uint32_t>((static_cast<uint64_t>(k + 1) * n) / (G + 1))
                                           : hi;
        lo = nlo;
        hi = nhi;
      }
    }
  }
  return lo;
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

}  // namespace hs
