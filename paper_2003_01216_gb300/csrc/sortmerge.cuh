// Per-packet sort (Sec. 3.2, Fig. 1) on the GPU:
//   k_tilesort  every packet is cut into tiles of TILE keys that start at the
//               packet's first key (the last tile of a packet may be short);
//               one CTA sorts one tile: a sorting network per thread over its
//               IPT keys in registers, then log2(BLOCK) merge-path merges in
//               shared memory.  This replaces the paper's per-thread sequential
//               quicksort of one data part.
//   k_corank    merge pass r, for every merge block (TILE outputs) the split
//               point of its first output between the two runs it merges
//               (merge path: binary search along the cross diagonal).
//   k_merge     merge pass r: one CTA writes TILE consecutive outputs of one
//               pair of runs of length TILE * 2^(r-1); runs never cross a
//               packet boundary.  Passes repeat until every packet is one run:
//               the non-recursive, bottom-up merge of Fig. 1(b) and Sec. 3.2,
//               with every CTA merging an equal share instead of one thread
//               per pair of lists.
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
#include "common.cuh"

namespace hs {

__device__ __forceinline__ int pad(int i) { return i + (i >> 5); }

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

// Geometry of merge block u in pass r (r >= 1) of its packet.
struct MergeGeom {
  uint64_t pstart;   // packet start (absolute)
  uint64_t a_start;  // first run of the pair, packet-relative
  uint32_t a_len, b_len;
  uint32_t diag0;    // first output of this block inside the pair
  uint32_t cnt;      // outputs of this block
  int passes;        // merge passes the packet needs
  bool last_in_pair; // the next merge block belongs to another pair (or packet)
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
  g.last_in_pair = (g.diag0 + g.cnt) == (g.a_len + g.b_len);
  return true;
}

// ---------------------------------------------------------------------------
// In-register sorting networks over N items (N a power of two).
// ---------------------------------------------------------------------------
template <class K>
__device__ __forceinline__ void cas_keys(K& a, K& b) {
  const K lo = min(a, b), hi = max(a, b);
  a = lo;
  b = hi;
}

// Batcher's odd-even merge sort network (keys only; not stable, which does not
// matter for keys alone).
template <int N, class K>
__device__ __forceinline__ void network_sort(K (&k)[N]) {
#pragma unroll
  for (int p = 1; p < N; p <<= 1) {
#pragma unroll
    for (int kk = p; kk >= 1; kk >>= 1) {
#pragma unroll
      for (int j = kk % p; j + kk < N; j += 2 * kk) {
#pragma unroll
        for (int i = 0; i < kk; ++i) {
          if (i + j + kk < N && (i + j) / (2 * p) == (i + j + kk) / (2 * p)) cas_keys(k[i + j], k[i + j + kk]);
        }
      }
    }
  }
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

// Serial merge of IPT outputs from sa[ai..aend) and sa[bi..bend) (padded
// shared-memory indices), equal keys from the A side first.  Outputs keep the
// shared-memory index they came from in idx[] (for values).
template <class K, int IPT>
__device__ __forceinline__ void serial_merge(const K* sk, int ai, int aend, int bi, int bend, int nout, K (&out)[IPT],
                                             int (&idx)[IPT]) {
  K ka = (ai < aend) ? sk[pad(ai)] : KT<K>::maxv();
  K kb = (bi < bend) ? sk[pad(bi)] : KT<K>::maxv();
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    if (j < nout) {
      const bool take_a = (bi >= bend) || ((ai < aend) && !(kb < ka));
      out[j] = take_a ? ka : kb;
      idx[j] = take_a ? ai : bi;
      if (take_a) {
        ++ai;
        ka = (ai < aend) ? sk[pad(ai)] : KT<K>::maxv();
      } else {
        ++bi;
        kb = (bi < bend) ? sk[pad(bi)] : KT<K>::maxv();
      }
    }
  }
}

// Merge path inside shared memory: number of A items among the first `diag`
// outputs of merging A = sk[a0, a0+la) and B = sk[b0, b0+lb).
template <class K>
__device__ __forceinline__ int corank_smem(const K* sk, int a0, int la, int b0, int lb, int diag) {
  int lo = diag > lb ? diag - lb : 0;
  int hi = diag < la ? diag : la;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (!(sk[pad(b0 + diag - 1 - mid)] < sk[pad(a0 + mid)])) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Shared-memory elements for n padded items (one pad slot per 32).
__host__ __device__ constexpr int padded(int n) { return n + (n >> 5) + 1; }

// ---------------------------------------------------------------------------
// k_tilesort
// ---------------------------------------------------------------------------
template <class K, bool HAS_V, int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK) k_tilesort(const K* __restrict__ kw, const uint32_t* __restrict__ vw, K* ku,
                                                     uint32_t* vu, K* kw_out, uint32_t* vw_out, uint32_t npk,
                                                     int force_w, Tables tb) {
  constexpr int TILE = BLOCK * IPT;
  extern __shared__ __align__(16) unsigned char s_raw[];
  K* sk = reinterpret_cast<K*>(s_raw);
  uint32_t* sv = reinterpret_cast<uint32_t*>(sk + padded(TILE));
  const int tid = threadIdx.x;
  const uint32_t total = tb.unit_prefix[npk];

  for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {
    const uint32_t p = find_pkt(tb.unit_prefix, npk, u);
    const uint32_t up0 = tb.unit_prefix[p], ntiles = tb.unit_prefix[p + 1] - up0;
    const int passes = ceil_log2(ntiles);
    const bool to_w = force_w || (passes & 1);
    const uint64_t pstart = tb.pkt_off[p];
    const uint64_t beg = pstart + static_cast<uint64_t>(u - up0) * TILE;
    const int cnt = static_cast<int>(min64(TILE, tb.pkt_off[p + 1] - beg));

    // coalesced load into shared memory; missing keys become the largest key
#pragma unroll
    for (int c = 0; c < IPT; ++c) {
      const int i = c * BLOCK + tid;
      sk[pad(i)] = (i < cnt) ? kw[beg + i] : KT<K>::maxv();
      if constexpr (HAS_V) sv[pad(i)] = (i < cnt) ? vw[beg + i] : 0u;
    }
    __syncthreads();
    K k[IPT];
    uint32_t v[IPT];
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      k[j] = sk[pad(tid * IPT + j)];
      if constexpr (HAS_V) v[j] = sv[pad(tid * IPT + j)];
    }
    if constexpr (HAS_V) transposition_sort<IPT>(k, v);
    else network_sort<IPT>(k);

    // merge levels: runs of `run` items -> 2 * run
#pragma unroll 1
    for (int run = IPT; run < TILE; run <<= 1) {
      __syncthreads();
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        sk[pad(tid * IPT + j)] = k[j];
        if constexpr (HAS_V) sv[pad(tid * IPT + j)] = v[j];
      }
      __syncthreads();
      const int tpg = (2 * run) / IPT;
      const int a0 = (tid / tpg) * 2 * run;
      const int diag = (tid % tpg) * IPT;
      const int i = corank_smem(sk, a0, run, a0 + run, run, diag);
      int idx[IPT];
      serial_merge<K, IPT>(sk, a0 + i, a0 + run, a0 + run + diag - i, a0 + 2 * run, IPT, k, idx);
      if constexpr (HAS_V) {
#pragma unroll
        for (int j = 0; j < IPT; ++j) v[j] = sv[pad(idx[j])];
      }
    }
    // blocked registers -> shared -> coalesced stores
    __syncthreads();
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      sk[pad(tid * IPT + j)] = k[j];
      if constexpr (HAS_V) sv[pad(tid * IPT + j)] = v[j];
    }
    __syncthreads();
    K* kd = to_w ? kw_out : ku;
    uint32_t* vd = to_w ? vw_out : vu;
#pragma unroll
    for (int c = 0; c < IPT; ++c) {
      const int i = c * BLOCK + tid;
      if (i < cnt) {
        kd[beg + i] = sk[pad(i)];
        if constexpr (HAS_V) vd[beg + i] = sv[pad(i)];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Merge pass r, step 1 -- k_corank: for every merge block, the split of its
// first and of its one-past-last output between the two runs it merges (the
// merge path co-ranks), packed into a record the merge kernel reads once.
// Each thread runs both searches interleaved as 8-ary searches (7 independent
// probes per round), so a run of 2^27 keys takes 9 dependent rounds.
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
// B[0, lb) with A first on ties; two diagonals at once.
template <class K>
__device__ __forceinline__ void corank2(const K* __restrict__ A, uint32_t la, const K* __restrict__ B, uint32_t lb,
                                        uint32_t d0, uint32_t d1, uint32_t& r0, uint32_t& r1) {
  uint32_t lo0 = d0 > lb ? d0 - lb : 0, hi0 = min(d0, la);
  uint32_t lo1 = d1 > lb ? d1 - lb : 0, hi1 = min(d1, la);
  // g(i) = A[i] <= B[d - 1 - i] is true for i below the answer, false from it on
  while (hi0 > lo0 || hi1 > lo1) {
    const uint32_t st0 = (hi0 - lo0 + 7) >> 3, st1 = (hi1 - lo1 + 7) >> 3;
    uint32_t t0 = 0, t1 = 0;
#pragma unroll
    for (int j = 1; j <= 8; ++j) {
      const uint32_t p0 = lo0 + (j - 1) * st0, p1 = lo1 + (j - 1) * st1;
      if (hi0 > lo0 && p0 < hi0 && !(B[d0 - 1 - p0] < A[p0])) ++t0;
      if (hi1 > lo1 && p1 < hi1 && !(B[d1 - 1 - p1] < A[p1])) ++t1;
    }
    // t probes true: the answer lies in (lo + (t-1)*st, lo + t*st]
    if (hi0 > lo0) {
      if (t0 == 0) hi0 = lo0;
      else {
        const uint32_t nl = lo0 + (t0 - 1) * st0 + 1;
        hi0 = min(hi0, lo0 + t0 * st0);
        lo0 = min(nl, hi0);
      }
    }
    if (hi1 > lo1) {
      if (t1 == 0) hi1 = lo1;
      else {
        const uint32_t nl = lo1 + (t1 - 1) * st1 + 1;
        hi1 = min(hi1, lo1 + t1 * st1);
        lo1 = min(nl, hi1);
      }
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
// blockIdx.x, +gridDim.x, ...  A two-stage pipeline of asynchronous copies
// (cp.async, global -> padded shared memory) loads block k+1's A and B items
// while block k is merged; block k+2's record is fetched one block ahead.
// ---------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sa), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

template <class K, bool HAS_V, int BLOCK, int IPT>
__device__ __forceinline__ void merge_issue(const MergeRec& rec, K* sk, uint32_t* sv, const K* ku, const uint32_t* vu,
                                            const K* kw, const uint32_t* vw) {
  const bool srcw = (rec.a & kSrcW) != 0;
  const K* ks = srcw ? kw : ku;
  const uint32_t* vs = srcw ? vw : vu;
  const uint64_t a = rec.a & ~kSrcW;
  const int la = static_cast<int>(rec.la), cnt = static_cast<int>(rec.la + rec.lb);
#pragma unroll
  for (int c = 0; c < IPT; ++c) {
    const int e = c * BLOCK + static_cast<int>(threadIdx.x);
    if (e < cnt) {
      const uint64_t gi = (e < la) ? a + e : rec.b + (e - la);
      cp_async<sizeof(K)>(&sk[pad(e)], ks + gi);
      if constexpr (HAS_V) cp_async<4>(&sv[pad(e)], vs + gi);
    }
  }
}

template <class K, bool HAS_V, int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK, HAS_V ? 2 : 4) k_merge(K* ku, uint32_t* vu, K* kw, uint32_t* vw,
                                                  const MergeRec* __restrict__ recs, uint32_t npk, Tables tb) {
  constexpr int TILE = BLOCK * IPT;
  constexpr int SP = padded(TILE);
  extern __shared__ __align__(16) unsigned char s_raw[];
  K* skb = reinterpret_cast<K*>(s_raw);                         // 2 stages of SP keys
  uint32_t* svb = reinterpret_cast<uint32_t*>(skb + 2 * SP);    // 2 stages of SP values (pairs)
  const int tid = threadIdx.x;
  const uint32_t total = tb.unit_prefix[npk];
  const uint32_t G = gridDim.x;
  uint32_t u = blockIdx.x;
  if (u >= total) return;
  const MergeRec none{0, 0, 0, 0, 0};
  MergeRec cur = recs[u];
  MergeRec nxt = (u + G < total) ? recs[u + G] : none;
  merge_issue<K, HAS_V, BLOCK, IPT>(cur, skb, svb, ku, vu, kw, vw);
  cp_async_commit();
  int s = 0;
  for (; u < total; u += G) {
    const MergeRec nn = (u + 2 * G < total) ? recs[u + 2 * G] : none;
    merge_issue<K, HAS_V, BLOCK, IPT>(nxt, skb + (s ^ 1) * SP, svb + (s ^ 1) * SP, ku, vu, kw, vw);
    cp_async_commit();
    cp_async_wait_1();  // this thread's copies for block `cur` have landed
    __syncthreads();    // ... and every other thread's
    K* sk = skb + s * SP;
    uint32_t* sv = svb + s * SP;
    const int la = static_cast<int>(cur.la), cnt = static_cast<int>(cur.la + cur.lb);
    K k[IPT];
    int idx[IPT];
    const int d = tid * IPT;
    if (d < cnt) {
      const int i = corank_smem(sk, 0, la, la, cnt - la, d);
      serial_merge<K, IPT>(sk, i, la, la + d - i, cnt, min(IPT, cnt - d), k, idx);
    }
    uint32_t v[IPT];
    if constexpr (HAS_V) {
#pragma unroll
      for (int j = 0; j < IPT; ++j)
        if (d + j < cnt) v[j] = sv[pad(idx[j])];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      if (d + j < cnt) {
        sk[pad(d + j)] = k[j];
        if constexpr (HAS_V) sv[pad(d + j)] = v[j];
      }
    }
    __syncthreads();
    const bool srcw = (cur.a & kSrcW) != 0;
    K* out = (srcw ? ku : kw) + cur.out;
    uint32_t* vout = (srcw ? vu : vw) + cur.out;
#pragma unroll
    for (int c = 0; c < IPT; ++c) {
      const int e = c * BLOCK + tid;
      if (e < cnt) {
        out[e] = sk[pad(e)];
        if constexpr (HAS_V) vout[e] = sv[pad(e)];
      }
    }
    __syncthreads();  // stage s is free for block k+2's copies
    cur = nxt;
    nxt = nn;
    s ^= 1;
  }
}

}  // namespace hs
