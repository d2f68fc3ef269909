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
// k_corank: merge-path split of the first output of every merge block of
// pass r, by binary search in global memory.
// ---------------------------------------------------------------------------
template <class K, int TILE>
__global__ void k_corank(const K* __restrict__ ku, const K* __restrict__ kw, uint32_t npk, int r, Tables tb) {
  const uint32_t total = tb.unit_prefix[npk];
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x) {
    MergeGeom g;
    if (!merge_geom<TILE>(tb, npk, u, r, g)) continue;
    const K* src = ((g.passes - r + 1) & 1) ? kw : ku;  // buffer holding pass r-1
    const K* A = src + g.pstart + g.a_start;
    const K* B = A + g.a_len;
    const uint32_t diag = g.diag0;
    uint32_t lo = diag > g.b_len ? diag - g.b_len : 0;
    uint32_t hi = min(diag, g.a_len);
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (!(B[diag - 1 - mid] < A[mid])) lo = mid + 1; else hi = mid;
    }
    tb.corank[u] = lo;
  }
}

// ---------------------------------------------------------------------------
// k_merge: merge pass r.
// ---------------------------------------------------------------------------
template <class K, bool HAS_V, int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK) k_merge(K* ku, uint32_t* vu, K* kw, uint32_t* vw, uint32_t npk, int r,
                                                  Tables tb) {
  constexpr int TILE = BLOCK * IPT;
  extern __shared__ __align__(16) unsigned char s_raw[];
  K* sk = reinterpret_cast<K*>(s_raw);
  uint32_t* sv = reinterpret_cast<uint32_t*>(sk + padded(TILE));
  const int tid = threadIdx.x;
  const uint32_t total = tb.unit_prefix[npk];

  for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {
    MergeGeom g;
    if (!merge_geom<TILE>(tb, npk, u, r, g)) continue;  // block-uniform
    const bool src_w = ((g.passes - r + 1) & 1) != 0;
    const K* ks = src_w ? kw : ku;
    const uint32_t* vs = src_w ? vw : vu;
    K* kd = src_w ? ku : kw;
    uint32_t* vd = src_w ? vu : vw;
    const uint32_t i0 = tb.corank[u];
    const uint32_t i1 = g.last_in_pair ? g.a_len : tb.corank[u + 1];
    const uint32_t j0 = g.diag0 - i0;
    const int la = static_cast<int>(i1 - i0), cnt = static_cast<int>(g.cnt);
    const K* A = ks + g.pstart + g.a_start;
    const K* B = A + g.a_len;
    const uint32_t* VA = vs + g.pstart + g.a_start;
    const uint32_t* VB = VA + g.a_len;

#pragma unroll
    for (int c = 0; c < IPT; ++c) {
      const int e = c * BLOCK + tid;
      if (e < cnt) {
        const bool fa = e < la;
        sk[pad(e)] = fa ? A[i0 + e] : B[j0 + (e - la)];
        if constexpr (HAS_V) sv[pad(e)] = fa ? VA[i0 + e] : VB[j0 + (e - la)];
      }
    }
    __syncthreads();
    K k[IPT];
    int idx[IPT];
    const int d = tid * IPT;
    if (d < cnt) {
      const int lb = cnt - la;
      const int i = corank_smem(sk, 0, la, la, lb, d);
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
    K* out = kd + g.pstart + g.a_start + g.diag0;
    uint32_t* vout = vd + g.pstart + g.a_start + g.diag0;
#pragma unroll
    for (int c = 0; c < IPT; ++c) {
      const int e = c * BLOCK + tid;
      if (e < cnt) {
        out[e] = sk[pad(e)];
        if constexpr (HAS_V) vout[e] = sv[pad(e)];
      }
    }
    __syncthreads();
  }
}

}  // namespace hs
