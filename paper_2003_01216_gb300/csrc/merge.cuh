// Bottom-up merge passes (Fig. 1(b), Sec. 3.2): co-rank records and the
// persistent merge kernel (see blockmerge.cuh for the shared pieces).
#pragma once
#include "blockmerge.cuh"

namespace hs {

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
constexpr uint64_t kFinal = 1ull << 62;  // merge queue: the block is in its packet's last pass

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

// Record of one merge block from its geometry and the co-ranks i0, i1 of its
// first and one-past-last output.
__device__ __forceinline__ MergeRec make_rec(const MergeGeom& g, bool srcw, uint32_t i0, uint32_t i1) {
  const uint64_t abs_a = g.pstart + g.a_start;
  MergeRec rec;
  rec.a = (abs_a + i0) | (srcw ? kSrcW : 0ull);
  rec.b = abs_a + g.a_len + (g.diag0 - i0);
  rec.out = abs_a + g.diag0;
  rec.la = i1 - i0;
  rec.lb = g.cnt - rec.la;
  return rec;
}

// Records of the active lanes, packed densely at pass_ctl[r] (their order
// does not matter).  Called by all 32 lanes.
__device__ __forceinline__ void push_recs(bool writer, const MergeRec& rec, MergeRec* recs, uint32_t* ctr, int lane) {
  const uint32_t mask = __ballot_sync(0xffffffffu, writer);
  if (mask) {
    uint32_t slot = 0;
    if (lane == __ffs(mask) - 1) slot = atomicAdd(ctr, __popc(mask));
    slot = __shfl_sync(0xffffffffu, slot, __ffs(mask) - 1);
    if (writer) recs[slot + __popc(mask & ((1u << lane) - 1u))] = rec;
  }
}

// G == 1: one thread per merge block, its two searches interleaved.
// G > 1: 2G lanes per merge block, G per search (group_search), for passes
// with few merge blocks, which are bound by the latency of the search chain.
template <class K, int TILE, int G>
__global__ void k_corank(const K* __restrict__ ku, const K* __restrict__ kw, MergeRec* __restrict__ recs,
                         uint32_t npk, int r, Tables tb) {
  griddep_open();
  if (static_cast<uint32_t>(r) > tb.pass_ctl[0]) return;  // no packet needs pass r
  const uint32_t total = tb.unit_prefix[npk];
  const int lane = threadIdx.x & 31;
  if constexpr (G == 1) {
    const uint32_t stride = gridDim.x * blockDim.x;
    // warp-uniform trip count: lanes past the end take part in the ballot
    for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total; base += stride) {
      const uint32_t u = base + lane;
      MergeGeom g;
      MergeRec rec{0, 0, 0, 0, 0};
      const bool active = u < total && merge_geom<TILE>(tb, npk, u, r, g);
      if (active) {
        const bool srcw = ((g.passes - r + 1) & 1) != 0;  // the buffer holding pass r-1
        const K* A = (srcw ? kw : ku) + g.pstart + g.a_start;
        const K* B = A + g.a_len;
        uint32_t i0, i1;
        corank2(A, g.a_len, B, g.b_len, g.diag0, g.diag0 + g.cnt, i0, i1);
        rec = make_rec(g, srcw, i0, i1);
      }
      push_recs(active, rec, recs, &tb.pass_ctl[r], lane);
    }
  } else {
    constexpr int L = 2 * G;     // lanes per merge block
    constexpr int BPW = 32 / L;  // merge blocks per warp
    const int sub = lane % L, q = sub / G, j = sub % G;
    const int gbase = lane - j;  // first lane of this lane's search group
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t w = warp; w * BPW < total; w += nwarps) {  // warp-uniform
      const uint32_t u = w * BPW + lane / L;
      MergeGeom g;
      const bool active = u < total && merge_geom<TILE>(tb, npk, u, r, g);
      const K* A = ku;
      const K* B = ku;
      bool srcw = false;
      uint32_t d = 0, lo = 0, hi = 0;
      if (active) {
        srcw = ((g.passes - r + 1) & 1) != 0;
        A = (srcw ? kw : ku) + g.pstart + g.a_start;
        B = A + g.a_len;
        d = g.diag0 + (q ? g.cnt : 0u);  // q = 0: first output, q = 1: one past the last
        lo = d > g.b_len ? d - g.b_len : 0u;
        hi = min(d, g.a_len);
      }
      // probe m is taken (the co-rank exceeds m) when B[d - 1 - m] does not
      // precede A[m]
      lo = group_search<G>(lo, hi, j, gbase, [&](uint32_t m) { return !(B[d - 1 - m] < A[m]); });
      const int l0 = lane - sub;  // lane holding the block's first co-rank
      const uint32_t i0 = __shfl_sync(0xffffffffu, lo, l0);
      const uint32_t i1 = __shfl_sync(0xffffffffu, lo, l0 + G);
      const bool writer = active && sub == 0;
      MergeRec rec{0, 0, 0, 0, 0};
      if (writer) rec = make_rec(g, srcw, i0, i1);
      push_recs(writer, rec, recs, &tb.pass_ctl[r], lane);
    }
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
  const uint64_t a = rec.a & ~(kSrcW | kFinal);
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
                                                                 const MergeRec* __restrict__ recs, int r,
                                                                 Tables tb) {
  griddep_open();
  constexpr int TILE = BLOCK * IPT;
  constexpr bool SEP = separate_out<K, HAS_V, TILE>();
  constexpr size_t KB = (region_elems(TILE) * sizeof(K) + 127) & ~size_t(127);
  constexpr size_t SB = merge_stage_bytes<K, HAS_V>(TILE);
  extern __shared__ __align__(128) unsigned char s_raw[];
  __shared__ __align__(8) uint64_t s_bar[2];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t total = tb.pass_ctl[r];  // active merge blocks, packed by k_corank
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
