// The tile sort: every tile of every packet sorted by one CTA (see
// blockmerge.cuh for the layout and the pieces it shares with the merge).
#pragma once
#include "blockmerge.cuh"

namespace hs {

// ---------------------------------------------------------------------------
// k_tilesort
// ---------------------------------------------------------------------------
// Merge levels a tile of cnt keys needs: runs of IPT << lv items are merged
// while the first run does not yet hold every real key.
template <int IPT, int TILE>
__device__ __forceinline__ int levels_for(int cnt) {
  int lv = 0;
  while ((IPT << lv) < TILE && (IPT << lv) < cnt) ++lv;
  return lv;
}

// Packet offsets of a short segment sorted whole (see k_seg_plan): the
// segment's class follows from its smallest key (a negative int32 key means
// the flipped image) and its largest; in sorted order the packets are
// contiguous, so the item at position i opens every packet in
// (packet of item i-1, packet of item i].  The staged region `st` holds all
// cnt sorted keys; each thread reads its own items (blocked, conflict-free).
template <class K, int NB, int IPT>
__device__ __forceinline__ void short_segment_offsets(const K* st, int cnt, uint64_t beg, uint64_t* po) {
  using U = typename KT<K>::U;
  const bool flip = KT<K>::negative(st[0]);
  const U umax = KT<K>::image(st[cnt - 1], flip);
  const int cls = (NB == 10) ? dec_class(umax) : bin_class(umax);
  const DigitRule rule = (NB == 10) ? rule_dec(cls) : make_rule_bin(cls);
  const int i0 = static_cast<int>(threadIdx.x) * IPT;
  int qp = (i0 == 0 || i0 >= cnt) ? -1 : static_cast<int>(packet_of<NB>(KT<K>::image(st[i0 - 1], flip), rule));
#pragma unroll 1
  for (int i = i0; i < min(i0 + IPT, cnt); ++i) {
    const int q = static_cast<int>(packet_of<NB>(KT<K>::image(st[i], flip), rule));
    for (int p = qp + 1; p <= q; ++p) po[p] = beg + static_cast<uint64_t>(i);
    if (i == cnt - 1)
      for (int p = q + 1; p < NB; ++p) po[p] = beg + static_cast<uint64_t>(cnt);
    qp = q;
  }
}

// Work items of one launch: first every tile of every packet (read from the
// packet layout, written to U or W), then every short segment (read from and
// written back to the caller's array, its packet offsets written too).
template <class K, bool HAS_V, int NB, int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK, (sizeof(K) == 4 && !HAS_V) ? 5 : 4) k_tilesort(const K* __restrict__ kw, const uint32_t* __restrict__ vw, K* ku,
                                                     uint32_t* vu, K* kw_out, uint32_t* vw_out, uint32_t npk,
                                                     int force_w, int debug_stuck, uint64_t limit_ns, Tables tb) {
  griddep_open();
  constexpr int TILE = BLOCK * IPT;
  constexpr int RE = region_elems(TILE);
  extern __shared__ __align__(128) unsigned char s_raw[];
  K* rk = reinterpret_cast<K*>(s_raw);
  uint32_t* rv = reinterpret_cast<uint32_t*>(s_raw + ((RE * sizeof(K) + 127) & ~size_t(127)));
  __shared__ __align__(8) uint64_t s_bar;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t total = tb.unit_prefix[npk];
  const uint32_t items = total + *tb.small_cnt;
  if (tid == 0) mbar_init(&s_bar, 1);
  mbar_fence_init();
  __syncthreads();
  uint32_t parity = 0;
  bool failed = false;

  for (uint32_t u = blockIdx.x; u < items; u += gridDim.x) {
    const bool short_seg = u >= total;
    uint32_t seg = 0;
    uint64_t beg;
    int cnt;
    const K* gk;
    const uint32_t* gv;
    K* kd;
    uint32_t* vd;
    if (!short_seg) {
      const uint32_t p = find_pkt(tb.unit_prefix, npk, u);
      const uint32_t up0 = tb.unit_prefix[p], ntiles = tb.unit_prefix[p + 1] - up0;
      const int passes = passes_of(ntiles, tb.fan_log2);
      const bool to_w = force_w || (passes & 1);
      beg = tb.pkt_off[p] + static_cast<uint64_t>(u - up0) * TILE;
      cnt = static_cast<int>(min64(TILE, tb.pkt_off[p + 1] - beg));
      gk = kw + beg;
      gv = HAS_V ? vw + beg : nullptr;
      kd = (to_w ? kw_out : ku) + beg;
      vd = HAS_V ? (to_w ? vw_out : vu) + beg : nullptr;
    } else {
      seg = tb.small_list[u - total];
      beg = tb.seg_off[seg];
      cnt = static_cast<int>(min64(TILE, tb.seg_off[seg + 1] - beg));  // at most a tile by construction
      gk = ku + beg;
      gv = HAS_V ? vu + beg : nullptr;
      kd = ku + beg;
      vd = HAS_V ? vu + beg : nullptr;
    }
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

    // merge levels: runs of `run` = IPT << lv items -> 2 * run, in the region
    // at offset 0; a pair of runs is merged by 2 << lv threads, IPT outputs each.
    // Once the first run holds all cnt real keys the tile is sorted (the rest
    // is padding), so a short tile (the last of a small packet) stops early.
    const int nlv = levels_for<IPT, TILE>(cnt);
#pragma unroll 1
    for (int lv = 0; lv < nlv; ++lv) {
      const int run = IPT << lv;
      __syncthreads();
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        rk[tid * IPT + j] = k[j];
        if constexpr (HAS_V) rv[tid * IPT + j] = v[j];
      }
      __syncthreads();
      const int g = tid >> (lv + 1);                    // pair of runs
      const int diag = (tid & ((2 << lv) - 1)) * IPT;   // first output inside the pair
      const int a0 = g * 2 * run;
      const K* sA = rk + a0;
      const K* sB = sA + run;
      const int i = corank_smem(sA, run, sB, run, diag);
      int src[IPT];
      serial_merge<K, IPT, true, HAS_V>(sA, i, run, sB, diag - i, run, IPT, k, src);
      if constexpr (HAS_V) {
#pragma unroll
        for (int j = 0; j < IPT; ++j) v[j] = (src[j] & 0x10000) ? rv[a0 + run + (src[j] & 0xffff)] : rv[a0 + src[j]];
      }
    }
    // blocked registers -> region at the destination's phase -> bulk store
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
    if constexpr (NB > 1) {
      if (short_seg) {  // block-uniform
        short_segment_offsets<K, NB, IPT>(rk + ok_ph, cnt, beg, tb.pkt_off + static_cast<size_t>(seg) * NB);
        __syncthreads();  // every read of the region is done before the next item's copy refills it
      }
    }
  }
  // a copy may still be in flight into the region: give it a bounded chance
  // to land before the CTA's shared memory is released
  if (failed) mbar_wait_bounded(&s_bar, parity, tb.err, limit_ns);
  if (tid == 0) bulk_wait0();
}

// ---------------------------------------------------------------------------
// k_copy_back_pass (testing): after merge pass r every packet's data is in the
// buffer that pass wrote -- W when the packet still needs passes after r and
// (passes - r) is odd, else the caller's array U (a packet that needed fewer
// passes finished in U).  Copies the W-resident tiles to U, one tile per CTA.
// ---------------------------------------------------------------------------
template <class K, bool HAS_V, int TILE>
__global__ void k_copy_back_pass(K* ku, uint32_t* vu, const K* __restrict__ kw, const uint32_t* __restrict__ vw,
                                 uint32_t npk, int r, Tables tb) {
  griddep_open();
  const uint32_t total = tb.unit_prefix[npk];
  for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {
    const uint32_t p = find_pkt(tb.unit_prefix, npk, u);
    const uint32_t up0 = tb.unit_prefix[p], ntiles = tb.unit_prefix[p + 1] - up0;
    const int passes = passes_of(ntiles, tb.fan_log2);
    if (r > passes || ((passes - r) & 1) == 0) continue;  // this packet's data is in U
    const uint64_t beg = tb.pkt_off[p] + static_cast<uint64_t>(u - up0) * TILE;
    const uint32_t cnt = static_cast<uint32_t>(min64(TILE, tb.pkt_off[p + 1] - beg));
    for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
      ku[beg + i] = kw[beg + i];
      if constexpr (HAS_V) vu[beg + i] = vw[beg + i];
    }
  }
}

}  // namespace hs
