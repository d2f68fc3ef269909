// Bottom-up merge passes (Fig. 1(b), Sec. 3.2) as ONE persistent launch: a
// device work queue of (packet, merge pass r, merge block) items drained by
// resident CTAs, each item started as soon as the two runs it merges are
// complete, with every dependency wait bounded.
//
// The paper's tree merge runs round by round: a round starts when the
// previous one has finished everywhere.  Here the items are handed out in
// pass-major order (tickets: pass 1's merge blocks of every packet, then
// pass 2's, ...), and a merge block of pass r waits only for the two runs it
// reads, i.e. for the blocks of pass r-1 that wrote them.  Packets that need
// fewer passes drop out, short passes of small packets overlap the long ones
// of large packets, and no kernel boundary separates the passes.
//
// Progress: a CTA takes tickets only while it runs, takes them in increasing
// order and finishes them in that order; an item depends only on items with
// smaller tickets.  The smallest unfinished ticket therefore never waits on
// anything unfinished, whatever the number of resident CTAs, so the queue
// always drains.  Every wait is bounded anyway (globaltimer): on expiry the
// CTA sets the device error word, every CTA that sees the word stops taking
// items, and the launch ends with HS_ERR_TIMEOUT reported to the caller.
//
// One CTA = BLOCK consumer threads (warps 0 .. BLOCK/32 - 1), which merge, and
// one producer warp, which claims tickets eight at a time, waits for the
// items' inputs (acquire loads of per-run completion counters), finds every
// item's merge-path co-ranks in global memory (two lanes per search, all
// sixteen searches of a round interleaved, see group_search), and passes the
// records to the consumers through a ring in shared memory (sleeping while
// the ring is full).  Consumer warp 0 issues the bulk copies of block k+1
// while block k is merged (two stages, as k_merge), stores the merged block
// by bulk copy and, once a store has completed, publishes it (release add on
// the counter of the run it belongs to).
//
// A second instantiation (TO_HOST) serves sorts of keys in pinned host
// memory: the blocks of every packet's last pass go from the stage straight
// to the caller's host array (plain 16-byte stores by all merging warps),
// and k_copy_unmerged moves the packets that needed no merge pass there.
// Those last passes are bound by the host link (~200 GB/s), the others by
// HBM, so the instantiation orders the work to overlap the two (for packet
// tables of at most kSchedSmemPackets entries): device tickets take every
// packet's passes but its last, packet by packet (packet 0's passes first,
// so its last pass can start early), and host tickets, from a second
// counter, the last passes, packet by packet.  The first min(32, grid / 8)
// CTAs take host tickets from the start; the others take device tickets and
// then host tickets once the device tickets run out.  A host ticket depends
// on device tickets only, a device ticket on smaller device tickets only, so
// the progress argument above holds for each counter.
#pragma once
#include "blockmerge.cuh"
#include "merge.cuh"

namespace hs {

constexpr int kSchedRing = 16;   // records in flight between producer and consumers
constexpr int kSchedRound = 8;   // tickets claimed by the producer at once (four lanes each)
constexpr uint32_t kSchedSmemPackets = 64;  // packet tables this small are read from shared memory
constexpr uint32_t kSigNone = 0xffffffffu;
constexpr uint32_t kSchedHostCtas = 32;  // TO_HOST: CTAs that take host tickets from the start (at most)

// last p in [0, npk) with pre[p] <= t (pre non-decreasing)
__device__ __forceinline__ uint32_t find_pre64(const uint64_t* pre, uint32_t npk, uint64_t t) {
  uint32_t lo = 0, hi = npk;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (pre[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(uint32_t* p, uint32_t v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// order this thread's global accesses of the asynchronous proxy (bulk
// copies) with its generic ones
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
// barrier of the consumer warps only (named barrier 1); returns whether any
// consumer thread passed `pred`
__device__ __forceinline__ bool consumers_sync_or(bool pred, int nthreads) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"(pred ? 1u : 0u), "r"(nthreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void consumers_sync(int nthreads) {
  asm volatile("barrier.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Completion counter of the run that pass r's pair starting at unit `ps`
// writes: done[r * units + ps].
__device__ __forceinline__ uint32_t* run_counter(uint32_t* done, uint32_t units, int r, uint32_t ps) {
  return done + static_cast<size_t>(r) * units + ps;
}

// Bounded spin until *p >= need; false (and kErrTimeout) when the limit
// passes, false without a new error bit when another CTA already failed.
// idle() runs between tests (the producer publishes its CTA's finished
// blocks there, so two CTAs never wait on each other's publications).
template <class Idle>
__device__ __forceinline__ bool wait_count(const uint32_t* p, uint32_t need, uint32_t* err, uint64_t limit_ns,
                                           Idle idle) {
  if (ld_acquire_u32(p) >= need) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    idle();
    __nanosleep(it < 64 ? 32 : 256);
    if (ld_acquire_u32(p) >= need) return true;
    if ((it & 15) == 0) {
      if (*reinterpret_cast<volatile uint32_t*>(err) != 0) return false;
      if (globaltimer_ns() - t0 > limit_ns) {
        atomicOr(err, kErrTimeout);
        return false;
      }
    }
  }
}

// Bounded wait on an mbarrier phase that backs off with nanosleep between
// tests, for waits that can be long (a full record ring): a thread spinning
// on try_wait would take issue slots from the warps that merge.  idle() as
// for wait_count.
template <class Idle>
__device__ __forceinline__ bool mbar_wait_sleepy(uint64_t* bar, uint32_t parity, uint32_t* err, uint64_t limit_ns,
                                                 Idle idle) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    idle();
    __nanosleep(it < 8 ? 128 : 512);
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 15) == 0 && globaltimer_ns() - t0 > limit_ns) {
      atomicOr(err, kErrTimeout);
      return false;
    }
  }
}

__device__ __forceinline__ uint32_t ld_acquire_cta_shared(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.cta.shared.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_cta_shared(uint32_t* p, uint32_t v) {
  asm volatile("st.release.cta.shared.u32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}

struct SchedArgs {
  uint32_t* done;       // (passes + 1) x units completion counters, zeroed
  uint32_t* ticket;     // next ticket (64-bit), zeroed; TO_HOST: next host ticket at ticket + 2 (64-bit), zeroed
  int pass_limit;       // passes to run (testing: stop after pass r), else kMaxPasses
  int debug_drop;       // testing: the block of ticket 0 never publishes its completion
  uint64_t limit_ns;    // bound of every wait
  void* host_out;       // keys only: nullptr, or the caller's pinned host array (device-addressable):
                        // blocks of a packet's last pass are written there instead of to U
};

// TO_HOST (keys only, host-buffer calls): the blocks of a packet's last pass
// are written to sa.host_out instead of U; a separate instantiation, so the
// device-only kernel carries none of it.
template <class K, bool HAS_V, int BLOCK, int IPT, bool TO_HOST = false>
__global__ void __launch_bounds__(BLOCK + 32, (HAS_V || sizeof(K) == 8) ? 2 : 3)
    k_merge_sched(K* ku, uint32_t* vu, K* kw, uint32_t* vw, uint32_t npk, Tables tb, SchedArgs sa) {
  griddep_open();
  constexpr int TILE = BLOCK * IPT;
  constexpr size_t KB = (region_elems(TILE) * sizeof(K) + 127) & ~size_t(127);
  constexpr size_t SB = merge_stage_bytes<K, HAS_V>(TILE);
  constexpr int R = kSchedRing;
  // (two stages; the merged block is always staged in the stage it was read from)
  extern __shared__ __align__(128) unsigned char s_raw[];
  __shared__ __align__(8) uint64_t s_full[2];      // stage loads landed
  __shared__ __align__(8) uint64_t s_rfull[R];     // record written (producer -> consumers)
  __shared__ __align__(8) uint64_t s_rempty[R];    // record consumed (consumers -> producer)
  __shared__ __align__(16) MergeRec s_rec[R];
  __shared__ uint32_t s_sig[R];                    // counter index to publish, kSigNone: none; bit 31 of
                                                   // s_tkt: end of the queue
  __shared__ uint32_t s_tkt[R];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int NW = BLOCK / 32;
  const uint32_t units = tb.unit_prefix[npk];
  const int passes = min(static_cast<int>(tb.pass_ctl[0]), sa.pass_limit);
  const uint64_t total = static_cast<uint64_t>(passes) * units;
  // Publication of finished blocks (see the consumer part): thread 0 notes
  // each block's counter index in s_pend when its store is issued and raises
  // s_ready once the store is complete; the producer warp releases them.
  constexpr uint32_t kPend = 64;
  __shared__ uint32_t s_pend[kPend];
  __shared__ uint32_t s_ready;      // blocks 0 .. s_ready - 1 have complete stores
  __shared__ uint32_t s_npub;       // blocks published so far (producer)
  __shared__ uint32_t s_publock;    // one producer lane publishes at a time
  __shared__ uint32_t s_cons_done;  // the consumers have left their loop
  if (tid == 0) {
    s_ready = s_npub = s_publock = s_cons_done = 0;
    mbar_init(&s_full[0], 1);
    mbar_init(&s_full[1], 1);
    for (int i = 0; i < R; ++i) {
      mbar_init(&s_rfull[i], 1);
      mbar_init(&s_rempty[i], 1);
    }
  }
  mbar_fence_init();
  __syncthreads();
  if (total == 0) return;

  if (wid == NW) {
    // ---------------- producer warp ----------------
    // small packet tables (plain sorts: ten packets) are searched in shared
    // memory instead of global memory
    __shared__ uint32_t s_up[kSchedSmemPackets + 1];
    __shared__ uint64_t s_po[kSchedSmemPackets + 1];
    Tables tbp = tb;
    if (npk <= kSchedSmemPackets) {
      for (uint32_t x = lane; x <= npk; x += 32) {
        s_up[x] = tb.unit_prefix[x];
        s_po[x] = tb.pkt_off[x];
      }
      __syncwarp();
      tbp.unit_prefix = s_up;
      tbp.pkt_off = s_po;
    }
    // TO_HOST, staged order: per packet the first device ticket (its passes
    // 1 .. P-1, pass-major inside the packet) and the first host ticket (its
    // pass P), in packet order
    bool staged = false;
    uint64_t dtotal = total, htotal = 0;
    [[maybe_unused]] uint64_t* s_dpre = nullptr;
    [[maybe_unused]] uint32_t* s_hpre = nullptr;
    if constexpr (TO_HOST) {
      __shared__ uint64_t s_dpre_[kSchedSmemPackets + 1];
      __shared__ uint32_t s_hpre_[kSchedSmemPackets + 1];
      s_dpre = s_dpre_;
      s_hpre = s_hpre_;
      staged = npk <= kSchedSmemPackets;
      if (staged) {
        if (lane == 0) {
          uint64_t d = 0;
          uint32_t h = 0;
          for (uint32_t p = 0; p < npk; ++p) {
            s_dpre[p] = d;
            s_hpre[p] = h;
            const uint32_t n = s_up[p + 1] - s_up[p];
            const int P = min(ceil_log2(n), passes);
            if (P >= 1) {
              d += static_cast<uint64_t>(P - 1) * n;
              h += n;
            }
          }
          s_dpre[npk] = d;
          s_hpre[npk] = h;
        }
        __syncwarp();
        dtotal = s_dpre[npk];
        htotal = s_hpre[npk];
      }
    }
    bool host_mode = staged && blockIdx.x < min(kSchedHostCtas, gridDim.x / 8);
    // Release the CTA's blocks whose stores are complete (any one lane at a
    // time; a lane that finds another one at it moves on).  Consecutive
    // blocks of the same run are added with one release: a release waits
    // for the releasing thread's earlier memory operations and costs about a
    // microsecond under full HBM load.
    auto pub = [&]() {
      if (atomicCAS(&s_publock, 0u, 1u) != 0u) return;
      const uint32_t hi = ld_acquire_cta_shared(&s_ready);
      uint32_t n = *reinterpret_cast<volatile uint32_t*>(&s_npub);
      while (n < hi) {
        const uint32_t sig = s_pend[n % kPend];
        uint32_t c = 1;
        while (n + c < hi && s_pend[(n + c) % kPend] == sig) ++c;
        if (sig != kSigNone) red_release_add(sa.done + sig, c);
        n += c;
      }
      st_release_cta_shared(&s_npub, n);
      atomicExch(&s_publock, 0u);
    };
    uint32_t kp = 0;  // records produced
    bool stop = false;
    while (!stop) {
      uint64_t t0 = 0;
      if constexpr (TO_HOST) {
        uint32_t hm = host_mode ? 1u : 0u;
        if (lane == 0) {
          pub();
          if (!hm) {
            t0 = atomicAdd(reinterpret_cast<unsigned long long*>(sa.ticket), kSchedRound);
            if (staged && t0 >= dtotal) hm = 1;  // device tickets done: on to the host tickets
          }
          if (hm) t0 = atomicAdd(reinterpret_cast<unsigned long long*>(sa.ticket) + 1, kSchedRound);
        }
        host_mode = __shfl_sync(0xffffffffu, hm, 0) != 0;
      } else {
        if (lane == 0) {
          pub();
          t0 = atomicAdd(reinterpret_cast<unsigned long long*>(sa.ticket), kSchedRound);
        }
      }
      t0 = __shfl_sync(0xffffffffu, t0, 0);
      const uint64_t lim = staged ? (host_mode ? htotal : dtotal) : total;
      if (t0 >= lim || *reinterpret_cast<volatile uint32_t*>(tb.err) != 0) break;
      // lanes 4i .. 4i+3 serve ticket t0 + i: two searches of two lanes
      const int i = lane >> 2, q = (lane >> 1) & 1, j = lane & 1;
      const uint64_t t = t0 + static_cast<uint64_t>(i);
      int r = static_cast<int>(t / units) + 1;
      uint32_t u = static_cast<uint32_t>(t % units);
      if constexpr (TO_HOST) {
        if (staged && t < lim) {
          if (host_mode) {  // pass P of the packet
            const uint32_t p = find_pkt(s_hpre, npk, static_cast<uint32_t>(t));
            const uint32_t n = s_up[p + 1] - s_up[p];
            r = min(ceil_log2(n), passes);
            u = s_up[p] + static_cast<uint32_t>(t - s_hpre[p]);
          } else {  // pass 1 + local / n of the packet, unit local % n
            const uint32_t p = find_pre64(s_dpre, npk, t);
            const uint32_t n = s_up[p + 1] - s_up[p];
            const uint64_t local = t - s_dpre[p];
            r = static_cast<int>(local / n) + 1;
            u = s_up[p] + static_cast<uint32_t>(local % n);
          }
        }
      }
      MergeGeom g;
      const bool active = t < lim && merge_geom<TILE>(tbp, npk, u, r, g);
      // the runs of pass r-1 that this block reads, and the counter it publishes
      uint32_t sig = kSigNone;
      const uint32_t* dep0 = nullptr;
      const uint32_t* dep1 = nullptr;
      uint32_t need0 = 0, need1 = 0;
      if (active) {
        const uint32_t p = find_pkt(tbp.unit_prefix, npk, u);
        const uint32_t up0 = tbp.unit_prefix[p], ntiles = tbp.unit_prefix[p + 1] - up0;
        const uint32_t ps = up0 + (((u - up0) >> r) << r);  // first unit of this block's pair
        if (r < g.passes) sig = static_cast<uint32_t>(r) * units + ps;
        if (r > 1) {
          const uint32_t half = 1u << (r - 1);
          const uint32_t endu = up0 + ntiles;
          dep0 = run_counter(sa.done, units, r - 1, ps);
          need0 = min(half, endu - ps);
          if (ps + half < endu) {
            dep1 = run_counter(sa.done, units, r - 1, ps + half);
            need1 = min(half, endu - ps - half);
          }
        }
      }
      const bool lead = (lane & 3) == 0;  // lane 4i: waits, writes ticket i's record
      auto deps_met = [&]() {
        return (!dep0 || ld_acquire_u32(dep0) >= need0) && (!dep1 || ld_acquire_u32(dep1) >= need1);
      };
      auto deps_wait = [&]() {
        bool ok = !dep0 || wait_count(dep0, need0, tb.err, sa.limit_ns, pub);
        if (ok && dep1) ok = wait_count(dep1, need1, tb.err, sa.limit_ns, pub);
        return ok;
      };
      const bool srcw = active && ((g.passes - r + 1) & 1) != 0;  // the buffer holding pass r-1
      // co-ranks of the first (q = 0) and one-past-last (q = 1) output of the
      // selected tickets' blocks, then their records into the ring, densely,
      // in ticket order; false when a ring slot did not free up in time
      auto emit = [&](bool sel) {
        const bool go = active && sel;
        const K* A = ku;
        const K* B = ku;
        uint32_t d = 0, lo = 0, hi = 0;
        if (go) {
          A = (srcw ? kw : ku) + g.pstart + g.a_start;
          B = A + g.a_len;
          d = g.diag0 + (q ? g.cnt : 0u);
          lo = d > g.b_len ? d - g.b_len : 0u;
          hi = min(d, g.a_len);
        }
        lo = group_search<2>(lo, hi, j, lane & ~1,
                             [&](uint32_t m) { return !(__ldcg(B + (d - 1 - m)) < __ldcg(A + m)); });
        const uint32_t i0 = __shfl_sync(0xffffffffu, lo, lane & ~3);
        const uint32_t i1 = __shfl_sync(0xffffffffu, lo, (lane & ~3) + 2);
        const uint32_t amask = __ballot_sync(0xffffffffu, go && lead);
        bool ok = true;
        if (go && lead) {
          const uint32_t k = kp + __popc(amask & ((1u << lane) - 1u));
          const int slot = static_cast<int>(k % R);
          if (!mbar_wait_sleepy(&s_rempty[slot], ((k / R) & 1) ^ 1, tb.err, sa.limit_ns, pub)) {
            ok = false;
          } else {
            MergeRec rec = make_rec(g, srcw, i0, i1);
            if (TO_HOST && r == g.passes) rec.a |= kFinal;
            s_rec[slot] = rec;
            s_sig[slot] = (sa.debug_drop && t == 0) ? kSigNone : sig;
            s_tkt[slot] = 0;
            mbar_arrive(&s_rfull[slot]);
          }
        }
        kp += __popc(amask);
        return !__any_sync(0xffffffffu, !ok);
      };
      // Usually every block of the round can start: all of them together.
      // Otherwise wait only for the earliest ticket not yet handed out, then
      // hand out in one go the run of consecutive tickets from it whose inputs
      // are complete, and repeat: a later ticket of the round may read the
      // runs an earlier one writes, so no wait ever precedes the record of an
      // earlier ticket.
      uint32_t left = __ballot_sync(0xffffffffu, active && lead);  // leads of tickets still to hand out
      while (left && !stop) {
        const int first = __ffs(left) - 1;  // lead lane of the earliest one
        bool ok = true;
        if (lane == first) ok = deps_wait();
        if (__any_sync(0xffffffffu, !ok)) {
          stop = true;
          break;
        }
        const uint32_t met = __ballot_sync(0xffffffffu, ((left >> lane) & 1u) && (lane == first || deps_met()));
        // the ready tickets from `first` on, up to the first one still waiting
        uint32_t run = 0;
        for (int x = first; x < 32; x += 4) {
          if (!((left >> x) & 1u)) continue;  // no block to hand out for this ticket
          if (!((met >> x) & 1u)) break;
          run |= 1u << x;
        }
        if (!emit(((run >> (lane & ~3)) & 1u) != 0)) stop = true;
        left &= ~run;
      }
    }
    // end of the queue (or of this CTA's part after an error)
    if (lane == 0) {
      const int slot = static_cast<int>(kp % R);
      if (mbar_wait_sleepy(&s_rempty[slot], ((kp / R) & 1) ^ 1, tb.err, sa.limit_ns, pub)) {
        s_rec[slot] = MergeRec{0, 0, 0, 0, 0};
        s_sig[slot] = kSigNone;
        s_tkt[slot] = 0x80000000u;
        mbar_arrive(&s_rfull[slot]);
      }
    }
    // the consumers' last blocks: publish until they are done (bounded)
    if (lane == 0) {
      const uint64_t t0 = globaltimer_ns();
      while (!ld_acquire_cta_shared(&s_cons_done)) {
        pub();
        __nanosleep(256);
        if (globaltimer_ns() - t0 > sa.limit_ns) {
          atomicOr(tb.err, kErrTimeout);
          break;
        }
      }
      pub();
    }
    return;
  }

  // ---------------- consumer warps ----------------
  // kc: records consumed; the record of block kc sits in slot kc % R.  A
  // record is read by the consumers only after a consumer barrier that
  // follows warp 0's wait for it.
  uint32_t kc = 0;
  uint32_t par0 = 0, par1 = 0;       // phase parity of each stage's barrier
  bool infl0 = false, infl1 = false;  // warp 0: a copy into the stage is not yet waited for
  bool failed = false;        // every consumer thread: leave the loop (set only by a consumer barrier)
  bool w0_failed = false;     // warp 0: a record did not arrive in time; reported at the next barrier
  // warp 0: the loads of block k into stage st (an end record completes the
  // stage's barrier with nothing to load)
  auto issue = [&](uint32_t k, int st) {
    const int sl = static_cast<int>(k % R);
    __syncwarp();  // lane 0 saw the record arrive: the lanes read it after this
    if (s_tkt[sl] & 0x80000000u) {
      if (lane == 0) mbar_arrive(&s_full[st]);
    } else {
      unsigned char* sb = s_raw + st * SB;
      if (lane == 0) {
        bulk_wait_read0();           // the store staged in this stage has read it
        fence_proxy_async();
        fence_proxy_async_global();  // the inputs were published by other CTAs' bulk stores
      }
      __syncwarp();
      merge_issue<K, HAS_V>(s_rec[sl], reinterpret_cast<K*>(sb), reinterpret_cast<uint32_t*>(sb + KB), &s_full[st], ku,
                            vu, kw, vw, lane);
    }
    if (st) infl1 = true; else infl0 = true;
  };
  // Publication.  Thread 0 issues every store and notes the block's counter
  // index in s_pend; once the store is complete (kPubLag blocks later: a
  // store completes well after the next blocks are merged) it raises
  // s_ready, and the producer warp releases the counters.  A release waits
  // for the releasing thread's earlier memory operations: thread 0 always has
  // the next block's copies in flight, so it never releases itself.
  constexpr uint32_t kPubLag = 6;
  auto note_ready = [&](uint32_t nready) {  // thread 0: blocks 0 .. nready - 1 have complete stores
    fence_proxy_async_global();
    st_release_cta_shared(&s_ready, nready);
  };
  // warp 0: wait for record k, then issue its loads; false when the wait expired
  auto wait_and_issue = [&](uint32_t k) {
    bool ok = true;
    if (lane == 0) ok = mbar_wait_bounded(&s_rfull[k % R], (k / R) & 1, tb.err, sa.limit_ns);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) issue(k, static_cast<int>(k & 1));
    return ok;
  };
  if (wid == 0) w0_failed = !wait_and_issue(0);
  // Every consumer thread runs every iteration up to its barriers: a failure
  // seen by some threads only is carried to the next consumer barrier, which
  // all of them leave together.
  while (!failed) {
    const int s = static_cast<int>(kc & 1);
    const int slot = static_cast<int>(kc % R);
    // warp 0: the next block's loads, if its record is already there (never
    // wait for it here: it may depend on this very block)
    bool issued_next = false;
    if (wid == 0 && !w0_failed) {
      bool rdy = false;
      if (lane == 0) rdy = mbar_try_wait(&s_rfull[(kc + 1) % R], ((kc + 1) / R) & 1);
      rdy = __shfl_sync(0xffffffffu, rdy, 0);
      if (rdy) issue(kc + 1, s ^ 1);
      issued_next = rdy;
    }
    const bool ok = !(wid == 0 && w0_failed) && mbar_wait_bounded(&s_full[s], s ? par1 : par0, tb.err, sa.limit_ns);
    if (ok) {
      if (s) { par1 ^= 1; infl1 = false; } else { par0 ^= 1; infl0 = false; }
    }
    if (consumers_sync_or(!ok, BLOCK)) {
      failed = true;
      break;
    }
    if (s_tkt[slot] & 0x80000000u) break;  // end of the queue
    const MergeRec cur = s_rec[slot];
    const uint32_t cur_sig = s_sig[slot];
    K* rk = reinterpret_cast<K*>(s_raw + s * SB);
    uint32_t* rv = reinterpret_cast<uint32_t*>(s_raw + s * SB + KB);
    const bool srcw = (cur.a & kSrcW) != 0;
    const bool to_host = TO_HOST && !HAS_V && (cur.a & kFinal) != 0;
    const uint64_t a = cur.a & ~(kSrcW | kFinal);
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
    consumers_sync(BLOCK);  // every read of the stage is done: stage the outputs in it
    K* kd = (srcw ? ku : kw) + cur.out;
    uint32_t* vd = HAS_V ? (srcw ? vu : vw) + cur.out : nullptr;
    const uint32_t ok_ph = phase_of(kd);
    const uint32_t ov_ph = HAS_V ? phase_of(vd) : 0u;
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      if (d + j < cnt) {
        rk[ok_ph + d + j] = k[j];
        if constexpr (HAS_V) rv[ov_ph + d + j] = v[j];
      }
    }
    fence_proxy_async();
    consumers_sync(BLOCK);
    if constexpr (TO_HOST) {
      if (to_host) {  // consumer-uniform
        // the block's outputs are final: every consumer thread writes its
        // share of the staged block to the host array by plain coalesced
        // stores, and the stage is read completely before warp 0 refills it
        K* hd = static_cast<K*>(sa.host_out) + cur.out;
        const K* sk = rk + ok_ph;
        if (phase_of(hd) == ok_ph) {
          // same 16-byte phase as the staged block: 16-byte stores for the
          // aligned interior, single elements at the two ends
          const Window w = plan_window<sizeof(K)>(hd, static_cast<uint32_t>(cnt));
          const uint32_t nsingle = w.head + w.tail;
          for (uint32_t x = tid; x < nsingle; x += BLOCK) {
            const uint32_t e = (x < w.head) ? x : static_cast<uint32_t>(cnt) - w.tail + (x - w.head);
            hd[e] = sk[e];
          }
          uint4* hv = reinterpret_cast<uint4*>(hd + w.head);
          const uint4* sv = reinterpret_cast<const uint4*>(sk + w.head);
          for (uint32_t x = tid; x < w.body_bytes / 16; x += BLOCK) hv[x] = sv[x];
        } else {
          for (int x = tid; x < cnt; x += BLOCK) hd[x] = sk[x];
        }
        consumers_sync(BLOCK);
      }
    }
    if (wid == 0) {
      if (cnt > 0 && !to_host) {
        store_window(kd, rk + ok_ph, cnt, lane);
        if constexpr (HAS_V) store_window(vd, rv + ov_ph, cnt, lane);
      }
      __syncwarp();  // the lanes' single-element stores precede lane 0's note of completion
      if (lane == 0) {
        bulk_commit();
        // the slot is free once the producer has published block kc - kPend
        // (it publishes while it waits, so this wait ends)
        if (kc >= kPend) {
          const uint64_t t0 = globaltimer_ns();
          while (ld_acquire_cta_shared(&s_npub) + kPend <= kc) {
            __nanosleep(64);
            if (globaltimer_ns() - t0 > sa.limit_ns) {
              atomicOr(tb.err, kErrTimeout);
              break;
            }
          }
        }
        s_pend[kc % kPend] = cur_sig;
        if (kc >= kPubLag) {
          // all but the last kPubLag stores are complete
          asm volatile("cp.async.bulk.wait_group %0;" ::"n"(kPubLag) : "memory");
          note_ready(kc - kPubLag + 1);
        }
        mbar_arrive(&s_rempty[slot]);  // the record is no longer needed
      }
      ++kc;
      // the next block's loads were not issued above: its record may wait
      // for this very block, so publish it first, then wait for the record
      if (!issued_next) {
        // it usually arrives within moments; if not, publish this block
        // (the record may wait for it) and wait for the record
        bool rdy = false;
        if (lane == 0)
          for (int x = 0; x < 8 && !rdy; ++x) rdy = mbar_try_wait(&s_rfull[kc % R], (kc / R) & 1);
        rdy = __shfl_sync(0xffffffffu, rdy, 0);
        if (rdy) {
          issue(kc, static_cast<int>(kc & 1));
        } else {
          if (lane == 0) {
            bulk_wait0();
            note_ready(kc);  // the producer publishes them while it waits
          }
          __syncwarp();
          if (!wait_and_issue(kc)) w0_failed = true;  // reported at the next consumer barrier
        }
      }
    } else {
      ++kc;
    }
  }
  if (wid == 0) {
    // copies may still be in flight into a stage: bounded waits before the
    // CTA's shared memory is released
    if (infl0) mbar_wait_bounded(&s_full[0], par0, tb.err, sa.limit_ns);
    if (infl1) mbar_wait_bounded(&s_full[1], par1, tb.err, sa.limit_ns);
    if (lane == 0) {
      bulk_wait0();
      if (!failed && !w0_failed) note_ready(kc);
      st_release_cta_shared(&s_cons_done, 1u);  // the producer publishes the rest and leaves
    }
  }
}

// ---------------------------------------------------------------------------
// k_copy_unmerged (host-buffer calls whose last merge passes write to host
// memory): the packets that need no merge pass (at most one tile, sorted by
// the tile sort into U) are copied from U to the caller's host array; one
// CTA per packet, plain coalesced stores.
// ---------------------------------------------------------------------------
template <class K>
__global__ void k_copy_unmerged(const K* __restrict__ ku, K* hout, uint32_t npk, Tables tb) {
  griddep_open();
  for (uint32_t p = blockIdx.x; p < npk; p += gridDim.x) {
    if (tb.unit_prefix[p + 1] - tb.unit_prefix[p] > 1) continue;  // merged: written by its last pass
    const uint64_t b = tb.pkt_off[p], e = tb.pkt_off[p + 1];
    for (uint64_t i = b + threadIdx.x; i < e; i += blockDim.x) hout[i] = ku[i];
  }
}

}  // namespace hs
