// Shared device definitions of the sm_103a sort kernels: key traits, the
// packet rule as the GPU evaluates it, relaxed global loads/stores and the
// bounded wait used by every spin loop.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hs {

constexpr int kWarp = 32;

__host__ __device__ __forceinline__ uint64_t min64(uint64_t a, uint64_t b) { return a < b ? a : b; }

// Device error word bits (one error word per device).
enum : uint32_t {
  kErrTimeout = 1u,     // a bounded wait gave up
  kErrBadOffsets = 2u,  // batch offsets not monotone / not ending at n
  kErrBounds = 4u,      // a computed position fell outside its packet
};

// ---------------------------------------------------------------------------
// Key traits.  U is the unsigned image type the packet step reads digits of.
// ---------------------------------------------------------------------------
template <class K> struct KT;
template <> struct KT<int32_t> {
  using U = uint32_t;
  static constexpr int kBits = 32;
  static __host__ __device__ __forceinline__ int32_t maxv() { return 0x7fffffff; }
  static __device__ __forceinline__ U image(int32_t k, bool flip) {
    return static_cast<uint32_t>(k) ^ (flip ? 0x80000000u : 0u);
  }
  static __device__ __forceinline__ bool negative(int32_t k) { return k < 0; }
};
template <> struct KT<uint32_t> {
  using U = uint32_t;
  static constexpr int kBits = 32;
  static __host__ __device__ __forceinline__ uint32_t maxv() { return 0xffffffffu; }
  static __device__ __forceinline__ U image(uint32_t k, bool) { return k; }
  static __device__ __forceinline__ bool negative(uint32_t) { return false; }
};
template <> struct KT<uint64_t> {
  using U = uint64_t;
  static constexpr int kBits = 64;
  static __host__ __device__ __forceinline__ uint64_t maxv() { return ~0ull; }
  static __device__ __forceinline__ U image(uint64_t k, bool) { return k; }
  static __device__ __forceinline__ bool negative(uint64_t) { return false; }
};

// ---------------------------------------------------------------------------
// Packet rule, GPU form.  A "class" summarises the largest key image of a
// group of keys: for the decimal step it is the digit count D of that image
// (1..20), for the 256-bucket ablation its bit length B (0..64).  Given a
// class, a key's packet is
//   decimal: floor(u / 10^(D-1)),
//   256:     u >> max(0, B - 8).
// ---------------------------------------------------------------------------
constexpr int kDecClasses = 21;  // D = 1..20 (row 0 unused)
constexpr int kBinClasses = 65;  // B = 0..64

__host__ __device__ __forceinline__ uint64_t pow10_u64(int e) {
  uint64_t p = 1;
  for (int i = 0; i < e; ++i) p *= 10ull;
  return p;
}

// Decimal digit count of v: 1 + number of powers 10^k (k >= 1) not above v.
struct Pow10Table {
  uint64_t p[20];
};
__host__ __device__ constexpr Pow10Table make_pow10() {
  Pow10Table t{};
  uint64_t v = 1;
  for (int k = 0; k < 20; ++k) {
    t.p[k] = v;
    v *= 10ull;
  }
  return t;
}
static __constant__ Pow10Table c_pow10 = make_pow10();
__device__ __forceinline__ int dec_class(uint32_t v) {  // 32-bit images: at most 10 digits
  int d = 1;
#pragma unroll
  for (int k = 1; k <= 9; ++k) d += (v >= c_pow10.p[k]) ? 1 : 0;
  return d;
}
__device__ __forceinline__ int dec_class(uint64_t v) {
  int d = 1;
#pragma unroll
  for (int k = 1; k <= 19; ++k) d += (v >= c_pow10.p[k]) ? 1 : 0;
  return d;
}
__device__ __forceinline__ int bin_class(uint32_t v) { return 32 - __clz(v); }
__device__ __forceinline__ int bin_class(uint64_t v) { return 64 - __clzll(v); }

// Everything a kernel needs to evaluate packet(u) for one class.
struct DigitRule {
  uint64_t mult;     // decimal, 32-bit images: ceil(2^64 / 10^(D-1)) (0 when D == 1)
  uint64_t thr[9];   // decimal, 64-bit images: j * 10^(D-1) - 1, saturated at 2^64 - 1
  uint32_t shift;    // 256-bucket: max(0, B - 8)
};

__host__ __device__ constexpr DigitRule rule_dec_c(int D) {
  DigitRule r{};
  uint64_t div = 1;
  for (int i = 1; i < D; ++i) div *= 10ull;
  r.mult = (div == 1) ? 0ull : (~0ull / div) + 1ull;
  const uint64_t lim = ~0ull / div;  // largest j with j * div representable
  for (int j = 1; j <= 9; ++j)
    r.thr[j - 1] = (static_cast<uint64_t>(j) <= lim) ? static_cast<uint64_t>(j) * div - 1ull : ~0ull;
  r.shift = 0;
  return r;
}
struct DecRuleTable {
  DigitRule r[kDecClasses];
};
__host__ __device__ constexpr DecRuleTable make_dec_rules() {
  DecRuleTable t{};
  for (int D = 1; D < kDecClasses; ++D) t.r[D] = rule_dec_c(D);
  return t;
}
// The decimal rules of every digit width, built at compile time (the 64-bit
// divisions they need never run on the device).
static __constant__ DecRuleTable c_dec_rules = make_dec_rules();

__device__ __forceinline__ const DigitRule& rule_dec(int D) { return c_dec_rules.r[D]; }
__device__ __forceinline__ DigitRule make_rule_bin(int B) {
  DigitRule r{};
  r.shift = B > 8 ? static_cast<uint32_t>(B - 8) : 0u;
  return r;
}

// Decimal packet of a 32-bit image: the quotient u / 10^(D-1) by a multiply-
// high with the rounded-up reciprocal m = ceil(2^64 / d) (Granlund &
// Montgomery, PLDI 1994).  For u < 2^32 and d = 10^k <= 10^9 the product's
// error term u * (m - 2^64/d) / 2^64 stays below 2^-32 < 1/d, so the floor is
// exact; the quotient is at most 9 because u < 10^D.
// With m = mh * 2^32 + ml, the high 64 bits of u * m are
// floor((u * mh + floor(u * ml / 2^32)) / 2^32): the dropped low part of u * ml
// is below 2^32 and cannot carry into bit 64.
__device__ __forceinline__ uint32_t packet_dec(uint32_t u, const DigitRule& r) {
  const uint32_t mh = static_cast<uint32_t>(r.mult >> 32), ml = static_cast<uint32_t>(r.mult);
  const uint64_t t = static_cast<uint64_t>(u) * mh + __umulhi(u, ml);
  return r.mult ? static_cast<uint32_t>(t >> 32) : u;
}
// Decimal packet of a 64-bit image: how many of the nine thresholds
// j * 10^(D-1) (j = 1..9) the image reaches.
__device__ __forceinline__ uint32_t packet_dec(uint64_t u, const DigitRule& r) {
  uint32_t p = 0;
#pragma unroll
  for (int j = 0; j < 9; ++j) p += (u > r.thr[j]) ? 1u : 0u;
  return p;
}
__device__ __forceinline__ uint32_t packet_bin(uint32_t u, const DigitRule& r) { return u >> r.shift; }
__device__ __forceinline__ uint32_t packet_bin(uint64_t u, const DigitRule& r) {
  return static_cast<uint32_t>(u >> r.shift);
}

template <int NB, class U>
__device__ __forceinline__ uint32_t packet_of(U u, const DigitRule& r) {
  if constexpr (NB == 10) return packet_dec(u, r);
  else return packet_bin(u, r);
}

// ---------------------------------------------------------------------------
// Relaxed device-scope global accesses for the look-back status words.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Programmatic dependent launch: every kernel of the library opens with
// griddep_open(), which waits until the previous kernel of the stream has
// completed and its memory is visible (a no-op when the launch was not
// programmatic).  The next kernel is released when this one completes.
__device__ __forceinline__ void griddep_open() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Work-space tables shared by the kernels of one call.
struct Tables {
  uint64_t* seg_off;      // nseg + 1 absolute segment starts
  uint32_t* blk_prefix;   // nseg + 1: first packet-step block of each segment
  uint32_t* cls_raw;      // blocks: class of each block's largest key image
  uint32_t* cnt_raw;      // blocks * NB: each block's packet counts under its own class
  uint32_t* flat;         // blocks * NB: counts under the segment class in (segment, packet, block)
                          // order, then scanned in place into absolute first positions
  uint32_t* scan_part;    // scan partials
  uint32_t* seg_neg;      // nseg: segment holds a negative int32 key
  uint32_t* any_neg;      // 1 word: some segment holds a negative int32 key
  uint32_t* pass_ctl;     // [0]: merge passes the largest packet needs; [r]: merge blocks active in pass r
  uint32_t* seg_cmax;     // nseg * 2: largest block class (identity image, flipped image)
  uint32_t* seg_class;    // nseg: final class (D or B) of the segment
  uint32_t* seg_flip;     // nseg: sign flip in use
  uint64_t* pkt_off;      // nseg * NB + 1 absolute packet starts
  uint32_t* unit_prefix;  // nseg * NB + 1: first tile of each packet (tile = merge block)
  uint32_t* small_before; // nseg + 1: keys of short segments (sorted whole by one CTA) before each segment
  uint32_t* small_list;   // nseg: the short segments, in order
  uint32_t* small_cnt;    // 1 word: number of short segments
  uint32_t* err;          // device error word
  int fan_log2;           // log2 of the merge fan-in: 1 (two runs per merge) or 2 (four)
};

// Merge passes a packet of `tiles` sorted tiles needs at fan-in 2^fan_log2:
// ceil(log_F(tiles)) = ceil(ceil(log2(tiles)) / fan_log2) for F = 2, 4.
__host__ __device__ __forceinline__ int passes_of(uint32_t tiles, int fan_log2) {
  int k = 0;
  while (k < 32 && (1ull << k) < tiles) ++k;
  return fan_log2 == 2 ? (k + 1) >> 1 : k;
}

}  // namespace hs
