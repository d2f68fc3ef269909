// Oracle for the hybrid MSD-radix / quicksort / merge sort of Alghamdi &
// Alaghband, "High Performance Parallel Sort for Shared and Distributed Memory
// MIMD" (arXiv 2003.01216).
//
// TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, single-threaded CPU
// restatement of the method, used to check the GPU library.  Only the tests,
// the smoke check and the benchmark's CPU-baseline leg may load it; the GPU
// library neither includes nor links it, and it includes nothing of the GPU
// library.  It follows the paper's steps in the paper's order:
//
//   1. one MSD-radix step: the master divides the keys into ten packets by
//      their most significant decimal digit (Sec. 2.1, Sec. 3.4);
//   2. inside each packet, the data is split among T "threads" (T a power of
//      two, Sec. 3.2) and every part is sorted sequentially by quicksort
//      (Fig. 1(c); or by the non-recursive merge sort of Fig. 1(b));
//   3. the sorted parts are merged pairwise, bottom-up, in a binary tree whose
//      active width halves every round (Sec. 3.2);
//   4. every sorted packet lands at its place in the original array (Sec. 3.4).
//
// Readings taken where the paper is silent (each is also listed in the design
// notes): packets use a fixed digit width D = decimal digits of the largest key
// image, so packet(u) = floor(u / 10^(D-1)); int32 keys are mapped to an
// order-preserving unsigned image (flip the sign bit) only when a negative key
// is present; key-value sorts are stable, ties broken by input index; the last
// part of a packet takes the remainder when T does not divide its length.  A
// 256-bucket variant (bucket = top 8 significant bits of the largest image) is
// the ablation partition; nbuckets = 1 skips the MSD step (the whole array is
// one packet: the shared-memory hybrid of Sec. 3.2 alone).
//
// All arithmetic is integer and exact.

#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>  // std::swap, std::min only

namespace {

enum { DT_INT32 = 0, DT_UINT32 = 1, DT_UINT64 = 2 };
enum { CHUNK_QUICKSORT = 0, CHUNK_MERGESORT = 1 };

// ---------------------------------------------------------------------------
// Records.  A keys-only sort orders plain keys.  A key-value sort orders
// (key, input index) pairs, so equal keys keep their input order (stability).
// ---------------------------------------------------------------------------
template <class K>
struct Rec {
  K key;
  uint32_t val;
  uint32_t idx;
};

template <class K>
inline bool rec_less(const Rec<K>& a, const Rec<K>& b) {
  if (a.key != b.key) return a.key < b.key;
  return a.idx < b.idx;
}
template <class K>
inline bool key_less(const K& a, const K& b) { return a < b; }

template <class T>
struct Less;
template <>
struct Less<int32_t> { bool operator()(int32_t a, int32_t b) const { return a < b; } };
template <>
struct Less<uint32_t> { bool operator()(uint32_t a, uint32_t b) const { return a < b; } };
template <>
struct Less<uint64_t> { bool operator()(uint64_t a, uint64_t b) const { return a < b; } };
template <class K>
struct Less<Rec<K>> { bool operator()(const Rec<K>& a, const Rec<K>& b) const { return rec_less(a, b); } };

template <class K> inline K key_of(const K& k) { return k; }
template <class K> inline K key_of(const Rec<K>& r) { return r.key; }

// ---------------------------------------------------------------------------
// Key image.  The MSD step reads digits of a non-negative integer.  Unsigned
// keys are their own image.  int32 keys are their own image when none is
// negative; otherwise every key is mapped by flipping the sign bit, which is
// order-preserving onto [0, 2^32).
// ---------------------------------------------------------------------------
inline uint64_t image(int32_t k, bool flip) {
  uint32_t u = static_cast<uint32_t>(k);
  if (flip) u ^= 0x80000000u;
  return u;
}
inline uint64_t image(uint32_t k, bool) { return k; }
inline uint64_t image(uint64_t k, bool) { return k; }

template <class K> inline bool is_negative(K) { return false; }
template <> inline bool is_negative<int32_t>(int32_t k) { return k < 0; }

// Number of decimal digits of v (1 for v < 10), by repeated division.
inline uint32_t decimal_digits(uint64_t v) {
  uint32_t d = 1;
  while (v >= 10) {
    v /= 10;
    ++d;
  }
  return d;
}

inline uint64_t pow10u(uint32_t e) {
  uint64_t p = 1;
  for (uint32_t i = 0; i < e; ++i) p *= 10;
  return p;
}

// Number of significant bits of v (0 for v == 0), by repeated shifting.
inline uint32_t bit_length(uint64_t v) {
  uint32_t b = 0;
  while (v) {
    v >>= 1;
    ++b;
  }
  return b;
}

// What the MSD step of one array needs to know about its keys.
struct Digit {
  bool flip = false;     // int32 sign-bit flip in use
  uint32_t width = 0;    // decimal: D (digits of max image); 256: bit length of max image
  uint64_t divisor = 1;  // decimal: 10^(D-1)
  uint32_t shift = 0;    // 256: max(0, width - 8)
  int nbuckets = 10;

  uint32_t bucket(uint64_t u) const {
    if (nbuckets == 1) return 0;  // no MSD step: the whole array is one packet
    if (nbuckets == 10) return static_cast<uint32_t>(u / divisor);
    return static_cast<uint32_t>(u >> shift);
  }
};

template <class K>
Digit plan_digit(const K* keys, uint64_t n, int nbuckets) {
  Digit d;
  d.nbuckets = nbuckets;
  for (uint64_t i = 0; i < n; ++i)
    if (is_negative(keys[i])) d.flip = true;
  uint64_t maxu = 0;
  for (uint64_t i = 0; i < n; ++i) maxu = std::max(maxu, image(keys[i], d.flip));
  if (nbuckets == 10) {
    d.width = decimal_digits(maxu);
    d.divisor = pow10u(d.width - 1);
  } else {
    d.width = bit_length(maxu);
    d.shift = d.width > 8 ? d.width - 8 : 0;
  }
  return d;
}

// ---------------------------------------------------------------------------
// Step 1: one MSD-radix step (Sec. 2.1, Sec. 3.4).  Count the keys of every
// packet, take the exclusive prefix as packet offsets, and move the records
// into their packets in input order (a stable counting scatter).
// ---------------------------------------------------------------------------
template <class K, class R>
void msd_partition(const K* keys, const R* in, R* out, uint64_t n, const Digit& dg,
                   uint64_t* offsets /* nbuckets + 1 */) {
  const int nb = dg.nbuckets;
  std::vector<uint64_t> count(nb, 0);
  for (uint64_t i = 0; i < n; ++i) count[dg.bucket(image(keys[i], dg.flip))]++;
  offsets[0] = 0;
  for (int p = 0; p < nb; ++p) offsets[p + 1] = offsets[p] + count[p];
  std::vector<uint64_t> next(offsets, offsets + nb);
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t p = dg.bucket(image(keys[i], dg.flip));
    out[next[p]++] = in[i];
  }
}

// ---------------------------------------------------------------------------
// Sequential kernels of Sec. 3.1.
// ---------------------------------------------------------------------------

// Merge two sorted lists a[0..na) and b[0..nb) into out; on equal records the
// one from the first (left) list goes first, which keeps merge sort stable.
template <class R>
void merge_two(const R* a, uint64_t na, const R* b, uint64_t nb, R* out) {
  Less<R> lt;
  uint64_t i = 0, j = 0, o = 0;
  while (i < na && j < nb) {
    if (lt(b[j], a[i]))
      out[o++] = b[j++];
    else
      out[o++] = a[i++];
  }
  while (i < na) out[o++] = a[i++];
  while (j < nb) out[o++] = b[j++];
}

// Quicksort of Fig. 1(c) on the half-open range s[lo, hi): choose a pivot V,
// partition around it into S1 (< V) and S2 (> V), sort both.  The pivot is the
// median of the first, middle and last records; records equal to V form a
// third middle block (three-way partition) so runs of equal keys cost O(n).
// The smaller side recurses and the larger side loops, bounding the stack.
template <class R>
void quicksort(R* s, int64_t lo, int64_t hi) {
  Less<R> lt;
  while (hi - lo > 1) {
    int64_t mid = lo + (hi - lo) / 2;
    R a = s[lo], b = s[mid], c = s[hi - 1];
    R v;
    if (lt(a, b)) {
      if (lt(b, c)) v = b; else if (lt(a, c)) v = c; else v = a;
    } else {
      if (lt(a, c)) v = a; else if (lt(b, c)) v = c; else v = b;
    }
    // Dijkstra three-way partition: [lo,l) < v, [l,i) == v, [g,hi) > v.
    int64_t l = lo, i = lo, g = hi;
    while (i < g) {
      if (lt(s[i], v)) {
        std::swap(s[l], s[i]);
        ++l;
        ++i;
      } else if (lt(v, s[i])) {
        --g;
        std::swap(s[i], s[g]);
      } else {
        ++i;
      }
    }
    if (l - lo < hi - g) {
      quicksort(s, lo, l);
      lo = g;
    } else {
      quicksort(s, g, hi);
      hi = l;
    }
  }
}

// Non-recursive merge sort of Fig. 1(b): sort each two elements together,
// then keep merging neighbouring sorted lists, doubling their length, until
// one sorted list remains.
template <class R>
void nonrecursive_mergesort(R* s, uint64_t n) {
  if (n < 2) return;
  std::vector<R> tmp(n);
  R* src = s;
  R* dst = tmp.data();
  for (uint64_t width = 1; width < n; width *= 2) {
    for (uint64_t lo = 0; lo < n; lo += 2 * width) {
      uint64_t m = std::min(lo + width, n), hi = std::min(lo + 2 * width, n);
      merge_two(src + lo, m - lo, src + m, hi - m, dst + lo);
    }
    std::swap(src, dst);
  }
  if (src != s) std::memcpy(s, src, n * sizeof(R));
}

// ---------------------------------------------------------------------------
// Steps 2-3 inside one packet (Sec. 3.2, "Shared-Parallel Hybrid Quicksort and
// Merge Sort"): split the packet among T threads, each sorts its part, then
// merge pairwise in a binary tree until one list holds all the data.  The T
// threads run one after another here; the result does not depend on T.
// ---------------------------------------------------------------------------
template <class R>
void hybrid_sort_packet(R* s, uint64_t len, uint32_t T, int chunk_sort, std::vector<R>& tmp) {
  if (len < 2) return;
  // Part boundaries: T parts of floor(len/T) records, the last one takes the rest.
  std::vector<uint64_t> b(T + 1);
  uint64_t part = len / T;
  for (uint32_t t = 0; t < T; ++t) b[t] = t * part;
  b[T] = len;
  for (uint32_t t = 0; t < T; ++t) {
    if (chunk_sort == CHUNK_QUICKSORT)
      quicksort(s, static_cast<int64_t>(b[t]), static_cast<int64_t>(b[t + 1]));
    else
      nonrecursive_mergesort(s + b[t], b[t + 1] - b[t]);
  }
  // Binary-tree merge: in the round with step w, the thread owning part 2mw
  // merges its list with its neighbour's (part (2m+1)w); half of the threads
  // of the previous round are active.
  if (tmp.size() < len) tmp.resize(len);
  for (uint32_t w = 1; w < T; w *= 2) {
    for (uint32_t m = 0; m + w < T; m += 2 * w) {
      uint64_t lo = b[m], mid = b[m + w], hi = b[std::min<uint32_t>(m + 2 * w, T)];
      merge_two(s + lo, mid - lo, s + mid, hi - mid, tmp.data() + lo);
      std::memcpy(s + lo, tmp.data() + lo, (hi - lo) * sizeof(R));
    }
  }
}

// ---------------------------------------------------------------------------
// The whole method on one array (Sec. 3.4): MSD step, per-packet hybrid sort,
// every packet written back to its place in the original array.
// ---------------------------------------------------------------------------
template <class K>
void sort_keys_impl(K* keys, uint64_t n, int nbuckets, uint32_t T, int chunk_sort,
                    uint64_t* offsets_out) {
  Digit dg = plan_digit(keys, n, nbuckets);
  std::vector<K> packets(n);
  std::vector<uint64_t> off(nbuckets + 1);
  msd_partition(keys, keys, packets.data(), n, dg, off.data());
  std::vector<K> tmp;
  for (int p = 0; p < nbuckets; ++p)
    hybrid_sort_packet(packets.data() + off[p], off[p + 1] - off[p], T, chunk_sort, tmp);
  if (n) std::memcpy(keys, packets.data(), n * sizeof(K));
  if (offsets_out)
    for (int p = 0; p <= nbuckets; ++p) offsets_out[p] = off[p];
}

template <class K>
void sort_pairs_impl(K* keys, uint32_t* vals, uint64_t n, int nbuckets, uint32_t T,
                     int chunk_sort, uint64_t* offsets_out) {
  Digit dg = plan_digit(keys, n, nbuckets);
  std::vector<Rec<K>> recs(n), packets(n);
  for (uint64_t i = 0; i < n; ++i) recs[i] = Rec<K>{keys[i], vals[i], static_cast<uint32_t>(i)};
  std::vector<uint64_t> off(nbuckets + 1);
  msd_partition(keys, recs.data(), packets.data(), n, dg, off.data());
  std::vector<Rec<K>> tmp;
  for (int p = 0; p < nbuckets; ++p)
    hybrid_sort_packet(packets.data() + off[p], off[p + 1] - off[p], T, chunk_sort, tmp);
  for (uint64_t i = 0; i < n; ++i) {
    keys[i] = packets[i].key;
    vals[i] = packets[i].val;
  }
  if (offsets_out)
    for (int p = 0; p <= nbuckets; ++p) offsets_out[p] = off[p];
}

bool valid_args(int dtype, int nbuckets, uint32_t T, int chunk_sort) {
  if (dtype < DT_INT32 || dtype > DT_UINT64) return false;
  if (nbuckets != 1 && nbuckets != 10 && nbuckets != 256) return false;
  if (T == 0 || (T & (T - 1)) != 0) return false;  // power of two (Sec. 3.2)
  if (chunk_sort != CHUNK_QUICKSORT && chunk_sort != CHUNK_MERGESORT) return false;
  return true;
}

template <class K>
void digit_info_impl(const K* keys, uint64_t n, int nbuckets, uint32_t* width, int* flip) {
  Digit dg = plan_digit(keys, n, nbuckets);
  *width = dg.width;
  *flip = dg.flip ? 1 : 0;
}

template <class K>
void partition_impl(const K* keys, const uint32_t* vals, uint64_t n, int nbuckets, K* keys_out,
                    uint32_t* vals_out, uint64_t* offsets) {
  Digit dg = plan_digit(keys, n, nbuckets);
  if (!vals) {
    msd_partition(keys, keys, keys_out, n, dg, offsets);
    return;
  }
  std::vector<Rec<K>> recs(n), out(n);
  for (uint64_t i = 0; i < n; ++i) recs[i] = Rec<K>{keys[i], vals[i], static_cast<uint32_t>(i)};
  msd_partition(keys, recs.data(), out.data(), n, dg, offsets);
  for (uint64_t i = 0; i < n; ++i) {
    keys_out[i] = out[i].key;
    if (vals_out) vals_out[i] = out[i].val;
  }
}

// Sort each run [start, start + tile) of every packet independently (the run
// starts at the packet's first record; the last run of a packet may be
// shorter).  Records keep their order on equal keys.
template <class K>
void tile_sort_impl(K* keys, uint32_t* vals, const uint64_t* offsets, uint64_t npackets,
                    uint64_t tile) {
  for (uint64_t p = 0; p < npackets; ++p) {
    for (uint64_t lo = offsets[p]; lo < offsets[p + 1]; lo += tile) {
      uint64_t hi = std::min(lo + tile, offsets[p + 1]);
      if (!vals) {
        quicksort(keys, static_cast<int64_t>(lo), static_cast<int64_t>(hi));
        continue;
      }
      std::vector<Rec<K>> r(hi - lo);
      for (uint64_t i = lo; i < hi; ++i) r[i - lo] = Rec<K>{keys[i], vals[i], static_cast<uint32_t>(i - lo)};
      quicksort(r.data(), 0, static_cast<int64_t>(r.size()));
      for (uint64_t i = lo; i < hi; ++i) {
        keys[i] = r[i - lo].key;
        vals[i] = r[i - lo].val;
      }
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points.  dtype: 0 = int32, 1 = uint32, 2 = uint64.  nbuckets: 10
// (decimal MSD), 256 (top-8-bit ablation) or 1 (no MSD step).  T: parts per packet, a power of
// two.  chunk_sort: 0 = quicksort (Fig. 1(c)), 1 = non-recursive merge sort
// (Fig. 1(b)).  Every call returns 0 on success, 1 on an invalid argument.
// Pairs carry uint32 values and need n < 2^32.
// ---------------------------------------------------------------------------
extern "C" {

int hso_digit_info(int dtype, const void* keys, uint64_t n, int nbuckets, uint32_t* width,
                   int* flip) {
  if (!valid_args(dtype, nbuckets, 1, 0) || !width || !flip || (n && !keys)) return 1;
  switch (dtype) {
    case DT_INT32: digit_info_impl(static_cast<const int32_t*>(keys), n, nbuckets, width, flip); break;
    case DT_UINT32: digit_info_impl(static_cast<const uint32_t*>(keys), n, nbuckets, width, flip); break;
    default: digit_info_impl(static_cast<const uint64_t*>(keys), n, nbuckets, width, flip); break;
  }
  return 0;
}

// Step 1 alone: the packet layout (records moved stably into their packets)
// and the nbuckets + 1 packet offsets.  vals / vals_out may be null.
int hso_partition(int dtype, const void* keys, const uint32_t* vals, uint64_t n, int nbuckets,
                  void* keys_out, uint32_t* vals_out, uint64_t* offsets) {
  if (!valid_args(dtype, nbuckets, 1, 0) || !offsets || (n && (!keys || !keys_out))) return 1;
  if (vals && n > 0xffffffffull) return 1;
  switch (dtype) {
    case DT_INT32:
      partition_impl(static_cast<const int32_t*>(keys), vals, n, nbuckets, static_cast<int32_t*>(keys_out), vals_out, offsets);
      break;
    case DT_UINT32:
      partition_impl(static_cast<const uint32_t*>(keys), vals, n, nbuckets, static_cast<uint32_t*>(keys_out), vals_out, offsets);
      break;
    default:
      partition_impl(static_cast<const uint64_t*>(keys), vals, n, nbuckets, static_cast<uint64_t*>(keys_out), vals_out, offsets);
      break;
  }
  return 0;
}

// The whole method, in place.  vals null = keys only.  offsets_out (nullable)
// receives the nbuckets + 1 packet offsets.
int hso_sort(int dtype, void* keys, uint32_t* vals, uint64_t n, int nbuckets, uint32_t T,
             int chunk_sort, uint64_t* offsets_out) {
  if (!valid_args(dtype, nbuckets, T, chunk_sort) || (n && !keys)) return 1;
  if (vals && n > 0xffffffffull) return 1;
  switch (dtype) {
    case DT_INT32:
      if (vals) sort_pairs_impl(static_cast<int32_t*>(keys), vals, n, nbuckets, T, chunk_sort, offsets_out);
      else sort_keys_impl(static_cast<int32_t*>(keys), n, nbuckets, T, chunk_sort, offsets_out);
      break;
    case DT_UINT32:
      if (vals) sort_pairs_impl(static_cast<uint32_t*>(keys), vals, n, nbuckets, T, chunk_sort, offsets_out);
      else sort_keys_impl(static_cast<uint32_t*>(keys), n, nbuckets, T, chunk_sort, offsets_out);
      break;
    default:
      if (vals) sort_pairs_impl(static_cast<uint64_t*>(keys), vals, n, nbuckets, T, chunk_sort, offsets_out);
      else sort_keys_impl(static_cast<uint64_t*>(keys), n, nbuckets, T, chunk_sort, offsets_out);
      break;
  }
  return 0;
}

// Segmented form: every segment [offsets[s], offsets[s+1]) is an array of its
// own and goes through the whole method independently.
int hso_sort_batch(int dtype, void* keys, uint32_t* vals, const uint64_t* offsets, uint64_t nseg,
                   int nbuckets, uint32_t T, int chunk_sort) {
  if (!valid_args(dtype, nbuckets, T, chunk_sort) || (nseg && !offsets)) return 1;
  for (uint64_t s = 0; s < nseg; ++s)
    if (offsets[s + 1] < offsets[s]) return 1;
  size_t es = dtype == DT_UINT64 ? 8 : 4;
  for (uint64_t s = 0; s < nseg; ++s) {
    uint64_t lo = offsets[s], len = offsets[s + 1] - offsets[s];
    if (!len) continue;
    char* kp = static_cast<char*>(keys) + lo * es;
    int rc = hso_sort(dtype, kp, vals ? vals + lo : nullptr, len, nbuckets, T, chunk_sort, nullptr);
    if (rc) return rc;
  }
  return 0;
}

// Sorts every tile-long run of every packet on its own (the intermediate
// product of a tiled per-packet sort).  offsets: npackets + 1 entries.
int hso_tile_sort(int dtype, void* keys, uint32_t* vals, const uint64_t* offsets,
                  uint64_t npackets, uint64_t tile) {
  if (dtype < DT_INT32 || dtype > DT_UINT64 || tile == 0 || !offsets) return 1;
  switch (dtype) {
    case DT_INT32: tile_sort_impl(static_cast<int32_t*>(keys), vals, offsets, npackets, tile); break;
    case DT_UINT32: tile_sort_impl(static_cast<uint32_t*>(keys), vals, offsets, npackets, tile); break;
    default: tile_sort_impl(static_cast<uint64_t*>(keys), vals, offsets, npackets, tile); break;
  }
  return 0;
}

}  // extern "C"
