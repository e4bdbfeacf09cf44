// Device-side building blocks of libsrla: recorder stamps, the hash family, the slice
// control block and the open-addressing host sets used to de-duplicate candidates.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "srla.h"

namespace srla {

constexpr uint64_t kP61 = (1ull << 61) - 1;
constexpr unsigned kFull = 0xFFFFFFFFu;

// Candidate sort geometry: a tile of 4096 keys ranked by 16 warps, 8-bit radix digits.
constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kKeysPerWarp = 256;
constexpr int kSortTile = kSortWarps * kKeysPerWarp;  // 4096
constexpr int kRadix = 256;
constexpr size_t kSortSmallSmem = (size_t)kSortTile * sizeof(uint32_t);  // bitonic buffer

// Hash coefficients, one (a, b) per role: rows 0..u-1, SLE cell, SRE cell, sampling.
struct Coef {
  uint64_t a[SRLA_N_HASH];
  uint64_t b[SRLA_N_HASH];
};

// Geometry and per-handle constants, passed by value to every kernel.
struct Geo {
  uint32_t u, v, g, gl;          // rows, columns, SRE and SLE recorders per estimator
  uint32_t vmask, gmask, glmask;  // v-1, g-1, gl-1
  uint32_t k;                     // window in slices
  uint32_t P;                     // stamp modulus 2^z - 1 (= the paper's "too old" distance)
  uint32_t samp_mask;             // LSB(h) >= tau  <=>  (h & samp_mask) == 0
  uint32_t rho_g;                 // ceil(rho * g)
  uint32_t theta;
};

// Slice control block, resident in the workspace.  Kernels read the open slice from here,
// so a captured launch sequence stays valid from slice to slice.
struct Ctl {
  unsigned long long T;           // open slice index
  unsigned int tm;                // T mod P
  unsigned int w_star;            // least w with estimate >= theta (gl + 1 if none)
  unsigned int n_sampled;         // distinct sampled hosts appended in the open slice
  unsigned int n_new;             // of which passed the union SRE test
  unsigned int cat_count[2];      // candidate list length, by slice parity
  unsigned int overflow;          // SRLA overflow bits of the open slice
  unsigned int overflow_next;     // overflow bits raised for the next slice (carry list)
  unsigned int blocks_done;       // blocks of the estimate kernel that have finished
  unsigned int bar_count;         // grid barrier of the cooperative sort: arrivals
  unsigned int bar_gen;           // grid barrier of the cooperative sort: generation
  unsigned int pair_mode;         // 1: the scan consults the per-slice pair table
  unsigned int n_miss;            // block-table misses of the open slice that claimed a pair-table slot
  unsigned int n_gdup;            // of which the per-slice pair table found already scanned
  unsigned int heavy_mode;        // 1: the scan blocks track one heavy host each (HeavyTrack)
  unsigned int sat_hint;          // bit 0 / 1: this slice's census sweep records saturated SLE /
                                  // SRE estimators (the previous slice was nearly saturated)
  double up;                      // UP of Eq. 8 for the open slice (set at its end)
  unsigned long long n_scan;      // pairs of the open slice scanned (their SLE recorders set)
  unsigned long long n_scan_samp; // of which sampled (their SRE recorders set too)
  unsigned long long n_probe;     // sampled-host set insertions tried (one probe load each)
  unsigned long long n_heavy;     // heavy events (three or more sampled lanes of one host in a drain)
  unsigned long long sre_post;    // SRE recorders inside the post-slide window (age + 1 < k), all
                                  // rows; counted only in slices with sat_hint bit 0
  unsigned long long census[SRLA_MAX_ROWS];
};

// Scan counters of a thread (miss, gdup, probe, heavy) or of its warp (scan, samp: the same
// value in every lane), added to the control block once per block.
struct ScanCount {
  uint32_t miss, gdup, scan, samp, probe, heavy;
};

// The pair-table mode of the slice after a slice T that ran with pair_mode and counted n_miss
// claims of which n_gdup were repeats: on while at least a quarter of the claims find
// repeats, and tried again every 16 slices.  The slice close sets it; the host derives the
// same value from the slice's statistics to pick the next scans' build.
__host__ __device__ inline uint32_t next_pair_mode(uint32_t pair_mode, uint64_t n_miss, uint64_t n_gdup, uint64_t T) {
  const bool worth = 4ull * n_gdup >= n_miss;
  return ((pair_mode != 0 && worth) || (T + 1) % 16 == 0) ? 1u : 0u;
}

// The heavy-host mode of the slice after a slice that scanned n_scan pairs and saw n_heavy
// heavy events: heavy events in at least 1/8 of its 32-pair scan drains (n_scan / 32 of
// them).  Set by the slice close, derived by the host as above.
__host__ __device__ inline uint32_t next_heavy_mode(uint64_t n_scan, uint64_t n_heavy) {
  return (n_scan > 0 && 256ull * n_heavy >= n_scan) ? 1u : 0u;
}

// ---------------------------------------------------------------------------- hashing

// One member of the polynomial family, h(x) = (a*x + b) mod (2^61 - 1), low 32 bits.
// a < 2^61 is split as a = ah*2^32 + al so that every product fits in 64 bits:
//   a*x = (ah*x)*2^32 + al*x, and 2^61 = 1 (mod 2^61 - 1).
__device__ __forceinline__ uint32_t hash61(uint64_t a, uint64_t b, uint32_t x) {
  const uint64_t lo = (uint64_t)(uint32_t)a * x;  // < 2^64
  const uint64_t hi = (a >> 32) * x;              // < 2^61
  uint64_t r = (lo & kP61) + (lo >> 61) + (hi >> 29) + ((hi & 0x1FFFFFFFull) << 32) + b;
  r = (r & kP61) + (r >> 61);
  r = (r >= kP61) ? r - kP61 : r;
  return (uint32_t)r;
}

// ------------------------------------------------------------------- recorder stamps
//
// A recorder holds the paper's distance d in [0, P] (Section 3.2) as a stamp code:
// 0 = empty (d = P); otherwise 1 + (slice of the last DRset mod P).  At open slice T with
// tm = T mod P, a code c != 0 has age d = (tm - (c - 1)) mod P.  The sweep at each slice
// end clears the codes whose age would reach P, so ages never alias.

__device__ __forceinline__ uint32_t stamp_age(uint32_t c, uint32_t tm, uint32_t P) {
  int age = (int)tm - (int)c + 1;
  age += (age < 0) ? (int)P : 0;
  return (uint32_t)age;
}


// ------------------------------------------------------------------ one-bit recorders
//
// With z = 1 the window is one slice (k = 1, the discrete window of Section 3.1) and a
// recorder only says whether it was set in the open slice.  Such recorders are packed 32 to a
// 32-bit word: recorder x of an array is bit (x mod 32) of word x / 32; set = DRset in the open
// slice (distance 0), clear = empty (distance 1 = 2^z - 1).  `Bit` selects this storage in the
// templates below; its arrays are only ever addressed as words.
struct Bit {};

template <typename CellT>
inline constexpr bool kIsBit = std::is_same_v<CellT, Bit>;

// 32-bit words holding the run of `cells` recorders of one estimator (runs of fewer than 32
// one-bit recorders share a word and never straddle two).
template <typename CellT>
__host__ __device__ constexpr uint32_t run_words(uint32_t cells) {
  if constexpr (kIsBit<CellT>)
    return cells >= 32u ? cells / 32u : 1u;
  else
    return cells * (uint32_t)sizeof(CellT) / 4u;
}

// Bytes of an array of n recorders.
template <typename CellT>
__host__ __device__ constexpr size_t cell_array_bytes(size_t n) {
  if constexpr (kIsBit<CellT>)
    return n / 8;
  else
    return n * sizeof(CellT);
}

// The recorders from index x of `arr` on (x a multiple of 32 for one-bit storage).
template <typename CellT>
__host__ __device__ inline CellT* cells_from(CellT* arr, size_t x) {
  return reinterpret_cast<CellT*>(reinterpret_cast<char*>(arr) + cell_array_bytes<CellT>(x));
}

// The same, as 32-bit words (x a multiple of 32 recorders, or of 4 bytes of byte cells).
template <typename CellT>
__host__ __device__ inline uint32_t* words_at(CellT* arr, size_t x) {
  return reinterpret_cast<uint32_t*>(cells_from(arr, x));
}

// The stamp a DRset writes in the open slice (tm = T mod P).
template <typename CellT>
__device__ __forceinline__ CellT stamp_code(uint32_t tm) {
  if constexpr (kIsBit<CellT>)
    return CellT{};
  else
    return (CellT)(tm + 1u);
}

// The word holding one-bit recorder idx, as this SM sees it.  Within a slice bits are only
// ever set (the sweep that clears them is another launch), so a bit seen set is set.
template <typename CellT>
__device__ __forceinline__ uint32_t bit_peek(const CellT* arr, size_t idx) {
  return reinterpret_cast<const uint32_t*>(arr)[idx >> 5];
}

// DRset of recorder idx.  Every writer of a slice writes the same stamp, so a plain store
// suffices for byte cells; one-bit recorders share words, so they are set with an atomic OR.
template <typename CellT>
__device__ __forceinline__ void dr_set(CellT* __restrict__ arr, size_t idx, CellT code) {
  if constexpr (kIsBit<CellT>)
    atomicOr(reinterpret_cast<uint32_t*>(arr) + (idx >> 5), 1u << (idx & 31u));
  else
    arr[idx] = code;
}

// The stamps inside the window of the last `lim` slices (ages 0 .. lim-1) are the codes
// 1 + ((tm - j) mod P), j < lim: one cyclic interval of codes ending at hi = tm + 1, either
// [lo, hi] or, when it wraps past P, [lo, P] and [1, hi].  Empty cells (code 0) are never in
// it.  Cells are tested one by one (the per-byte SIMD compare intrinsics are emulated on
// this GPU and cost more).
struct Win {
  uint32_t lo, hi, len;
  bool wrap, none;
};

template <typename CellT>
__device__ __forceinline__ uint32_t splat(uint32_t x) {
  return sizeof(CellT) == 1 ? x * 0x01010101u : x * 0x00010001u;
}

template <typename CellT>
__device__ __forceinline__ Win make_win(uint32_t tm, uint32_t P, uint32_t lim) {
  Win w;
  w.none = lim == 0;
  w.len = lim;
  w.hi = tm + 1u;
  w.wrap = !kIsBit<CellT> && lim > w.hi;
  w.lo = w.wrap ? w.hi + P - lim + 1u : w.hi - lim + 1u;
  return w;
}

// Per-cell mask of a 32-bit word of cells: all ones in the cells inside the window.  Without
// wrap a cell c is inside iff c - lo < len in 32-bit arithmetic (code 0 wraps to a huge value).
template <typename CellT>
__device__ __forceinline__ uint32_t window_mask(uint32_t word, const Win& w) {
  if (w.none) return 0u;
  if constexpr (kIsBit<CellT>) {
    return word;  // a set bit is inside any window of at least one slice
  } else {
    constexpr int kCells = 4 / (int)sizeof(CellT);
    constexpr int kBits = 8 * (int)sizeof(CellT);
    constexpr uint32_t kMask = (1u << kBits) - 1u;
    uint32_t m = 0;
#pragma unroll
    for (int q = 0; q < kCells; q++) {
      const uint32_t c = (word >> (q * kBits)) & kMask;
      const bool in = w.wrap ? (c >= w.lo) | (c - 1u < w.hi) : (c - w.lo < w.len);
      m |= in ? (kMask << (q * kBits)) : 0u;
    }
    return m;
  }
}

// Number of cells set in a sum of popcounts of per-cell masks.
template <typename CellT>
__device__ __forceinline__ uint32_t cells_of_bits(uint32_t bits) {
  if constexpr (kIsBit<CellT>)
    return bits;
  else
    return bits / (8u * (uint32_t)sizeof(CellT));
}

// ------------------------------------------------------------------------- host sets
//
// Open addressing with linear probing over 64-bit slots (tag << 32 | key).  A slot whose
// tag is not the current slice's tag counts as empty, so the tables never need clearing
// between slices (the host clears them when the 31-bit slice tag wraps).

__device__ __forceinline__ uint32_t slice_tag(unsigned long long T) {
  return ((uint32_t)T & 0x7FFFFFFFu) | 0x80000000u;
}

__device__ __forceinline__ uint32_t slot_hash(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7FEB352Du;
  x ^= x >> 15;
  x *= 0x846CA68Bu;
  x ^= x >> 16;
  return x;
}

// Insert key with tag, or find it.  Returns 1 (inserted), 0 (present) or -1 (no free slot
// within the probe bound).  Every failed CAS turns a stale slot current, and a current
// slot never changes within a slice, so the loop is bounded by twice the capacity.
__device__ __forceinline__ int set_insert(unsigned long long* tab, uint32_t mask, uint32_t tag,
                                          uint32_t key, uint32_t* slot_out) {
  const unsigned long long want = ((unsigned long long)tag << 32) | key;
  uint32_t s = slot_hash(key) & mask;
  unsigned long long cur = tab[s];
  const uint32_t limit = 2u * mask + 4u;
  for (uint32_t it = 0; it < limit; it++) {
    if ((uint32_t)(cur >> 32) == tag) {
      if ((uint32_t)cur == key) {
        *slot_out = s;
        return 0;
      }
      s = (s + 1) & mask;
      cur = tab[s];
      continue;
    }
    const unsigned long long old = atomicCAS(tab + s, cur, want);
    if (old == cur) {
      *slot_out = s;
      return 1;
    }
    cur = old;
  }
  return -1;
}

// set_insert continued from a first probe already loaded: slot s holds cur.
__device__ __forceinline__ int set_insert_from(unsigned long long* tab, uint32_t mask, uint32_t tag, uint32_t key,
                                               uint32_t s, unsigned long long cur, uint32_t* slot_out) {
  const unsigned long long want = ((unsigned long long)tag << 32) | key;
  const uint32_t limit = 2u * mask + 4u;
  for (uint32_t it = 0; it < limit; it++) {
    if ((uint32_t)(cur >> 32) == tag) {
      if ((uint32_t)cur == key) {
        *slot_out = s;
        return 0;
      }
      s = (s + 1) & mask;
      cur = tab[s];
      continue;
    }
    const unsigned long long old = atomicCAS(tab + s, cur, want);
    if (old == cur) {
      *slot_out = s;
      return 1;
    }
    cur = old;
  }
  return -1;
}

// Find key with tag; returns the slot or 0xFFFFFFFF.
__device__ __forceinline__ uint32_t set_find(const unsigned long long* tab, uint32_t mask, uint32_t tag,
                                             uint32_t key) {
  uint32_t s = slot_hash(key) & mask;
  for (uint32_t it = 0; it <= mask; it++) {
    const unsigned long long cur = tab[s];
    if ((uint32_t)(cur >> 32) != tag) return 0xFFFFFFFFu;
    if ((uint32_t)cur == key) return s;
    s = (s + 1) & mask;
  }
  return 0xFFFFFFFFu;
}

// ------------------------------------------------------------------------ warp sums

__device__ __forceinline__ uint32_t warp_sum(uint32_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

// |U(aip)|^lim of Algorithm 1 over one recorder array (SRE or SLE): the number of cells j
// whose recorder is inside the window in every row i, i.e. whose DRjoin (max) over the u
// rows is below lim.  One warp per host; lane i < u holds the column of row i in `mycol`.
// Every lane runs the same number of trips (the shuffles need the whole warp).
// kFresh: the words may have been written by the running kernel (inline candidate test), so
// they are read through L2 instead of the read-only path.
template <int WPL, bool kFresh = false>
__device__ __forceinline__ void load_words(const uint32_t* run, uint32_t w0, uint32_t wd[WPL]) {
  if constexpr (WPL == 4) {
    const uint4* p = reinterpret_cast<const uint4*>(run + w0);
    const uint4 q4 = kFresh ? __ldcg(p) : __ldg(p);
    wd[0] = q4.x; wd[1] = q4.y; wd[2] = q4.z; wd[3] = q4.w;
  } else if constexpr (WPL == 2) {
    const uint2* p = reinterpret_cast<const uint2*>(run + w0);
    const uint2 q2 = kFresh ? __ldcg(p) : __ldg(p);
    wd[0] = q2.x; wd[1] = q2.y;
  } else {
    wd[0] = kFresh ? __ldcg(run + w0) : __ldg(run + w0);
  }
}

// Words w0.. of the run of estimator (row i, column c); a one-bit run shorter than a word is
// returned in wd[0], shifted down, to the lane with w0 = 0.
template <typename CellT, int WPL, bool kFresh = false>
__device__ __forceinline__ void load_run(const CellT* __restrict__ arr, uint32_t v, uint32_t cells, uint32_t i,
                                         uint32_t c, uint32_t w0, uint32_t wd[WPL]) {
  const size_t se = (size_t)i * v + c;
  if constexpr (kIsBit<CellT>) {
    const uint32_t* words = reinterpret_cast<const uint32_t*>(arr);
    if (cells >= 32u) {
      load_words<WPL, kFresh>(words + se * (cells / 32u), w0, wd);
    } else {
      const size_t bit = se * cells;
      const uint32_t word = kFresh ? __ldcg(words + (bit >> 5)) : __ldg(words + (bit >> 5));
      wd[0] = (word >> (bit & 31u)) & ((1u << cells) - 1u);
#pragma unroll
      for (int q = 1; q < WPL; q++) wd[q] = 0u;
    }
  } else {
    load_words<WPL, kFresh>(reinterpret_cast<const uint32_t*>(arr + se * cells), w0, wd);
  }
}

// Rows are fetched four at a time, all loads in flight before any is used.
template <typename CellT, int WPL, bool kFresh = false>
__device__ __forceinline__ uint32_t union_count_w(const CellT* __restrict__ arr, uint32_t v, uint32_t cells,
                                                  uint32_t u, uint32_t mycol, const Win& win, int lane) {
  const uint32_t R = run_words<CellT>(cells);
  const uint32_t trips = (R + 32u * WPL - 1) / (32u * WPL);
  uint32_t total = 0;
  for (uint32_t t = 0; t < trips; t++) {
    const uint32_t w0 = (t * 32u + (uint32_t)lane) * WPL;
    const bool ok = w0 < R;
    uint32_t m[WPL];
#pragma unroll
    for (int q = 0; q < WPL; q++) m[q] = 0xFFFFFFFFu;
    for (uint32_t i0 = 0; i0 < u; i0 += 4) {
      uint32_t wd[4][WPL];
#pragma unroll
      for (int r = 0; r < 4; r++) {
        const uint32_t i = i0 + (uint32_t)r;
        const uint32_t c = __shfl_sync(kFull, mycol, (int)(i & 31u));
        if (ok && i < u) load_run<CellT, WPL, kFresh>(arr, v, cells, i, c, w0, wd[r]);
      }
#pragma unroll
      for (int r = 0; r < 4; r++)
        if (ok && i0 + (uint32_t)r < u) {
#pragma unroll
          for (int q = 0; q < WPL; q++) m[q] &= window_mask<CellT>(wd[r][q], win);
        }
    }
    if (ok) {
#pragma unroll
      for (int q = 0; q < WPL; q++) total += __popc(m[q]);
    }
  }
  return cells_of_bits<CellT>(warp_sum(total));
}

template <typename CellT, bool kFresh = false>
__device__ __forceinline__ uint32_t union_count(const CellT* __restrict__ arr, uint32_t v, uint32_t cells,
                                                uint32_t u, uint32_t mycol, const Win& win, int lane) {
  const uint32_t R = run_words<CellT>(cells);
  if (R >= 128) return union_count_w<CellT, 4, kFresh>(arr, v, cells, u, mycol, win, lane);
  if (R >= 64) return union_count_w<CellT, 2, kFresh>(arr, v, cells, u, mycol, win, lane);
  return union_count_w<CellT, 1, kFresh>(arr, v, cells, u, mycol, win, lane);
}

// The count of union_count for H hosts at once (their row loads overlap), for a caller that
// only needs to know whether each reaches `need`: rows are joined one at a time, and a host
// stops as soon as fewer than `need` cells remain inside the window in every row so far (the
// union can only shrink).  A count is exact when it is >= need; below need it is some value
// < need.
template <typename CellT, int WPL, int H, bool kFresh = false>
__device__ __forceinline__ void union_count_atleast_w(const CellT* __restrict__ arr, uint32_t v, uint32_t cells,
                                                      uint32_t u, const uint32_t (&col)[H], const Win& win,
                                                      uint32_t need, int lane, uint32_t (&out)[H]) {
  const uint32_t R = run_words<CellT>(cells);
  const uint32_t w0 = (uint32_t)lane * WPL;
  const bool ok = w0 < R;
  uint32_t m[H][WPL];
  bool live[H];
#pragma unroll
  for (int h = 0; h < H; h++) {
    live[h] = true;
    out[h] = 0;
#pragma unroll
    for (int q = 0; q < WPL; q++) m[h][q] = ok ? 0xFFFFFFFFu : 0u;
  }
  bool any = true;
  for (uint32_t i = 0; i < u && any; i++) {
    uint32_t wd[H][WPL];
#pragma unroll
    for (int h = 0; h < H; h++) {  // every live host's row in flight before any is used
      const uint32_t c = __shfl_sync(kFull, col[h], (int)i);
      if (ok && live[h]) load_run<CellT, WPL, kFresh>(arr, v, cells, i, c, w0, wd[h]);
    }
    any = false;
#pragma unroll
    for (int h = 0; h < H; h++) {
      uint32_t p = 0;
#pragma unroll
      for (int q = 0; q < WPL; q++) {
        if (ok && live[h]) m[h][q] &= window_mask<CellT>(wd[h][q], win);
        p += __popc(m[h][q]);
      }
      if (live[h]) {
        out[h] = cells_of_bits<CellT>(warp_sum(p));
        live[h] = out[h] >= need;
      }
      any |= live[h];
    }
  }
}

// Lane i < u holds the hosts' columns of row i.
template <typename CellT, int H, bool kFresh = false>
__device__ __forceinline__ void union_count_atleast(const CellT* __restrict__ arr, uint32_t v, uint32_t cells,
                                                    uint32_t u, const uint32_t (&col)[H], const Win& win,
                                                    uint32_t need, int lane, uint32_t (&out)[H]) {
  const uint32_t R = run_words<CellT>(cells);
  if (R <= 32) return union_count_atleast_w<CellT, 1, H, kFresh>(arr, v, cells, u, col, win, need, lane, out);
  if (R <= 64) return union_count_atleast_w<CellT, 2, H, kFresh>(arr, v, cells, u, col, win, need, lane, out);
  if (R <= 128) return union_count_atleast_w<CellT, 4, H, kFresh>(arr, v, cells, u, col, win, need, lane, out);
#pragma unroll
  for (int h = 0; h < H; h++) out[h] = union_count<CellT, kFresh>(arr, v, cells, u, col[h], win, lane);
}

template <typename CellT, bool kFresh = false>
__device__ __forceinline__ void union_count_atleast2(const CellT* __restrict__ arr, uint32_t v, uint32_t cells,
                                                     uint32_t u, uint32_t col0, uint32_t col1, const Win& win,
                                                     uint32_t need, int lane, uint32_t& out0, uint32_t& out1) {
  const uint32_t col[2] = {col0, col1};
  uint32_t out[2];
  union_count_atleast<CellT, 2, kFresh>(arr, v, cells, u, col, win, need, lane, out);
  out0 = out[0];
  out1 = out[1];
}

}  // namespace srla
