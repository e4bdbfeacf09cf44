// Device building blocks of the SRLA hot path shared by the single-link and the multi-link
// kernels: the scan of Algorithm 2, the sweep, Eq. 8/9, the candidate filter and the close.
#pragma once

#include <math.h>

#include "device.cuh"

namespace srla {

// ------------------------------------------------------------------------------ scan
//
// Algorithm 2 for one pair, under the order-free candidate rule: DRset the SLE recorder
// selected by bip in each of the u estimators of aip; if LSB(H_S(bip)) >= tau, DRset the
// SRE recorder selected by bip in the same estimators and add aip to the slice's set of
// sampled hosts.  All writers of a slice write the same stamp, so plain stores are
// race-free (Section 4.3 makes the same observation for its bits and recorders).
//
// A pair seen again in the same slice writes exactly the same stamps into exactly the same
// recorders and samples the same host, so it can be skipped.  Each block keeps the pairs it
// scanned last in a small direct-mapped table in shared memory; hot pairs (heavy sources
// talk to few peers) then cost one shared-memory probe instead of u + u/2^tau scattered
// stores that would all land on the same L2 sectors.

constexpr int kSeenLog2 = 14;
constexpr int kSeen = 1 << kSeenLog2;                      // pairs remembered per block (one block per SM)
constexpr unsigned long long kNoPair = ~0ull;              // empty slot; that pair is never cached
constexpr int kScanThreads = 1024;                         // one block per SM shares one table
constexpr int kScanThreadsInline = 256;                    // the inline-test variant (more registers)
constexpr int kPairProbes = 2;                             // probes into the slice's pair table

// Behind the per-block table sits one table of the pairs scanned anywhere on the GPU in the
// open slice (cleared at every slice end).  A pair that missed its block's table claims a
// slot with one compare-and-swap: the first claimant scans the pair, later ones skip it.  A
// pair that finds no slot within kPairProbes probes is simply scanned, so a full table costs
// speed, never correctness.  The table pays off only when pairs repeat across blocks: the
// scan counts block misses and GPU-wide repeats, and the slice close switches the table off
// for the next slice when fewer than a quarter of the misses were repeats (re-trying it
// every 16 slices).
__device__ __forceinline__ uint32_t pair_home(unsigned long long key, uint32_t pmask) {
  return (uint32_t)((key * 0xD6E8FEB86659FD93ull) >> 32) & pmask;
}

// Probes after the first: true if the pair is to be scanned (claimed, or no slot found).
__device__ __forceinline__ bool pair_claim_from(unsigned long long* __restrict__ ptab, uint32_t pmask,
                                                unsigned long long key, uint32_t s) {
#pragma unroll 1
  for (int i = 1; i < kPairProbes; i++) {
    const unsigned long long old = atomicCAS(ptab + s, kNoPair, key);
    if (old == kNoPair) return true;   // first in the slice: scan it
    if (old == key) return false;      // already scanned in this slice
    s = (s + 1) & pmask;
  }
  return true;
}

// Heavy sources.  One host that talks to very many destinations in a slice (a scanner, a
// flood victim, a super point far above the threshold) sends all of its recorder stores to
// the same u runs of g' SLE and g SRE recorders, whose few L2 lines then take them one after
// another.  When the previous slice close saw such a host (heavy_mode), the scan runs its
// heavy build (a separate instantiation, so the plain build carries none of this), in which
// every scan block tracks one heavy host: the first host found filling at least kHeavyLanes of a warp's 32
// scanned pairs.  For that host the block keeps a bitmap of the recorders it has stamped in
// this launch (u*g' + u*g bits in shared memory) and stores each recorder once; a stamped
// recorder keeps the slice's stamp until the slice ends (no other writer changes it), so the
// skipped stores are exact.  The heavy_mode hint comes from the sampled-host insertion,
// which already groups a warp's sampled lanes by host: a group of three or more sampled
// lanes of one host (about 4 of a drain's 32 pairs are sampled at the paper's rate, so such a
// host holds a large share of the slice's scanned pairs) is a heavy event; heavy_mode is set
// for the next slice when heavy events occur in at least 1/8 of the 32-pair scan drains.
// Weaker signals switched the heavy build on for small links whose busiest host has only a
// few hundred pairs, where the tracking costs more than it saves.
constexpr int kHeavyLanes = 4;
constexpr uint32_t kHeavyLeBits = 4096;  // u * g' recorders a block can track
constexpr uint32_t kHeavyReBits = 2048;  // u * g recorders a block can track

struct HeavyTrack {
  unsigned long long host;  // 0: none yet; else (1 << 32) | aip
  uint32_t le[kHeavyLeBits / 32];
  uint32_t re[kHeavyReBits / 32];
};

// True if the geometry's runs fit the block's bitmaps.
__device__ __forceinline__ bool heavy_fits(const Geo& geo) {
  return geo.u * geo.gl <= kHeavyLeBits && geo.u * geo.g <= kHeavyReBits;
}

// Clear the tracking state (all threads of the block; the caller synchronises after).
__device__ __forceinline__ void heavy_reset(HeavyTrack* hv) {
  uint32_t* w = reinterpret_cast<uint32_t*>(hv);
  for (uint32_t x = threadIdx.x; x < sizeof(HeavyTrack) / 4; x += blockDim.x) w[x] = 0u;
}

template <int kLog2 = kSeenLog2>
__device__ __forceinline__ uint32_t seen_slot(unsigned long long key) {
  return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - kLog2));
}

// Full scan of one pair per lane (a dense batch): Algorithm 2's DRsets, and the sampled host
// into the slice's set (one probe per distinct host of the warp, one append counter update
// per warp).  All 32 lanes call it; `ok` marks the lanes that hold a pair.
template <typename CellT, bool kInline = false, bool kElide = false, bool kHeavy = false>
__device__ __forceinline__ unsigned scan_dense(uint32_t aip, uint32_t bip, bool ok, const Geo& geo, const Coef& coef,
                                           CellT code, CellT* __restrict__ re, CellT* __restrict__ le,
                                           Ctl* __restrict__ ctl, unsigned long long* __restrict__ utab,
                                           uint32_t umask, uint32_t* __restrict__ ulist, uint32_t umax, uint32_t tag,
                                           int lane, ScanCount& sc, HeavyTrack* hv) {
  const uint32_t u = geo.u;
  bool samp = false;
  // Heavy-host tracking (the heavy build only: 8/16-bit recorders; hv is non-null when the
  // geometry fits the bitmaps, the same for the whole warp).  Every lane takes part in the
  // ballot and the match (full mask), including the lanes without a pair; only then is the
  // result combined with `ok`.  In the other builds `track` is the constant false.
  bool track = false;
  if constexpr (kHeavy && !kIsBit<CellT> && !kElide && !kInline) {
    if (hv) {
      const unsigned okm = __ballot_sync(kFull, ok);
      const unsigned peers = __match_any_sync(kFull, aip) & okm;
      const bool lead = ok && (peers & ((1u << lane) - 1u)) == 0 && __popc(peers) >= kHeavyLanes;
      if (lead && *reinterpret_cast<volatile unsigned long long*>(&hv->host) == 0ull)
        atomicCAS(&hv->host, 0ull, (1ull << 32) | aip);  // the block's first heavy host wins
      __syncwarp();
      const unsigned long long hh = *reinterpret_cast<volatile unsigned long long*>(&hv->host);
      track = ok && (hh >> 32) != 0ull && (uint32_t)hh == aip;
    }
  }
  if (ok) {
    const uint32_t jl = hash61(coef.a[u], coef.b[u], bip) & geo.glmask;
    const uint32_t jr = hash61(coef.a[u + 1], coef.b[u + 1], bip) & geo.gmask;
    const uint32_t hs = hash61(coef.a[u + 2], coef.b[u + 2], bip);
    samp = (hs & geo.samp_mask) == 0;
    if constexpr (kIsBit<CellT>) {
      // Four rows at a time: their words are read first (all loads in flight), and only
      // the bits not yet set are OR-ed in.  Under heavy sources most bits of a run are set
      // early in the slice; skipping those ORs keeps their hot L2 lines from serialising.
      for (uint32_t i0 = 0; i0 < u; i0 += 4) {
        uint32_t c[4], h[4];
        size_t x[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
          const uint32_t i = i0 + (uint32_t)r;
          c[r] = i < u ? hash61(coef.a[i], coef.b[i], aip) & geo.vmask : 0u;
          x[r] = ((size_t)i * geo.v + c[r]) * geo.gl + jl;
          h[r] = i < u ? bit_peek(le, x[r]) : ~0u;
        }
#pragma unroll
        for (int r = 0; r < 4; r++)
          if (!((h[r] >> (x[r] & 31u)) & 1u)) dr_set<CellT>(le, x[r], code);
        if (samp) {
#pragma unroll
          for (int r = 0; r < 4; r++) {
            const uint32_t i = i0 + (uint32_t)r;
            x[r] = ((size_t)i * geo.v + c[r]) * geo.g + jr;
            h[r] = i < u ? bit_peek(re, x[r]) : ~0u;
          }
#pragma unroll
          for (int r = 0; r < 4; r++)
            if (!((h[r] >> (x[r] & 31u)) & 1u)) dr_set<CellT>(re, x[r], code);
        }
      }
    } else if constexpr (kElide) {
      // Four rows at a time, their cells read first; a cell already holding the slice's
      // stamp 1 + (T mod P) is not written again.  That skip is exact because no cell holds
      // this code when slice T opens: the sweep of the transition into T (the ageing step of
      // Algorithm 3) clears every cell whose code is 1 + (T mod P) (the cells whose distance
      // reaches 2^z - 1), before the census when k < P and after the close when k = P.  So
      // every cell with that code was stamped in slice T by one of its writers, and an equal
      // value, even a stale one from this SM's L1, is current.  Chosen when most pairs are
      // new (the pair table is off): then a good share of the stores would repeat a stamp
      // already there.
      for (uint32_t i0 = 0; i0 < u; i0 += 4) {
        size_t xl[4], xr[4];
        CellT hl[4], hr[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
          const uint32_t i = i0 + (uint32_t)r;
          const uint32_t c = i < u ? hash61(coef.a[i], coef.b[i], aip) & geo.vmask : 0u;
          const size_t se = (size_t)i * geo.v + c;
          xl[r] = se * geo.gl + jl;
          xr[r] = se * geo.g + jr;
          hl[r] = i < u ? le[xl[r]] : code;
          hr[r] = (samp && i < u) ? re[xr[r]] : code;
        }
#pragma unroll
        for (int r = 0; r < 4; r++) {
          if (hl[r] != code) dr_set<CellT>(le, xl[r], code);
          if (hr[r] != code) dr_set<CellT>(re, xr[r], code);
        }
      }
    } else if (track) {
      // the block's heavy host: each of its recorders is stored once per launch (bit i*g'+j
      // of the SLE bitmap, i*g+j of the SRE bitmap, set by a shared-memory atomic OR)
      for (uint32_t i = 0; i < u; i++) {
        const uint32_t c = hash61(coef.a[i], coef.b[i], aip) & geo.vmask;
        const size_t se = (size_t)i * geo.v + c;
        const uint32_t bl = i * geo.gl + jl;
        if (!((atomicOr(&hv->le[bl >> 5], 1u << (bl & 31u)) >> (bl & 31u)) & 1u))
          dr_set<CellT>(le, se * geo.gl + jl, code);
        if (samp) {
          const uint32_t br = i * geo.g + jr;
          if (!((atomicOr(&hv->re[br >> 5], 1u << (br & 31u)) >> (br & 31u)) & 1u))
            dr_set<CellT>(re, se * geo.g + jr, code);
        }
      }
    } else {
#pragma unroll 4
      for (uint32_t i = 0; i < u; i++) {
        const uint32_t c = hash61(coef.a[i], coef.b[i], aip) & geo.vmask;
        const size_t se = (size_t)i * geo.v + c;
        dr_set<CellT>(le, se * geo.gl + jl, code);
        if (samp) dr_set<CellT>(re, se * geo.g + jr, code);
      }
    }
  }
  const unsigned sm = __ballot_sync(kFull, samp);
  if constexpr (kInline) return sm;  // the inline test replaces the set of sampled hosts
  int r = -2;
  if (samp) {
    const unsigned peers = __match_any_sync(sm, aip);
    if ((peers & ((1u << lane) - 1u)) == 0) {
      uint32_t slot;
      sc.probe++;
      sc.heavy += __popc(peers) >= 3 ? 1u : 0u;  // a heavy event (see HeavyTrack)
      r = set_insert(utab, umask, tag, aip, &slot);
      if (r < 0) atomicOr(&ctl->overflow, 1u);
    }
  }
  const unsigned ins = __ballot_sync(kFull, r == 1);
  if (ins) {
    const int first = __ffs(ins) - 1;
    unsigned base = 0;
    if (lane == first) base = atomicAdd(&ctl->n_sampled, (unsigned)__popc(ins));
    base = __shfl_sync(kFull, base, first);
    if (r == 1) {
      const unsigned idx = base + (unsigned)__popc(ins & ((1u << lane) - 1u));
      if (idx < umax)
        ulist[idx] = aip;
      else
        atomicOr(&ctl->overflow, 1u);
    }
  }
  return sm;
}

// ------------------------------------------------------------ inline candidate test
//
// Algorithm 2 as printed (SRLA_MODE_INLINE): right after a sampled pair has updated the SRE,
// its host is tested by its union SRE (Algorithm 1: at least ceil(rho g) cells inside the
// window in every row); if it passes and its super point indicator bit (Section 4.1) is not
// yet set in all of its u estimators, the bits are set and the host enters the open slice's
// candidate set.  Threads race between the test and the set, so a host can pass twice; the
// candidate set keeps one copy.
struct InlineArgs {
  uint32_t* si[2];  // super point indicator bits (low 16 bits of a word) per estimator, by parity
  unsigned long long* ctab[2];
  uint32_t* cflags[2];
  uint32_t* clist[2];
  uint32_t cmask, cmax;
};

// The SI bit of a host: bits 28..31 of the sampling-role hash applied to aip.
__device__ __forceinline__ uint32_t si_bit(const Coef& coef, uint32_t u, uint32_t aip) {
  return hash61(coef.a[u + 2], coef.b[u + 2], aip) >> 28;
}

// Hosts of the lanes in `sm` (sampled, their SRE stores issued), two at a time.
template <typename CellT>
__device__ __forceinline__ void inline_test(unsigned sm, uint32_t aip, const Geo& geo, const Coef& coef,
                                            const CellT* __restrict__ re, const Win& win, Ctl* __restrict__ ctl,
                                            const InlineArgs& ia, int lane) {
  const unsigned long long T = ctl->T;
  const int par = (int)(T & 1);
  const uint32_t tag = slice_tag(T);
  const bool mine = (uint32_t)lane < geo.u;
  while (sm) {
    const int j0 = __ffs(sm) - 1;
    sm &= sm - 1;
    const bool two = sm != 0;
    const int j1 = two ? __ffs(sm) - 1 : j0;
    if (two) sm &= sm - 1;
    const uint32_t a0 = __shfl_sync(kFull, aip, j0), a1 = __shfl_sync(kFull, aip, j1);
    const uint32_t c0 = mine ? hash61(coef.a[lane], coef.b[lane], a0) & geo.vmask : 0u;
    const uint32_t c1 = mine ? hash61(coef.a[lane], coef.b[lane], a1) & geo.vmask : 0u;
    uint32_t n0, n1;
    __syncwarp();  // the warp's own SRE stores are ordered before its reads (through L2)
    union_count_atleast2<CellT, true>(re, geo.v, geo.g, geo.u, c0, c1, win, geo.rho_g, lane, n0, n1);
    for (int h = 0; h < (two ? 2 : 1); h++) {
      const uint32_t a = h ? a1 : a0, c = h ? c1 : c0, n = h ? n1 : n0;
      if (n < geo.rho_g) continue;  // n is the same in every lane
      const uint32_t b = si_bit(coef, geo.u, a);
      uint32_t* w = mine ? ia.si[par] + (size_t)lane * geo.v + c : nullptr;
      const bool set = mine ? ((*w >> b) & 1u) != 0u : true;
      if (__all_sync(kFull, set)) continue;  // USI(aip) has the bit: already a candidate
      if (mine) atomicOr(w, 1u << b);
      if (lane == 0) {
        uint32_t slot;
        const int r = set_insert(ia.ctab[par], ia.cmask, tag, a, &slot);
        if (r == 1) {
          ia.cflags[par][slot] = SRLA_NEW;
          atomicAdd(&ctl->n_new, 1u);
          const unsigned at = atomicAdd(&ctl->cat_count[par], 1u);
          if (at < ia.cmax)
            ia.clist[par][at] = a;
          else
            atomicOr(&ctl->overflow, 2u);
        } else if (r < 0) {
          atomicOr(&ctl->overflow, 2u);
        }
      }
    }
  }
}

// Per-warp work queues in shared memory.  Pairs that miss the block's table go to queue 1;
// 32 at a time they claim their slot in the slice's pair table with every lane busy, and
// the pairs still to be scanned go to queue 2, scanned 32 at a time.  Divergent lanes would
// otherwise pay for the whole scan path whenever any lane of the warp needs it.
constexpr int kQueue = 64;

struct ScanQueues {
  volatile unsigned long long* q1;
  volatile unsigned long long* q2;
  uint32_t n1, n2;  // warp-uniform fill levels, both < 32 between drains
};

__device__ __forceinline__ void queue_push(volatile unsigned long long* q, uint32_t& n, bool pred,
                                           unsigned long long key, int lane) {
  const unsigned m = __ballot_sync(kFull, pred);
  if (pred) q[n + (uint32_t)__popc(m & ((1u << lane) - 1u))] = key;
  n += (uint32_t)__popc(m);
  __syncwarp();
}

// Take the first min(n, 32) entries, one per lane; move the rest to the front.
__device__ __forceinline__ bool queue_take(volatile unsigned long long* q, uint32_t& n, int lane,
                                           unsigned long long& key) {
  const bool ok = (uint32_t)lane < n;
  key = ok ? q[lane] : 0ull;
  const uint32_t rest = n > 32u ? n - 32u : 0u;
  const unsigned long long mv = (uint32_t)lane < rest ? q[32 + lane] : 0ull;
  __syncwarp();
  if ((uint32_t)lane < rest) q[lane] = mv;
  __syncwarp();
  n = rest;
  return ok;
}

template <typename CellT, bool kInline = false, bool kElide = false, bool kHeavy = false>
__device__ __forceinline__ void drain_scan(ScanQueues& Q, ScanCount& sc, const Geo& geo, const Coef& coef,
                                           CellT code, CellT* __restrict__ re, CellT* __restrict__ le,
                                           Ctl* __restrict__ ctl, unsigned long long* __restrict__ utab,
                                           uint32_t umask, uint32_t* __restrict__ ulist, uint32_t umax, uint32_t tag,
                                           int lane, HeavyTrack* hv, const InlineArgs* ia = nullptr,
                                           const Win* win = nullptr) {
  unsigned long long key;
  const uint32_t took = min(Q.n2, 32u);  // pairs of this drain (the same in every lane)
  const bool ok = queue_take(Q.q2, Q.n2, lane, key);
  const uint32_t aip = (uint32_t)(key >> 32);
  const unsigned sm = scan_dense<CellT, kInline, kElide, kHeavy>(aip, (uint32_t)key, ok, geo, coef, code, re, le, ctl,
                                                                 utab, umask, ulist, umax, tag, lane, sc, hv);
  sc.scan += took;            // warp-uniform counts: every lane holds the warp's total
  sc.samp += (uint32_t)__popc(sm);
  if constexpr (kInline) inline_test<CellT>(sm, aip, geo, coef, re, *win, ctl, *ia, lane);
}

template <typename CellT, bool kElide = false, bool kHeavy = false>
__device__ __forceinline__ void drain_claim(ScanQueues& Q, ScanCount& sc, unsigned long long* __restrict__ ptab,
                                            uint32_t pmask, const Geo& geo, const Coef& coef, CellT code,
                                            CellT* __restrict__ re, CellT* __restrict__ le, Ctl* __restrict__ ctl,
                                            unsigned long long* __restrict__ utab, uint32_t umask,
                                            uint32_t* __restrict__ ulist, uint32_t umax, uint32_t tag, int lane,
                                            HeavyTrack* hv) {
  unsigned long long key;
  const bool ok = queue_take(Q.q1, Q.n1, lane, key);
  bool scan = false;
  if (ok) {
    const uint32_t home = pair_home(key, pmask);
    const unsigned long long old = atomicCAS(ptab + home, kNoPair, key);
    bool dup = old == key;
    if (old != kNoPair && !dup) dup = !pair_claim_from(ptab, pmask, key, (home + 1) & pmask);
    scan = !dup;
    sc.miss += 1;
    sc.gdup += dup;
  }
  queue_push(Q.q2, Q.n2, scan, key, lane);
  if (Q.n2 >= 32)
    drain_scan<CellT, false, kElide, kHeavy>(Q, sc, geo, coef, code, re, le, ctl, utab, umask, ulist, umax, tag, lane,
                                             hv);
}

// The block's scan counters into the control block: one shared-memory sum per block, one
// global atomic per nonzero counter.  `acc` (6 words) is zeroed by the caller before a
// barrier that precedes the scan; all threads of the block call this; the caller
// synchronises again before it reuses `acc`.
__device__ __forceinline__ void scan_count_flush(ScanCount sc, Ctl* __restrict__ ctl, unsigned* acc, int lane) {
  // miss, gdup, probe and heavy are per lane; scan and samp are the warp's totals in every lane
  const uint32_t v[6] = {warp_sum(sc.miss), warp_sum(sc.gdup), sc.scan, sc.samp, warp_sum(sc.probe),
                         warp_sum(sc.heavy)};
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < 6; i++)
      if (v[i]) atomicAdd(&acc[i], v[i]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (acc[0]) atomicAdd(&ctl->n_miss, acc[0]);
    if (acc[1]) atomicAdd(&ctl->n_gdup, acc[1]);
    if (acc[2]) atomicAdd(&ctl->n_scan, (unsigned long long)acc[2]);
    if (acc[3]) atomicAdd(&ctl->n_scan_samp, (unsigned long long)acc[3]);
    if (acc[4]) atomicAdd(&ctl->n_probe, (unsigned long long)acc[4]);
    if (acc[5]) atomicAdd(&ctl->n_heavy, (unsigned long long)acc[5]);
  }
}

template <bool kVec>
__device__ __forceinline__ void load_pairs(const uint32_t* __restrict__ pairs, uint64_t n, uint64_t base, int lane,
                                           uint32_t a[4], uint32_t b[4], bool ok[4]) {
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const uint64_t p = base + (uint64_t)h * 64 + (uint64_t)lane * 2;
    if (kVec && p + 1 < n) {
      const uint4 q = __ldcs(reinterpret_cast<const uint4*>(pairs) + (p >> 1));
      a[2 * h] = q.x; b[2 * h] = q.y; a[2 * h + 1] = q.z; b[2 * h + 1] = q.w;
      ok[2 * h] = true; ok[2 * h + 1] = true;
    } else {
      ok[2 * h] = p < n;
      ok[2 * h + 1] = p + 1 < n;
      a[2 * h] = ok[2 * h] ? pairs[2 * p] : 0u;
      b[2 * h] = ok[2 * h] ? pairs[2 * p + 1] : 0u;
      a[2 * h + 1] = ok[2 * h + 1] ? pairs[2 * p + 2] : 0u;
      b[2 * h + 1] = ok[2 * h + 1] ? pairs[2 * p + 3] : 0u;
    }
  }
}

// ------------------------------------------------------------- sweep and row census
//
// Census (Section 4.2): count the SLE recorders of a row inside the window at the open slice
// (age < k).  Reset: clear the stamps whose age would reach P after the slide, i.e. the code
// 1 + ((T + 1) mod P); this is the DRslide of Algorithm 3 at the point where a distance
// saturates at 2^z - 1.
// The in-window stamps of the sweep: [lo, hi] (lo + len = hi + 1), or [lo, P] and [1, hi]
// when the window wraps past P.
struct SweepWin {
  uint32_t lo, hi, len;
  bool wrap;
};

template <typename CellT>
__device__ __forceinline__ SweepWin make_sweep_win(uint32_t tm, uint32_t P, uint32_t k) {
  SweepWin sw;
  sw.hi = tm + 1u;
  sw.wrap = k > sw.hi;
  sw.lo = sw.wrap ? sw.hi + P - k + 1u : sw.hi - k + 1u;
  sw.len = k;
  return sw;
}

// In-window cells of one 32-bit word (the interval form of the window, one compare per cell;
// the SIMD compare intrinsics are slower here).  Without wrap, a cell c is inside iff
// c - lo < len in 32-bit arithmetic (the empty code 0 wraps to a huge value).  kWrap fixes
// the form at compile time (the caller picks the loop once), so the cell loop carries one
// form only.
template <typename CellT, bool kWrap>
__device__ __forceinline__ uint32_t count_in_window(uint32_t word, const SweepWin& sw) {
  if constexpr (kIsBit<CellT>) {
    return (uint32_t)__popc(word);  // the window is the open slice
  } else {
    constexpr int kCells = 4 / (int)sizeof(CellT);
    constexpr int kBits = 8 * (int)sizeof(CellT);
    constexpr uint32_t kMask = (1u << kBits) - 1u;
    uint32_t n = 0;
#pragma unroll
    for (int q = 0; q < kCells; q++) {
      const uint32_t c = (word >> (q * kBits)) & kMask;
      n += kWrap ? (uint32_t)((c >= sw.lo) | (c - 1u < sw.hi)) : (uint32_t)(c - sw.lo < sw.len);
    }
    return n;
  }
}

// Nonzero iff some cell of the word equals the splatted stamp (exact zero-cell test).
template <typename CellT>
__device__ __forceinline__ uint32_t has_stamp(uint32_t word, uint32_t asplat) {
  if constexpr (kIsBit<CellT>) return word;  // every set bit carries the open slice's stamp
  const uint32_t x = word ^ asplat;
  return sizeof(CellT) == 1 ? ((x - 0x01010101u) & ~x & 0x80808080u) : ((x - 0x00010001u) & ~x & 0x80008000u);
}

template <typename CellT>
__device__ __forceinline__ uint32_t clear_stamp(uint32_t word, uint32_t alias) {
  if constexpr (kIsBit<CellT>) return 0u;
  constexpr int kCells = 4 / (int)sizeof(CellT);
  constexpr int kBits = 8 * (int)sizeof(CellT);
  constexpr uint32_t kMask = (1u << kBits) - 1u;
#pragma unroll
  for (int q = 0; q < kCells; q++)
    if (((word >> (q * kBits)) & kMask) == alias) word &= ~(kMask << (q * kBits));
  return word;
}

// Returns the number of cells of the vector inside the window (0 when not counting).
template <typename CellT, bool kWrap>
__device__ __forceinline__ uint32_t sweep_vec(uint4* base, size_t x, uint4 q, bool count, bool reset,
                                              const SweepWin& sw, uint32_t alias, uint32_t asplat) {
  const uint32_t n4 = count ? count_in_window<CellT, kWrap>(q.x, sw) + count_in_window<CellT, kWrap>(q.y, sw) +
                                  count_in_window<CellT, kWrap>(q.z, sw) + count_in_window<CellT, kWrap>(q.w, sw)
                            : 0u;
  if (reset && (has_stamp<CellT>(q.x, asplat) | has_stamp<CellT>(q.y, asplat) | has_stamp<CellT>(q.z, asplat) |
                has_stamp<CellT>(q.w, asplat))) {
    uint4 r;
    r.x = clear_stamp<CellT>(q.x, alias);
    r.y = clear_stamp<CellT>(q.y, alias);
    r.z = clear_stamp<CellT>(q.z, alias);
    r.w = clear_stamp<CellT>(q.w, alias);
    base[x] = r;
  }
  return n4;
}

// Saturated estimators.  While it counts, the sweep also records, one byte per estimator
// (row i, column c) of the array, whether all of its recorders are inside the counted
// window (SLE: the census window; SRE: the post-slide window of the carry test).  A host
// whose u estimators are all saturated has a union count equal to the run length, so the
// estimate and the carry test need not gather its recorders.  Recorded when a run is a
// power-of-two number spv <= 32 of 16-byte vectors and the row is a whole number of warps'
// vectors: then each warp step of the sweep covers 32/spv whole runs, and the first lane of
// each run writes its byte (every byte is rewritten at every sweep, so no clearing).  `vx` is
// this lane's vector index within the row; all 32 lanes of the warp call it together.
template <typename CellT>
__device__ __forceinline__ void sat_mark(uint8_t* __restrict__ sat_row, uint32_t spv, size_t vx, uint32_t n4) {
  constexpr uint32_t kCellsPerVec = 16u / (uint32_t)sizeof(CellT);
  const unsigned full = __ballot_sync(kFull, n4 == kCellsPerVec);
  const uint32_t lane = threadIdx.x & 31u;
  if ((lane & (spv - 1u)) == 0u) {
    const uint32_t m = spv == 32u ? kFull : ((1u << spv) - 1u);
    sat_row[vx / spv] = ((full >> lane) & m) == m ? 1u : 0u;
  }
}

// One block's part of one row: grid-stride over the row's vectors from `x`, four loads in
// flight per thread.  kSat: also record the row's saturated-estimator bytes in sat_row (see
// sat_mark; a separate instantiation, so the plain sweep carries none of it); vbase is the
// row index of base[0], in vectors.
template <typename CellT, bool kWrap, bool kSat>
__device__ __forceinline__ uint32_t sweep_part(uint4* base, size_t nvec, size_t x, size_t stride, bool count,
                                               bool reset, const SweepWin& sw, uint32_t alias, uint32_t asplat,
                                               uint8_t* sat_row, uint32_t spv, size_t vbase) {
  uint32_t cnt = 0;
  for (; x + 3 * stride < nvec; x += 4 * stride) {
    uint4 q[4];
#pragma unroll
    for (int j = 0; j < 4; j++) q[j] = base[x + j * stride];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const uint32_t n4 = sweep_vec<CellT, kWrap>(base, x + j * stride, q[j], count, reset, sw, alias, asplat);
      cnt += n4;
      if constexpr (kSat && !kIsBit<CellT>) sat_mark<CellT>(sat_row, spv, vbase + x + j * stride, n4);
    }
  }
  for (; x < nvec; x += stride) {
    const uint32_t n4 = sweep_vec<CellT, kWrap>(base, x, base[x], count, reset, sw, alias, asplat);
    cnt += n4;
    if constexpr (kSat && !kIsBit<CellT>) sat_mark<CellT>(sat_row, spv, vbase + x, n4);
  }
  return cnt;
}

// The four forms of sweep_part (window wrapped or not, saturated-estimator bytes or not).
template <typename CellT>
__device__ __forceinline__ uint32_t sweep_any(uint4* base, size_t nvec, size_t x, size_t stride, bool count,
                                              bool reset, const SweepWin& sw, uint32_t alias, uint32_t asplat,
                                              uint8_t* sat_row, uint32_t spv, size_t vbase) {
  if (sat_row)
    return sw.wrap ? sweep_part<CellT, true, true>(base, nvec, x, stride, count, reset, sw, alias, asplat, sat_row, spv,
                                                   vbase)
                   : sweep_part<CellT, false, true>(base, nvec, x, stride, count, reset, sw, alias, asplat, sat_row,
                                                    spv, vbase);
  return sw.wrap ? sweep_part<CellT, true, false>(base, nvec, x, stride, count, reset, sw, alias, asplat, nullptr, 0, 0)
                 : sweep_part<CellT, false, false>(base, nvec, x, stride, count, reset, sw, alias, asplat, nullptr, 0,
                                                   0);
}

// Hint for the next slice's sweep: record saturated estimators when at least 15/16 of the
// SLE recorders of every row (bit 0), or of all SRE recorders in the post-slide window with
// k < 2^z - 1 (bit 1), were inside the window in this slice.
__device__ __forceinline__ uint32_t sat_hint_of(const Geo& geo, const Ctl& c) {
  unsigned long long min_census = ~0ull;
  for (uint32_t i = 0; i < geo.u; i++) min_census = min(min_census, c.census[i]);
  const bool le = 16ull * min_census >= 15ull * geo.v * geo.gl;
  const bool re = geo.k != geo.P && 16ull * c.sre_post >= 15ull * geo.u * geo.v * geo.g;
  return (le ? 1u : 0u) | (re ? 2u : 0u);
}

// True if every estimator of the host (lane i < u holds its column of row i) is marked
// saturated in the byte map `sat` (u rows of v bytes).  All lanes call it.
__device__ __forceinline__ bool host_saturated(const uint8_t* __restrict__ sat, uint32_t v, uint32_t u,
                                               uint32_t mycol, int lane) {
  const bool mine = (uint32_t)lane < u;
  const bool s = !mine || __ldcg(sat + (size_t)lane * v + mycol) != 0;
  return __all_sync(kFull, s);
}

// The same test for the host `aip` of this lane alone (its u estimators' bytes, all loads in
// flight), so that a warp tests the hosts of a whole run of candidates at once.
__device__ __forceinline__ bool own_host_saturated(const uint8_t* __restrict__ sat, const Geo& geo, const Coef& coef,
                                                   uint32_t aip) {
  uint32_t all = 1u;
#pragma unroll 4
  for (uint32_t i = 0; i < geo.u; i++)
    all &= __ldcg(sat + (size_t)i * geo.v + (hash61(coef.a[i], coef.b[i], aip) & geo.vmask)) != 0 ? 1u : 0u;
  return all != 0u;
}

// ---------------------------------------------------------------- state export
//
// Recorder stamps -> the paper's distances (2^z - 1 = empty), at the open slice: the
// checkpoint form of the recorders (single links and group links).
template <typename CellT>
__global__ void k_decode(const CellT* __restrict__ cells, uint16_t* __restrict__ out, size_t n,
                         const Ctl* __restrict__ ctl, uint32_t P) {
  const uint32_t tm = ctl->tm;
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x) {
    if constexpr (kIsBit<CellT>) {
      const uint32_t word = reinterpret_cast<const uint32_t*>(cells)[x >> 5];
      out[x] = (uint16_t)(((word >> (x & 31u)) & 1u) ? 0u : P);
    } else {
      const uint32_t c = cells[x];
      out[x] = (uint16_t)(c == 0 ? P : stamp_age(c, tm, P));
    }
  }
}

// ------------------------------------------------------------- Eq. 8 and Eq. 9 (b2)
//
// UP = prod_i |LDR(i)|^k / (g' v) from the row census, and Eq. 9 for a union weight w, both
// in FP64; the estimate is rounded once to FP32 when reported.  Edges: w <= g' UP gives 0;
// w = g' or UP = 1 gives +inf (saturated).  The super point decision (estimate >= theta,
// Definition 2) is taken in FP64.
__device__ __forceinline__ double slice_up(const Geo& geo, const Ctl* ctl) {
  const double cells = (double)geo.gl * (double)geo.v;
  double up = 1.0;
  for (uint32_t i = 0; i < geo.u; i++) up *= (double)ctl->census[i] / cells;
  return up;
}

__device__ __forceinline__ double eq9(uint32_t w, uint32_t gl, double up, uint32_t theta, uint32_t* flags) {
  const double g = (double)gl;
  if (w == gl || up >= 1.0) {
    *flags = SRLA_SATURATED | SRLA_SUPER;
    return INFINITY;
  }
  *flags = 0;
  if ((double)w <= g * up) return 0.0;
  const double est = -g * log(1.0 - ((double)w - g * up) / (g * (1.0 - up)));
  if (est >= (double)theta) *flags = SRLA_SUPER;
  return est;
}

// A host that passes the union SRE test enters the open slice's candidate set (or, if it
// was carried in, gains the NEW flag).
__device__ __forceinline__ void filter_admit(Ctl* ctl, unsigned long long* ctab, uint32_t* cflags, uint32_t cmask,
                                             uint32_t* clist, uint32_t cmax, int par, uint32_t tag, uint32_t aip,
                                             bool pass) {
  if (!pass) return;
  atomicAdd(&ctl->n_new, 1u);
  uint32_t slot;
  const int r = set_insert(ctab, cmask, tag, aip, &slot);
  if (r == 1) {
    cflags[slot] = SRLA_NEW;
    const unsigned at = atomicAdd(&ctl->cat_count[par], 1u);
    if (at < cmax)
      clist[at] = aip;
    else
      atomicOr(&ctl->overflow, 2u);
  } else if (r == 0) {
    atomicOr(&cflags[slot], SRLA_NEW);
  } else {
    atomicOr(&ctl->overflow, 2u);
  }
}

// ------------------------------------------------------------------ close the slice
//
// Statistics of the closed slice T, then the control block opens slice T+1: stamp phase
// advanced, per-slice counters cleared, the candidate list of T emptied (the carried list of
// T+1 stays), and the pair-table policy for T+1 chosen from T's counts (kept on while it
// finds repeats for at least a quarter of the block misses; re-tried every 16 slices).
// Every field is loaded before anything is written, so the single closing thread waits for
// one round trip, not one per field.
__device__ __forceinline__ void close_slice(const Geo& geo, Ctl* __restrict__ ctl, srla_slice_stats* __restrict__ st,
                                            uint32_t umax, uint32_t cmax) {
  const Ctl c = *ctl;
  const unsigned long long T = c.T;
  const int par = (int)(T & 1);
  srla_slice_stats s;
  s.slice = T;
  s.n_pkts = 0;
  s.n_sampled = min(c.n_sampled, umax);
  s.n_new = c.n_new;
  s.n_candidates = min(c.cat_count[par], cmax);
  s.n_carry_out = min(c.cat_count[par ^ 1], cmax);
  s.w_star = min(c.w_star, geo.gl + 1u);
  s.overflow = c.overflow;
  s.up = c.up;
  s.pair_table = c.pair_mode;
  s.n_claims = c.n_miss;
  s.n_claim_repeats = c.n_gdup;
  s.n_scanned = c.n_scan;
  s.n_scanned_sampled = c.n_scan_samp;
  s.n_set_probes = c.n_probe;
  s.heavy_hosts = c.heavy_mode;
  s.n_heavy_events = c.n_heavy;
  Ctl n = c;
  for (int i = 0; i < SRLA_MAX_ROWS; i++) {
    s.census[i] = c.census[i];
    n.census[i] = 0;
  }
  *st = s;
  n.T = T + 1;
  n.tm = (c.tm + 1u == geo.P) ? 0u : c.tm + 1u;
  n.n_sampled = 0;
  n.n_new = 0;
  n.cat_count[par] = 0;
  n.overflow = c.overflow_next;
  n.overflow_next = 0;
  n.blocks_done = 0;
  n.bar_count = 0;
  n.w_star = geo.gl + 1u;
  n.pair_mode = next_pair_mode(c.pair_mode, c.n_miss, c.n_gdup, T);
  n.n_miss = 0;
  n.n_gdup = 0;
  n.n_scan = 0;
  n.n_scan_samp = 0;
  n.n_probe = 0;
  n.heavy_mode = next_heavy_mode(c.n_scan, c.n_heavy);
  n.n_heavy = 0;
  n.sat_hint = sat_hint_of(geo, c);
  n.sre_post = 0;
  *ctl = n;
  __threadfence();
}

}  // namespace srla
