// Host-side helpers shared by the single-link and the multi-link C ABI: parameter checks,
// the workspace layout of one link, and the constants of Eq. 1 and Section 3.2.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "device.cuh"

namespace srla {
namespace host {

inline constexpr size_t kAlign = 256;
inline constexpr uint32_t kPrefetch = 2048;  // report entries copied with the slice's header
inline constexpr uint32_t kStateMagic = 0x53524C41u;  // "SRLA"
inline constexpr uint32_t kStateVersion = 1;

inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Header of an exported state (single links and group links): the geometry, the open slice
// and the number of carried hosts, followed by the SRE distances (u*v*g uint16), the SLE
// distances (u*v*gl uint16) and the carried hosts (n_carry uint32, ascending).
struct StateHeader {
  uint32_t magic, version;
  uint32_t u, v, g, gl, dr_bytes, z, k, theta;
  uint64_t slice;
  uint32_t n_carry, pad;
};

inline size_t state_bytes_of(const srla_params* p, uint32_t n_carry) {
  return sizeof(StateHeader) + (size_t)p->u * p->v * (p->g + p->gl) * 2 + (size_t)n_carry * 4;
}

inline bool pow2(uint64_t x) { return x && !(x & (x - 1)); }

inline uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

struct Layout {
  size_t ctl, re, le, staging, utab, ulist, ctab[2], cflags[2], clist[2], sort_tmp, sort_hist, lut_est,
      lut_flags, rep_stats[2], rep_entries[2], ptab[2], si[2], le_sat, re_sat, total;
  uint32_t le_spv, re_spv;  // 16-byte vectors per SLE / SRE run when the sweep records
                            // saturated estimators (one byte each, u*v per array); 0: not recorded
  uint64_t staging_pkts;
  uint32_t umask, cmask, ntiles, pmask;
  bool pairs;   // per-slice pair table present
  int n_ptab;   // pair tables: 2 (by slice parity), 1, or 0
};

// Eq. 1 on integers: the least n >= 0 with g * 2^n >= theta.
inline uint32_t tau_of(uint32_t theta, uint32_t g) {
  uint32_t n = 0;
  while ((uint64_t)g << n < (uint64_t)theta) n++;
  return n;
}

// ceil(rho * g) with rho = 0.99 (1 - e^{-1/3}) (Section 3.2), evaluated in FP64.
inline uint32_t rho_g_of(uint32_t g) { return (uint32_t)std::ceil(0.99 * (1.0 - std::exp(-1.0 / 3.0)) * (double)g); }

// Bytes of `cells` recorders: dr_bytes each, or one bit each when dr_bytes = 0.
inline size_t recorder_bytes(const srla_params* p, uint64_t cells) {
  return p->dr_bytes ? (size_t)cells * p->dr_bytes : (size_t)(cells / 8);
}

inline int check(const srla_params* p) {
  if (!p) return SRLA_E_INVAL;
  if (p->u < 1 || p->u > SRLA_MAX_ROWS) return SRLA_E_INVAL;
  if (!pow2(p->v) || !pow2(p->g) || !pow2(p->gl)) return SRLA_E_INVAL;
  if (p->dr_bytes > 2) return SRLA_E_INVAL;
  if (p->z < 1 || p->z > (p->dr_bytes ? 8 * p->dr_bytes : 1u)) return SRLA_E_INVAL;
  const uint32_t P = (1u << p->z) - 1u;
  if (p->k < 1 || p->k > P) return SRLA_E_INVAL;
  if (p->theta < 1) return SRLA_E_INVAL;
  if (p->dr_bytes && ((uint64_t)p->g * p->dr_bytes < 4 || (uint64_t)p->gl * p->dr_bytes < 4)) return SRLA_E_INVAL;
  if (!p->dr_bytes && (p->g < 4 || p->gl < 4)) return SRLA_E_INVAL;
  // every row of recorders is a whole number of 16-byte vectors
  if (recorder_bytes(p, (uint64_t)p->v * p->g) < 16 || recorder_bytes(p, (uint64_t)p->v * p->gl) < 16)
    return SRLA_E_INVAL;
  if ((uint64_t)p->v * p->gl > (1ull << 40) || (uint64_t)p->v * p->g > (1ull << 40)) return SRLA_E_INVAL;
  if (p->gl > (1u << 24)) return SRLA_E_INVAL;
  if (p->max_sampled < 1 || p->max_sampled > (1u << 30)) return SRLA_E_INVAL;
  if (p->max_candidates < 1 || p->max_candidates > (1u << 26)) return SRLA_E_INVAL;
  if (p->pair_slots_log2 != 0 && p->pair_slots_log2 != -1 && (p->pair_slots_log2 < 10 || p->pair_slots_log2 > 28))
    return SRLA_E_INVAL;
  if (p->mode != SRLA_MODE_ORDER_FREE && p->mode != SRLA_MODE_INLINE) return SRLA_E_INVAL;
  for (uint32_t r = 0; r < p->u + 3; r++) {
    if (p->hash_a[r] < 1 || p->hash_a[r] >= kP61) return SRLA_E_INVAL;
    if (p->hash_b[r] >= kP61) return SRLA_E_INVAL;
  }
  return SRLA_OK;
}

// Vectors of 16 bytes per run of `cells` 8/16-bit recorders when the sweep can record the
// saturated estimators of an array (the run is a power of two of at most 32 vectors and a row
// is a whole number of 32-vector warp steps), else 0.
inline uint32_t sat_spv(const srla_params* p, uint32_t cells) {
  if (!p->dr_bytes) return 0;
  const uint64_t bytes = (uint64_t)cells * p->dr_bytes;
  if (bytes % 16 || bytes / 16 == 0 || bytes / 16 > 32) return 0;
  const uint32_t spv = (uint32_t)(bytes / 16);
  return ((uint64_t)p->v * spv) % 32 == 0 ? spv : 0;
}

// n_pair_tables: 2 for a single link (the next slice's table is cleared while one slice is
// closed), 1 for a group link (the group sweep clears it).
inline Layout layout_of(const srla_params* p, int n_pair_tables = 2) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  L.staging_pkts = p->staging_pkts ? std::max<uint64_t>(p->staging_pkts, 8) : (1ull << 20);
  const uint64_t ucap = std::max<uint64_t>(64, next_pow2(2ull * p->max_sampled));
  const uint64_t ccap = std::max<uint64_t>(64, next_pow2(2ull * p->max_candidates));
  L.umask = (uint32_t)(ucap - 1);
  L.cmask = (uint32_t)(ccap - 1);
  L.ntiles = (p->max_candidates + kSortTile - 1) / kSortTile;
  L.ctl = take(sizeof(Ctl));
  L.re = take(recorder_bytes(p, (uint64_t)p->u * p->v * p->g));
  L.le = take(recorder_bytes(p, (uint64_t)p->u * p->v * p->gl));
  L.staging = take(L.staging_pkts * 8);
  L.utab = take(ucap * 8);
  L.ulist = take((size_t)p->max_sampled * 4);
  for (int q = 0; q < 2; q++) {
    L.ctab[q] = take(ccap * 8);
    L.cflags[q] = take(ccap * 4);
    L.clist[q] = take((size_t)p->max_candidates * 4);
  }
  L.sort_tmp = take((size_t)p->max_candidates * 4);
  L.sort_hist = take((size_t)L.ntiles * kRadix * 4);
  L.lut_est = take(((size_t)p->gl + 1) * 4);
  L.lut_flags = take(((size_t)p->gl + 1) * 4);
  for (int q = 0; q < 2; q++) {
    L.rep_stats[q] = take(sizeof(srla_slice_stats));
    L.rep_entries[q] = take((size_t)p->max_candidates * sizeof(srla_entry));
  }
  L.pairs = p->pair_slots_log2 != -1;
  const uint32_t plog = p->pair_slots_log2 > 0 ? (uint32_t)p->pair_slots_log2 : 21u;
  L.pmask = L.pairs ? (1u << plog) - 1u : 0u;
  // two pair tables by slice parity: the next slice's is cleared while this one is closed
  L.n_ptab = L.pairs ? n_pair_tables : 0;
  for (int q = 0; q < 2; q++) L.ptab[q] = take(q < L.n_ptab ? ((size_t)1 << plog) * 8 : 0);
  // inline mode: one 32-bit word of super point indicator bits per estimator, by parity
  for (int q = 0; q < 2; q++) L.si[q] = take(p->mode == SRLA_MODE_INLINE ? (size_t)p->u * p->v * 4 : 0);
  L.le_spv = sat_spv(p, p->gl);
  L.re_spv = sat_spv(p, p->g);
  L.le_sat = take(L.le_spv ? (size_t)p->u * p->v : 0);
  L.re_sat = take(L.re_spv ? (size_t)p->u * p->v : 0);
  L.total = off;
  return L;
}

// Bytes from a slice's statistics to its report entries: the entries' region follows the
// statistics' (one aligned step, the same for both slice parities), so one copy moves the
// statistics and the first entries together.
inline size_t report_gap(const Layout& L) { return L.rep_entries[0] - L.rep_stats[0]; }

}  // namespace host
}  // namespace srla
