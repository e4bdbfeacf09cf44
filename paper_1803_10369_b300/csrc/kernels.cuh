// The kernels of the SRLA hot path for one link: the per-packet scan (Algorithm 2) and the
// end-of-slice pass (Section 4.2: row census, Eq. 8, Eq. 9; Algorithm 3: slide and carry).
#pragma once

#include "scan_parts.cuh"

namespace srla {

// Packets are read as 16-byte vectors (two pairs) when the batch is 16-byte aligned.
// Each warp iteration covers 128 packets: lane l holds packets 2l, 2l+1, 64+2l, 65+2l; the
// next iteration's packets are loaded before the current ones are scanned.  kInline: the
// candidate test of Algorithm 2 runs at packet time (SRLA_MODE_INLINE); every packet is
// scanned (no pair de-duplication), since each one runs the test on the SRE as it stands.
// Shared memory of the scan: the block's table of recent pairs (not in the inline mode,
// which scans every packet) and two queues per warp.
template <bool kInline>
constexpr size_t scan_smem_bytes() {
  return (kInline ? 0 : (size_t)kSeen * 8) + (size_t)((kInline ? kScanThreadsInline : kScanThreads) / 32) * 2 * kQueue * 8;
}

template <typename CellT, bool kVec, bool kInline = false, bool kElide = false, bool kHeavy = false>
__global__ void __launch_bounds__(kInline ? kScanThreadsInline : kScanThreads, kInline ? 2 : 1) k_scan(const uint32_t* __restrict__ pairs, uint64_t n, Geo geo,
                                                          const __grid_constant__ Coef coef, CellT* __restrict__ re,
                                                          CellT* __restrict__ le, Ctl* __restrict__ ctl,
                                                          unsigned long long* __restrict__ utab, uint32_t umask,
                                                          uint32_t* __restrict__ ulist, uint32_t umax,
                                                          unsigned long long* __restrict__ ptab, uint32_t pmask,
                                                          const __grid_constant__ InlineArgs ia) {
  extern __shared__ unsigned long long scan_smem[];
  __shared__ HeavyTrack s_heavy;
  __shared__ unsigned s_cnt[6];
  if (threadIdx.x < 6) s_cnt[threadIdx.x] = 0u;
  volatile unsigned long long* seen = scan_smem;
  auto queue_mem = reinterpret_cast<unsigned long long(*)[2][kQueue]>(scan_smem + (kInline ? 0 : kSeen));
  if (!kInline)
    for (int x = threadIdx.x; x < kSeen; x += blockDim.x) seen[x] = kNoPair;
  if constexpr (kHeavy) heavy_reset(&s_heavy);
  __syncthreads();
  if (kInline || (ptab && ctl->pair_mode == 0)) ptab = nullptr;
  HeavyTrack* hv = (kHeavy && heavy_fits(geo)) ? &s_heavy : nullptr;
  const uint32_t tm = ctl->tm;
  const CellT code = stamp_code<CellT>(tm);
  const uint32_t tag = slice_tag(ctl->T);
  const Win win = make_win<CellT>(tm, geo.P, geo.k);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  ScanQueues Q{queue_mem[warp][0], queue_mem[warp][1], 0u, 0u};
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  uint64_t base = gw * 128;
  uint32_t a[4], b[4];
  bool ok[4];
  ScanCount sc{0u, 0u, 0u, 0u, 0u, 0u};
  load_pairs<kVec>(pairs, n, base, lane, a, b, ok);
  while (base < n) {
    const uint64_t next = base + nw * 128;
    uint32_t na[4], nb[4];
    bool nok[4];
    load_pairs<kVec>(pairs, n, next, lane, na, nb, nok);
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const unsigned long long key = ((unsigned long long)a[j] << 32) | b[j];
      bool miss = false;
      if (kInline) {
        miss = ok[j];
      } else if (ok[j]) {  // this block's table of recently scanned pairs
        const uint32_t h = seen_slot(key);
        if (key == kNoPair || seen[h] != key) {
          miss = true;
          if (key != kNoPair) seen[h] = key;
        }
      }
      if (ptab) {
        // the pair that marks empty slots cannot be claimed: it is always scanned
        queue_push(Q.q1, Q.n1, miss && key != kNoPair, key, lane);
        queue_push(Q.q2, Q.n2, miss && key == kNoPair, key, lane);
        if (Q.n2 >= 32)
          drain_scan<CellT, false, kElide, kHeavy>(Q, sc, geo, coef, code, re, le, ctl, utab, umask, ulist, umax, tag,
                                                   lane, hv);
        if (Q.n1 >= 32)
          drain_claim<CellT, kElide, kHeavy>(Q, sc, ptab, pmask, geo, coef, code, re, le, ctl, utab, umask, ulist, umax,
                                             tag, lane, hv);
      } else {
        queue_push(Q.q2, Q.n2, miss, key, lane);
        if (Q.n2 >= 32)
          drain_scan<CellT, kInline, kElide, kHeavy>(Q, sc, geo, coef, code, re, le, ctl, utab, umask, ulist, umax, tag,
                                                     lane, hv, &ia, &win);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
      a[j] = na[j]; b[j] = nb[j]; ok[j] = nok[j];
    }
    base = next;
  }
  // what is left in the queues
  if (ptab && Q.n1)
    drain_claim<CellT, kElide, kHeavy>(Q, sc, ptab, pmask, geo, coef, code, re, le, ctl, utab, umask, ulist, umax, tag,
                                       lane, hv);
  while (Q.n2)
    drain_scan<CellT, kInline, kElide, kHeavy>(Q, sc, geo, coef, code, re, le, ctl, utab, umask, ulist, umax, tag, lane,
                                               hv, &ia, &win);
  scan_count_flush(sc, ctl, s_cnt, lane);
}

// One streaming pass over the recorders: census and stamp ageing.  Each block sweeps one
// part of one row: gx_le blocks per SLE row, then (when ageing) gx_re blocks per SRE row, the
// counts chosen by the host in proportion to the row lengths so that every block moves about
// the same number of bytes.  Within its row a block walks grid-stride (neighbouring threads
// read neighbouring vectors), each thread with four vector loads in flight.
template <typename CellT>
__global__ void __launch_bounds__(256) k_sweep(Geo geo, CellT* __restrict__ re, CellT* __restrict__ le,
                                               Ctl* __restrict__ ctl, int do_census, int do_reset,
                                               int after_close, uint32_t gx_le, uint32_t gx_re,
                                               uint8_t* __restrict__ le_sat, uint8_t* __restrict__ re_sat,
                                               uint32_t le_spv, uint32_t re_spv) {
  const bool census = do_census != 0;
  const bool reset = do_reset != 0;
  const uint32_t n_le_blocks = (census || reset) ? geo.u * gx_le : 0u;
  const bool is_le = blockIdx.x < n_le_blocks;
  const uint32_t b = is_le ? blockIdx.x : blockIdx.x - n_le_blocks;
  const uint32_t gx = is_le ? gx_le : gx_re;
  const uint32_t row = b / gx, part = b % gx;
  if (row >= geo.u) return;
  // SLE rows: the census (in-window recorders at the open slice); SRE rows (present when the
  // sweep ages them), only when the previous slice's SLE was nearly saturated (sat_hint bit
  // 0): the recorders inside the window after the slide (age + 1 < k), which lets the
  // estimate skip the carry gathers when every SRE recorder passes
  const uint32_t hint = ctl->sat_hint;
  const bool count = census && (is_le || (!kIsBit<CellT> && (hint & 1u)));
  const size_t cells = (size_t)geo.v * (is_le ? geo.gl : geo.g);
  uint4* base = reinterpret_cast<uint4*>(words_at<CellT>(is_le ? le : re, (size_t)row * cells));
  const size_t nvec = cell_array_bytes<CellT>(cells) / 16;
  const uint32_t tm = ctl->tm, P = geo.P;
  // stamp of the slice that opens next: after the slice was closed, that is the open slice
  const uint32_t alias = 1u + (after_close ? tm : ((tm + 1u == P) ? 0u : tm + 1u));
  const uint32_t asplat = splat<CellT>(alias);
  const SweepWin sw = make_sweep_win<CellT>(tm, P, is_le ? geo.k : geo.k - 1u);
  const size_t stride = (size_t)gx * blockDim.x;
  const size_t x = (size_t)part * blockDim.x + threadIdx.x;
  // saturated-estimator bytes only when the previous slice was nearly saturated (sat_hint)
  const uint32_t spv = !count ? 0u : is_le ? ((hint & 1u) ? le_spv : 0u) : ((hint & 2u) ? re_spv : 0u);
  uint8_t* sat_row = spv ? (is_le ? le_sat : re_sat) + (size_t)row * geo.v : nullptr;
  uint32_t cnt = sweep_any<CellT>(base, nvec, x, stride, count, reset, sw, alias, asplat, sat_row, spv, 0);
  if (count) {
    __shared__ uint32_t part_sum[8];
    cnt = warp_sum(cnt);
    if ((threadIdx.x & 31) == 0) part_sum[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long s = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += part_sum[w];
      atomicAdd(is_le ? &ctl->census[row] : &ctl->sre_post, s);
    }
  }
}

// Eq. 8 (UP from the row census) and Eq. 9 for every union weight w in [0, g'], in FP64,
// rounded once to FP32: for a fixed slice the estimate depends on w alone, so the estimate
// kernel only looks it up.  Runs concurrently with the candidate filter and sort.
__global__ void k_lut(Geo geo, Ctl* __restrict__ ctl, float* __restrict__ lut_est, uint32_t* __restrict__ lut_flags) {
  __shared__ double s_up;
  if (threadIdx.x == 0) {
    s_up = slice_up(geo, ctl);
    if (blockIdx.x == 0) ctl->up = s_up;
  }
  __syncthreads();
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w <= geo.gl; w += gridDim.x * blockDim.x) {
    uint32_t f;
    const double e = eq9(w, geo.gl, s_up, geo.theta, &f);
    lut_est[w] = (float)e;
    lut_flags[w] = f;
    if (f & SRLA_SUPER) atomicMin(&ctl->w_star, w);
  }
}

// -------------------------------------------------------------- new candidates (b3)
//
// For every distinct host sampled in the open slice: |URE(aip)|^k at the end of the slice
// (before the slide).  Hosts with at least ceil(rho*g) in-window union cells enter the
// slice's candidate set, which already holds the hosts carried from the previous slice.
template <typename CellT>
__global__ void __launch_bounds__(256, 4) k_filter(Geo geo, const __grid_constant__ Coef coef,
                                                const CellT* __restrict__ re, Ctl* __restrict__ ctl,
                                                const uint32_t* __restrict__ ulist, uint32_t umax,
                                                unsigned long long* ctab0, unsigned long long* ctab1,
                                                uint32_t* cflags0, uint32_t* cflags1, uint32_t cmask,
                                                uint32_t* clist0, uint32_t* clist1, uint32_t cmax) {
  const unsigned long long T = ctl->T;
  const int par = (int)(T & 1);
  unsigned long long* ctab = par ? ctab1 : ctab0;
  uint32_t* cflags = par ? cflags1 : cflags0;
  uint32_t* clist = par ? clist1 : clist0;
  const uint32_t tag = slice_tag(T);
  const uint32_t n = min(ctl->n_sampled, umax);
  const Win win = make_win<CellT>(ctl->tm, geo.P, geo.k);
  const int lane = threadIdx.x & 31;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  // two hosts per warp and iteration, so that their gathers overlap
  for (uint32_t idx = 2 * gw; idx < n; idx += 2 * nw) {
    const bool two = idx + 1 < n;
    const uint32_t aip0 = ulist[idx];
    const uint32_t aip1 = two ? ulist[idx + 1] : aip0;
    const bool mine = (uint32_t)lane < geo.u;
    const uint32_t col0 = mine ? hash61(coef.a[lane], coef.b[lane], aip0) & geo.vmask : 0u;
    const uint32_t col1 = mine ? hash61(coef.a[lane], coef.b[lane], aip1) & geo.vmask : 0u;
    uint32_t cnt0, cnt1;
    union_count_atleast2<CellT>(re, geo.v, geo.g, geo.u, col0, col1, win, geo.rho_g, lane, cnt0, cnt1);
    if (lane == 0) {
      filter_admit(ctl, ctab, cflags, cmask, clist, cmax, par, tag, aip0, cnt0 >= geo.rho_g);
      if (two) filter_admit(ctl, ctab, cflags, cmask, clist, cmax, par, tag, aip1, cnt1 >= geo.rho_g);
    }
  }
}

// -------------------------------------------------- estimate (b4), carry (b5), close
//
// For every candidate of the sorted list: w = |ULE(aip)|^k (Algorithm 1), the Eq. 9
// estimate and super point flag, and the report entry at the same position.  Then the carry
// test of Algorithm 3 on the post-slide SRE (age + 1 < k); hosts that pass join the next
// slice's candidate set.  The last block to finish closes the slice: it writes the slice's
// statistics and opens the next slice in the control block.
template <typename CellT>
__global__ void __launch_bounds__(256) k_estimate(Geo geo, const __grid_constant__ Coef coef,
                                                  const CellT* __restrict__ re, const CellT* __restrict__ le,
                                                  Ctl* __restrict__ ctl, unsigned long long* ctab0,
                                                  unsigned long long* ctab1, uint32_t* cflags0, uint32_t* cflags1,
                                                  uint32_t cmask, uint32_t* clist0, uint32_t* clist1, uint32_t cmax,
                                                  srla_entry* rep0, srla_entry* rep1, srla_slice_stats* st0,
                                                  srla_slice_stats* st1, uint32_t umax,
                                                  const float* __restrict__ lut_est,
                                                  const uint32_t* __restrict__ lut_flags, uint32_t* si0,
                                                  uint32_t* si1, const uint8_t* __restrict__ le_sat,
                                                  const uint8_t* __restrict__ re_sat, uint32_t sat_maps) {
  __shared__ int s_last;
  const unsigned long long T = ctl->T;
  const int par = (int)(T & 1);
  const unsigned long long* ctab = par ? ctab1 : ctab0;
  const uint32_t* cflags = par ? cflags1 : cflags0;
  const uint32_t* clist = par ? clist1 : clist0;
  unsigned long long* ntab = par ? ctab0 : ctab1;
  uint32_t* nflags = par ? cflags0 : cflags1;
  uint32_t* nlist = par ? clist0 : clist1;
  srla_entry* rep = par ? rep1 : rep0;
  const uint32_t tag = slice_tag(T), ntag = slice_tag(T + 1);
  const uint32_t n = min(ctl->cat_count[par], cmax);
  const Win win = make_win<CellT>(ctl->tm, geo.P, geo.k);
  const Win win_post = make_win<CellT>(ctl->tm, geo.P, geo.k - 1u);  // age + 1 < k after the slide
  // Saturated sketches: when every SLE recorder of every row is inside the window (the
  // census is v*g' in each row, so UP = 1), every host's union SLE weight is g'; when every
  // SRE recorder is inside the post-slide window (counted by the sweep), every carry test
  // passes.  Both are exact, and spare the gathers.
  bool le_full = true;
  unsigned long long min_census = ~0ull;
  for (uint32_t i = 0; i < geo.u; i++) {
    le_full &= ctl->census[i] == (unsigned long long)geo.v * geo.gl;
    min_census = min(min_census, ctl->census[i]);
  }
  const bool re_full = ctl->sre_post == (unsigned long long)geo.u * geo.v * geo.g;
  // Nearly saturated sketches (at least 15/16 of the recorders inside the window): the
  // per-estimator bytes of the sweep (sat_mark) spare the gathers of hosts whose u estimators
  // are all saturated.  The SRE bytes exist when the census sweep aged the SRE (k < 2^z - 1).
  // (only in slices whose census sweep recorded them: sat_hint, set by the previous close)
  const uint32_t hint = ctl->sat_hint;
  const bool le_map = !le_full && (sat_maps & hint & 1u) && 16ull * min_census >= 15ull * geo.v * geo.gl;
  const bool re_map = !re_full && (sat_maps & hint & 2u) && geo.k != geo.P &&
                      16ull * ctl->sre_post >= 15ull * geo.u * geo.v * geo.g;
  const int lane = threadIdx.x & 31;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  // While there are no more candidates than warps, 2n tasks: task i < n estimates candidate
  // i (union SLE), task n + i runs its carry test (post-slide union SRE); the two gathers of
  // a candidate run in different warps.
  for (uint32_t idx = gw; n <= nw && idx < 2 * n; idx += nw) {
    const bool est = idx < n;
    const uint32_t i = est ? idx : idx - n;
    const uint32_t aip = clist[i];
    const uint32_t mycol = (uint32_t)lane < geo.u ? hash61(coef.a[lane], coef.b[lane], aip) & geo.vmask : 0u;
    if (est) {
      uint32_t origin = 0;
      if (lane == 0) {  // issued before the gather, used after it
        const uint32_t s = set_find(ctab, cmask, tag, aip);
        origin = (s != 0xFFFFFFFFu) ? cflags[s] : 0u;
      }
      const bool sat = le_full || (le_map && host_saturated(le_sat, geo.v, geo.u, mycol, lane));
      const uint32_t w = sat ? geo.gl : union_count<CellT>(le, geo.v, geo.gl, geo.u, mycol, win, lane);
      if (lane == 0) {
        srla_entry e;
        e.aip = aip;
        e.w = w;
        e.est = lut_est[w];
        e.flags = origin | lut_flags[w];
        rep[i] = e;
      }
      continue;
    }
    const bool sat = re_full || (re_map && host_saturated(re_sat, geo.v, geo.u, mycol, lane));
    const uint32_t cw = sat ? geo.g : union_count<CellT>(re, geo.v, geo.g, geo.u, mycol, win_post, lane);
    if (cw < geo.rho_g) continue;
    // inline mode: a carried host gets its SI bits in the next slice's indicators (Algorithm 3)
    uint32_t* si_next = par ? si0 : si1;
    if (si_next && (uint32_t)lane < geo.u)
      atomicOr(si_next + (size_t)lane * geo.v + mycol, 1u << si_bit(coef, geo.u, aip));
    if (lane == 0) {
      uint32_t slot;
      const int r = set_insert(ntab, cmask, ntag, aip, &slot);
      if (r == 1) {
        nflags[slot] = SRLA_CARRIED;
        const unsigned at = atomicAdd(&ctl->cat_count[par ^ 1], 1u);
        if (at < cmax)
          nlist[at] = aip;
        else
          atomicOr(&ctl->overflow_next, 2u);
      } else if (r < 0) {
        atomicOr(&ctl->overflow_next, 2u);
      }
    }
  }
  // Above that, two tasks per run of b consecutive candidates: one estimates them (union SLE),
  // one runs their carry test (post-slide union SRE).  b grows up to 32 so that a run's hosts,
  // origin flags, saturated-estimator tests, report entries and next-slice inserts are handled
  // with one lane per candidate, their round trips paid once per run; only the gathers of the
  // hosts that are not saturated go one candidate at a time.
  const uint32_t b = min(32u, max(1u, (n + nw - 1) / nw));
  const uint32_t runs = n > nw ? (n + b - 1) / b : 0u;
  for (uint32_t t = gw; t < 2 * runs; t += nw) {
    const bool est = t < runs;
    const uint32_t r0 = (est ? t : t - runs) * b;
    const uint32_t m = min(b, n - r0);  // candidates of this run, one per lane
    const bool mine = (uint32_t)lane < m;
    const uint32_t my_aip = mine ? clist[r0 + lane] : 0u;
    if (est) {
      uint32_t origin = 0;
      if (mine) {  // issued before the gathers, used after them
        const uint32_t s = set_find(ctab, cmask, tag, my_aip);
        origin = (s != 0xFFFFFFFFu) ? cflags[s] : 0u;
      }
      uint32_t my_w = geo.gl;  // a host whose u estimators are all saturated has w = g'
      const bool my_sat = le_full || (mine && le_map && own_host_saturated(le_sat, geo, coef, my_aip));
      for (unsigned todo = __ballot_sync(kFull, mine && !my_sat); todo; todo &= todo - 1u) {
        const int j = __ffs(todo) - 1;
        const uint32_t aip = __shfl_sync(kFull, my_aip, j);
        const uint32_t mycol = (uint32_t)lane < geo.u ? hash61(coef.a[lane], coef.b[lane], aip) & geo.vmask : 0u;
        const uint32_t w = union_count<CellT>(le, geo.v, geo.gl, geo.u, mycol, win, lane);
        if (lane == j) my_w = w;
      }
      if (mine) {
        srla_entry e;
        e.aip = my_aip;
        e.w = my_w;
        e.est = lut_est[my_w];
        e.flags = origin | lut_flags[my_w];
        rep[r0 + lane] = e;
      }
      continue;
    }
    // inline mode: a carried host gets its SI bits in the next slice's indicators (Algorithm 3)
    uint32_t* si_next = par ? si0 : si1;
    // a host whose u estimators are all saturated has union weight g >= ceil(rho g): it passes
    const bool my_sat = re_full || (mine && re_map && own_host_saturated(re_sat, geo, coef, my_aip));
    bool pass = mine && my_sat;
    for (unsigned todo = __ballot_sync(kFull, mine && !my_sat); todo; todo &= todo - 1u) {
      const int j = __ffs(todo) - 1;
      const uint32_t aip = __shfl_sync(kFull, my_aip, j);
      const uint32_t mycol = (uint32_t)lane < geo.u ? hash61(coef.a[lane], coef.b[lane], aip) & geo.vmask : 0u;
      const uint32_t cw = union_count<CellT>(re, geo.v, geo.g, geo.u, mycol, win_post, lane);
      if (lane == j) pass = cw >= geo.rho_g;
    }
    if (si_next) {
      for (unsigned pm = __ballot_sync(kFull, pass); pm; pm &= pm - 1u) {
        const uint32_t aip = __shfl_sync(kFull, my_aip, __ffs(pm) - 1);
        if ((uint32_t)lane < geo.u)
          atomicOr(si_next + (size_t)lane * geo.v + (hash61(coef.a[lane], coef.b[lane], aip) & geo.vmask),
                   1u << si_bit(coef, geo.u, aip));
      }
    }
    // the run's carried hosts join the next slice's candidate set and list together
    int r = -2;
    if (pass) {
      uint32_t slot;
      r = set_insert(ntab, cmask, ntag, my_aip, &slot);
      if (r == 1)
        nflags[slot] = SRLA_CARRIED;
      else if (r < 0)
        atomicOr(&ctl->overflow_next, 2u);
    }
    const unsigned ins = __ballot_sync(kFull, r == 1);
    if (ins) {
      const int first = __ffs(ins) - 1;
      unsigned at = 0;
      if (lane == first) at = atomicAdd(&ctl->cat_count[par ^ 1], (unsigned)__popc(ins));
      at = __shfl_sync(kFull, at, first) + (unsigned)__popc(ins & ((1u << lane) - 1u));
      if (r == 1) {
        if (at < cmax)
          nlist[at] = my_aip;
        else
          atomicOr(&ctl->overflow_next, 2u);
      }
    }
  }
  // the last block to get here closes the slice
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&ctl->blocks_done, 1u) == gridDim.x - 1u;
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  close_slice(geo, ctl, par ? st1 : st0, umax, cmax);
}

// Distances -> stamps at open slice with T mod P = tm (one-bit recorders: 32 per thread).
template <typename CellT>
__global__ void k_encode(const uint16_t* __restrict__ d, CellT* __restrict__ cells, size_t n, uint32_t tm,
                         uint32_t P) {
  if constexpr (kIsBit<CellT>) {
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n / 32; x += (size_t)gridDim.x * blockDim.x) {
      uint32_t word = 0;
      for (int b = 0; b < 32; b++) word |= (d[32 * x + b] < P ? 1u : 0u) << b;
      reinterpret_cast<uint32_t*>(cells)[x] = word;
    }
  } else {
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x) {
      const uint32_t dd = d[x];
      uint32_t c = 0;
      if (dd < P) {
        const int s = ((int)tm - (int)dd) % (int)P;
        c = 1u + (uint32_t)(s < 0 ? s + (int)P : s);
      }
      cells[x] = (CellT)c;
    }
  }
}

// Insert carried hosts (checkpoint import) into the open slice's candidate set, and set
// their SI bits in the open slice's indicators (inline mode, si non-null).
__global__ void k_insert_carried(const uint32_t* __restrict__ hosts, uint32_t n, Ctl* __restrict__ ctl,
                                 unsigned long long* ctab0, unsigned long long* ctab1, uint32_t* cflags0,
                                 uint32_t* cflags1, uint32_t cmask, uint32_t* clist0, uint32_t* clist1,
                                 uint32_t cmax, Geo geo, const __grid_constant__ Coef coef, uint32_t* si) {
  const unsigned long long T = ctl->T;
  const int par = (int)(T & 1);
  unsigned long long* ctab = par ? ctab1 : ctab0;
  uint32_t* cflags = par ? cflags1 : cflags0;
  uint32_t* clist = par ? clist1 : clist0;
  const uint32_t tag = slice_tag(T);
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
    uint32_t slot;
    const int r = set_insert(ctab, cmask, tag, hosts[x], &slot);
    if (si)
      for (uint32_t i = 0; i < geo.u; i++)
        atomicOr(si + (size_t)i * geo.v + (hash61(coef.a[i], coef.b[i], hosts[x]) & geo.vmask),
                 1u << si_bit(coef, geo.u, hosts[x]));
    if (r == 1) {
      cflags[slot] = SRLA_CARRIED;
      const unsigned at = atomicAdd(&ctl->cat_count[par], 1u);
      if (at < cmax)
        clist[at] = hosts[x];
      else
        atomicOr(&ctl->overflow, 2u);
    }
  }
}

// Random-store probe (the store roofline of the scan): n writes of one cell-sized value to
// pseudo-random cells of a footprint of `cells` cells, i.e. the access shape of the scan's
// DRsets without their hashing, de-duplication or sampling (every writer of a slice writes
// the same stamp, so the value is the same for all writes).  The cell of write i comes from
// a 64-bit mix of i (the SplitMix64 finaliser of Steele, Lea and Flood) scaled to [0, cells)
// by a multiply-high.  kPolicy selects how a write is made:
//   0  a plain store (what the scan does);
//   1  an atomic maximum: native on 32-bit cells; on 8- and 16-bit cells, which have no
//      atomic maximum, a compare-and-swap loop on the enclosing 32-bit word (at most 64
//      tries, so contention can only slow it down);
//   2  read before write: a load through L2, and a store only if the cell differs;
//   3  a compare-and-swap of a 64-bit slot from the empty key (all ones) to the value: the
//      claim of the scan's pair table (after the first claim of a slot the swap fails, which
//      is the same round trip);
//   4  a plain load through L2 (the probes of the sampled-host set), folded into a register
//      that is stored only if it equals a value no load returns.
enum : uint32_t { kProbeStore = 0, kProbeAtomicMax = 1, kProbeReadFirst = 2, kProbeCas = 3, kProbeLoad = 4 };

template <typename CellT>
__device__ __forceinline__ void probe_atomic_max(CellT* p, CellT val) {
  if constexpr (sizeof(CellT) == 4) {
    atomicMax(reinterpret_cast<unsigned*>(p), (unsigned)val);
  } else {
    unsigned* w = reinterpret_cast<unsigned*>(reinterpret_cast<uintptr_t>(p) & ~(uintptr_t)3);
    const unsigned sh = (unsigned)(reinterpret_cast<uintptr_t>(p) & 3u) * 8u;
    const unsigned m = (unsigned)(CellT)~(CellT)0 << sh;
    unsigned old = __ldcg(w);
    for (int it = 0; it < 64; it++) {
      if (((old & m) >> sh) >= (unsigned)val) break;
      const unsigned prev = atomicCAS(w, old, (old & ~m) | ((unsigned)val << sh));
      if (prev == old) break;
      old = prev;
    }
  }
}

template <typename CellT, uint32_t kPolicy>
__global__ void __launch_bounds__(256) k_scatter_probe(CellT* __restrict__ buf, uint64_t cells, uint64_t n,
                                                       uint64_t seed) {
  const CellT val = (CellT)(seed | 1u);
  CellT acc = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t z = i + seed * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    CellT* p = buf + __umul64hi(z, cells);
    if constexpr (kPolicy == kProbeStore) {
      *p = val;
    } else if constexpr (kPolicy == kProbeAtomicMax) {
      probe_atomic_max<CellT>(p, val);
    } else if constexpr (kPolicy == kProbeReadFirst) {
      if (__ldcg(p) != val) *p = val;
    } else if constexpr (kPolicy == kProbeCas) {
      static_assert(sizeof(CellT) == 8, "the claim probe swaps 64-bit slots");
      acc ^= (CellT)atomicCAS(reinterpret_cast<unsigned long long*>(p), ~0ull, (unsigned long long)val);
    } else {
      acc ^= __ldcg(p);
    }
  }
  // loads and swaps must not be optimised away: their folded results feed a store, taken
  // only in the rare case that they equal one fixed pattern (it writes one cell of the
  // caller's scratch buffer)
  if constexpr (kPolicy == kProbeCas || kPolicy == kProbeLoad)
    if (acc == (CellT)0x5A5A5A5A5A5A5A5Bull) buf[0] = acc;
}

}  // namespace srla
