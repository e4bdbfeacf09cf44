// Kernels of the multi-link group: the same scan and slice end as one link (scan_parts.cuh),
// run for every attached link in one launch each.  Links are independent estimator arrays
// (one per monitored edge router, Section 3.1); the kernels find their links, packet batches
// and sweep work in device-resident tables, so one captured graph serves any membership.
#pragma once

#include "scan_parts.cuh"
#include "sort_parts.cuh"

namespace srla {

// Everything a kernel needs to know about one attached link.
struct LinkDesc {
  Geo geo;
  Coef coef;
  uint32_t active;      // 0: free slot
  uint32_t cell_bytes;  // 1 or 2; 0: one-bit recorders
  uint32_t k_is_P;
  uint32_t umask, umax, cmask, cmax, ntiles, pmask;
  uint32_t scan_policy;  // SRLA_SCAN_POLICY_*: pair table and scan build of this link
  Ctl* ctl;
  void* re;
  void* le;
  unsigned long long* utab;
  uint32_t* ulist;
  unsigned long long* ctab[2];
  uint32_t* cflags[2];
  uint32_t* clist[2];
  uint32_t* sort_tmp;
  uint32_t* sort_hist;
  float* lut_est;
  uint32_t* lut_flags;
  srla_slice_stats* st[2];
  unsigned long long* ptab;  // per-slice pair table, or null
  uint8_t* le_sat;           // saturated-estimator bytes of the SLE / SRE (see sat_mark), or null
  uint8_t* re_sat;
  uint32_t le_spv, re_spv;   // vectors per run when those bytes are recorded, else 0
};

constexpr int kGroupSeenLog2 = 12;  // pairs remembered per group scan block (several per SM)

// One packet batch of one link for the group scan (at most kTaskPkts packets).
struct ScanTask {
  unsigned long long ptr;  // device address of interleaved (aip, bip) uint32 pairs
  uint32_t n;
  uint32_t link;
};
constexpr uint32_t kTaskPkts = 1u << 16;

// A streaming piece of per-slice sweep work.
struct SweepChunk {
  uint32_t link;
  uint32_t kind;   // 0: SLE row (census, ageing), 1: SRE row (ageing), 2: pair table (clear)
  uint32_t row;
  uint32_t pad;
  unsigned long long begin, count;  // 16-byte vectors
};

// Group control block (device).
struct GroupCtl {
  const SweepChunk* chunks;  // sweep work list (rebuilt when links attach or detach)
  const SweepChunk* post;    // post-close ageing work list
  unsigned int next_task;  // scan work counter
  unsigned int blocks_done;
  unsigned int bar_count, bar_gen;  // cooperative sort barrier
  unsigned int n_links;    // slots (active or not)
  unsigned int n_chunks;   // sweep chunks
  unsigned int n_post;     // post-close ageing chunks (links with k = 2^z - 1)
  unsigned int overflow;   // bit 2: a bounded wait gave up
  unsigned int rep_cap;    // entries of the group report buffer
  unsigned int pad[3];
};

// The per-slice task table: a 16-byte header (task count) followed by the tasks.
struct TaskHeader {
  unsigned int n_tasks;
  unsigned int pad[3];
};

// Calls f with a value of the link's recorder storage type.
template <typename F>
__device__ __forceinline__ void with_cells(uint32_t cell_bytes, F&& f) {
  if (cell_bytes == 1)
    f(uint8_t{});
  else if (cell_bytes == 2)
    f(uint16_t{});
  else
    f(Bit{});
}

// ------------------------------------------------------------------------ scan

// The link's aggregation policy for this slice: whether the scan consults the per-slice pair
// table (the adaptive policies follow the pair_mode the previous slice close chose), and
// whether it runs the read-first build (8/16-bit recorders only).
__device__ __forceinline__ bool policy_table(const LinkDesc& D, uint32_t pair_mode) {
  const bool adaptive = D.scan_policy == SRLA_SCAN_POLICY_ADAPTIVE || D.scan_policy == SRLA_SCAN_POLICY_ADAPTIVE_RF;
  return D.ptab && adaptive && pair_mode;
}

__device__ __forceinline__ bool policy_read_first(const LinkDesc& D, bool table) {
  if (D.cell_bytes == 0) return false;
  return D.scan_policy == SRLA_SCAN_POLICY_OFF_RF || (D.scan_policy == SRLA_SCAN_POLICY_ADAPTIVE_RF && !table);
}

template <typename CellT, bool kVec, bool kElide, bool kHeavy>
__device__ __forceinline__ void group_scan_task(const ScanTask& t, const LinkDesc& D, Ctl* ctl,
                                                volatile unsigned long long* seen, ScanQueues& Q, int lane, int warp,
                                                int nwarps, ScanCount& sc, bool table, HeavyTrack* hv, uint32_t tm,
                                                unsigned long long T) {
  const uint32_t* pairs = reinterpret_cast<const uint32_t*>(t.ptr);
  const uint64_t n = t.n;
  CellT* re = static_cast<CellT*>(D.re);
  CellT* le = static_cast<CellT*>(D.le);
  unsigned long long* ptab = table ? D.ptab : nullptr;
  const CellT code = stamp_code<CellT>(tm);
  const uint32_t tag = slice_tag(T);
  const Geo& geo = D.geo;
  const Coef& coef = D.coef;
  for (uint64_t base = (uint64_t)warp * 128; base < n; base += (uint64_t)nwarps * 128) {
    uint32_t a[4], b[4];
    bool ok[4];
    load_pairs<kVec>(pairs, n, base, lane, a, b, ok);
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const unsigned long long key = ((unsigned long long)a[j] << 32) | b[j];
      bool miss = false;
      if (ok[j]) {
        const uint32_t h = seen_slot<kGroupSeenLog2>(key);
        if (key == kNoPair || seen[h] != key) {
          miss = true;
          if (key != kNoPair) seen[h] = key;
        }
      }
      if (ptab) {
        queue_push(Q.q1, Q.n1, miss && key != kNoPair, key, lane);
        queue_push(Q.q2, Q.n2, miss && key == kNoPair, key, lane);
        if (Q.n2 >= 32)
          drain_scan<CellT, false, kElide, kHeavy>(Q, sc, geo, coef, code, re, le, ctl, D.utab, D.umask, D.ulist, D.umax, tag,
                                           lane, hv);
        if (Q.n1 >= 32)
          drain_claim<CellT, kElide, kHeavy>(Q, sc, ptab, D.pmask, geo, coef, code, re, le, ctl, D.utab, D.umask, D.ulist,
                                     D.umax, tag, lane, hv);
      } else {
        queue_push(Q.q2, Q.n2, miss, key, lane);
        if (Q.n2 >= 32)
          drain_scan<CellT, false, kElide, kHeavy>(Q, sc, geo, coef, code, re, le, ctl, D.utab, D.umask, D.ulist, D.umax, tag,
                                           lane, hv);
      }
    }
  }
  if (ptab && Q.n1)
    drain_claim<CellT, kElide, kHeavy>(Q, sc, ptab, D.pmask, geo, coef, code, re, le, ctl, D.utab, D.umask, D.ulist, D.umax,
                               tag, lane, hv);
  while (Q.n2)
    drain_scan<CellT, false, kElide, kHeavy>(Q, sc, geo, coef, code, re, le, ctl, D.utab, D.umask, D.ulist, D.umax, tag, lane,
                                     hv);
}

// Persistent blocks take scan tasks one at a time; a task is one link's batch, so the block's
// pair table and the link's parameters (in shared memory) serve the whole task.  kReadFirst
// adds the read-first build: it needs more registers than the others, so it sits in its own
// instantiation, and groups whose policies never choose it run the leaner kernel (two
// 512-thread blocks per SM at 64 registers).
template <int kThreads, bool kReadFirst>
__global__ void __launch_bounds__(kThreads, kThreads >= 512 ? 2 : 768 / kThreads) kg_scan(const LinkDesc* __restrict__ descs,
                                                    const TaskHeader* __restrict__ thdr, GroupCtl* __restrict__ gctl) {
  const ScanTask* tasks = reinterpret_cast<const ScanTask*>(thdr + 1);
  __shared__ unsigned long long seen_mem[1 << kGroupSeenLog2];
  __shared__ unsigned long long queue_mem[kThreads / 32][2][kQueue];
  __shared__ LinkDesc sdesc;
  __shared__ ScanTask stask;
  __shared__ unsigned s_task;
  __shared__ HeavyTrack s_heavy;
  __shared__ unsigned s_cnt[6];
  volatile unsigned long long* seen = seen_mem;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned n_tasks = thdr->n_tasks;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(&gctl->next_task, 1u);
    if (threadIdx.x < 6) s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    const unsigned ti = s_task;
    if (ti >= n_tasks) break;
    if (threadIdx.x == 0) stask = tasks[ti];
    __syncthreads();
    {  // the task's link parameters into shared memory
      const uint32_t* src = reinterpret_cast<const uint32_t*>(descs + stask.link);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&sdesc);
      for (int x = threadIdx.x; x < (int)(sizeof(LinkDesc) / 4); x += kThreads) dst[x] = src[x];
    }
    for (int x = threadIdx.x; x < (1 << kGroupSeenLog2); x += kThreads) seen[x] = kNoPair;
    heavy_reset(&s_heavy);
    __syncthreads();
    ScanQueues Q{queue_mem[warp][0], queue_mem[warp][1], 0u, 0u};
    ScanCount sc{0u, 0u, 0u, 0u, 0u, 0u};
    const bool vec = (stask.ptr & 15ull) == 0;
    Ctl* ctl = sdesc.ctl;
    // the control block fields of the task, loaded together (one round trip per task)
    const uint32_t pair_mode = ctl->pair_mode, heavy_mode = ctl->heavy_mode, tm = ctl->tm;
    const unsigned long long T = ctl->T;
    const bool table = policy_table(sdesc, pair_mode);
    const bool elide = kReadFirst && policy_read_first(sdesc, table);
    // the heavy build when the link's previous slice showed heavy hosts (see HeavyTrack)
    const bool heavy = sdesc.cell_bytes && !elide && heavy_mode && heavy_fits(sdesc.geo);
    HeavyTrack* hv = heavy ? &s_heavy : nullptr;
    const int nw = kThreads / 32;
    with_cells(sdesc.cell_bytes, [&](auto cell) {
      using CellT = decltype(cell);
      if constexpr (kIsBit<CellT>) {
        if (vec)
          group_scan_task<CellT, true, false, false>(stask, sdesc, ctl, seen, Q, lane, warp, nw, sc, table, hv, tm, T);
        else
          group_scan_task<CellT, false, false, false>(stask, sdesc, ctl, seen, Q, lane, warp, nw, sc, table, hv, tm, T);
      } else {
        if constexpr (kReadFirst) {
          if (elide) {
            if (vec)
              group_scan_task<CellT, true, true, false>(stask, sdesc, ctl, seen, Q, lane, warp, nw, sc, table, hv, tm, T);
            else
              group_scan_task<CellT, false, true, false>(stask, sdesc, ctl, seen, Q, lane, warp, nw, sc, table, hv, tm, T);
            return;
          }
        }
        if (heavy) {
          if (vec)
            group_scan_task<CellT, true, false, true>(stask, sdesc, ctl, seen, Q, lane, warp, nw, sc, table, hv, tm, T);
          else
            group_scan_task<CellT, false, false, true>(stask, sdesc, ctl, seen, Q, lane, warp, nw, sc, table, hv, tm, T);
        } else {
          if (vec)
            group_scan_task<CellT, true, false, false>(stask, sdesc, ctl, seen, Q, lane, warp, nw, sc, table, hv, tm, T);
          else
            group_scan_task<CellT, false, false, false>(stask, sdesc, ctl, seen, Q, lane, warp, nw, sc, table, hv, tm, T);
        }
      }
    });
    scan_count_flush(sc, ctl, s_cnt, lane);
    __syncthreads();
  }
}

// ----------------------------------------------------------------------- sweep

template <typename CellT>
__device__ __forceinline__ void group_sweep_chunk(const SweepChunk& c, const LinkDesc& D, int after_close) {
  Ctl* ctl = D.ctl;
  const bool is_le = c.kind == 0;
  const size_t cells = (size_t)D.geo.v * (is_le ? D.geo.gl : D.geo.g);
  uint4* base = reinterpret_cast<uint4*>(words_at(static_cast<CellT*>(is_le ? D.le : D.re), (size_t)c.row * cells)) +
                c.begin;
  const uint32_t tm = ctl->tm, P = D.geo.P;
  const uint32_t alias = 1u + (after_close ? tm : ((tm + 1u == P) ? 0u : tm + 1u));
  const uint32_t asplat = splat<CellT>(alias);
  // SLE rows: the census; SRE rows: the recorders inside the post-slide window, when the
  // previous slice's SLE was nearly saturated (see k_sweep)
  const uint32_t hint = ctl->sat_hint;
  const bool count = !after_close && (is_le || (!kIsBit<CellT> && (hint & 1u)));
  const bool reset = after_close ? true : !D.k_is_P;
  const SweepWin sw = make_sweep_win<CellT>(tm, P, is_le ? D.geo.k : D.geo.k - 1u);
  const size_t nvec = c.count;
  const uint32_t spv = !count ? 0u : is_le ? ((hint & 1u) ? D.le_spv : 0u) : ((hint & 2u) ? D.re_spv : 0u);
  uint8_t* sat_row = spv ? (is_le ? D.le_sat : D.re_sat) + (size_t)c.row * D.geo.v : nullptr;
  uint32_t cnt = sweep_any<CellT>(base, nvec, threadIdx.x, blockDim.x, count, reset, sw, alias, asplat, sat_row, spv,
                                  c.begin);
  if (count) {
    __shared__ uint32_t part[32];
    cnt = warp_sum(cnt);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long s = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += part[w];
      atomicAdd(is_le ? &ctl->census[c.row] : &ctl->sre_post, s);
    }
    __syncthreads();
  }
}

// Census and ageing of every link's recorders, and clearing of the pair tables.  The
// post-close variant ages the links with k = 2^z - 1 after their slice was closed.
// Index of the link whose half-open range [off[l], off[l+1]) holds item i (off ascending).
__device__ __forceinline__ unsigned link_of(const uint32_t* off, unsigned nl, uint32_t i) {
  unsigned lo = 0, hi = nl;  // off[lo] <= i < off[hi]
  while (hi - lo > 1) {
    const unsigned mid = (lo + hi) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(256, 4) kg_sweep(const LinkDesc* __restrict__ descs, const GroupCtl* __restrict__ gctl,
                                                int post) {
  const unsigned n = post ? gctl->n_post : gctl->n_chunks;
  const SweepChunk* __restrict__ chunks = post ? gctl->post : gctl->chunks;
  for (unsigned ci = blockIdx.x; ci < n; ci += gridDim.x) {
    const SweepChunk c = chunks[ci];
    const LinkDesc& D = descs[c.link];
    if (c.kind == 2) {
      uint4* p = reinterpret_cast<uint4*>(D.ptab) + c.begin;
      const uint4 ones = make_uint4(~0u, ~0u, ~0u, ~0u);
      for (size_t x = threadIdx.x; x < c.count; x += blockDim.x) p[x] = ones;
      continue;
    }
    with_cells(D.cell_bytes, [&](auto cell) { group_sweep_chunk<decltype(cell)>(c, D, post); });
  }
}

// ------------------------------------------------------------------ Eq. 8, Eq. 9

__global__ void kg_lut(const LinkDesc* __restrict__ descs, const GroupCtl* __restrict__ gctl) {
  __shared__ double s_up;
  for (unsigned l = blockIdx.x; l < gctl->n_links; l += gridDim.x) {
    const LinkDesc& D = descs[l];
    if (!D.active) continue;
    if (threadIdx.x == 0) {
      s_up = slice_up(D.geo, D.ctl);
      D.ctl->up = s_up;
    }
    __syncthreads();
    for (uint32_t w = threadIdx.x; w <= D.geo.gl; w += blockDim.x) {
      uint32_t f;
      const double e = eq9(w, D.geo.gl, s_up, D.geo.theta, &f);
      D.lut_est[w] = (float)e;
      D.lut_flags[w] = f;
      if (f & SRLA_SUPER) atomicMin(&D.ctl->w_star, w);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------- new candidates

// One pair of sampled hosts of one link (the second may be absent).
template <typename CellT>
__device__ __forceinline__ void group_filter_pair(const LinkDesc& D, uint32_t q, int lane) {
  Ctl* ctl = D.ctl;
  const unsigned long long T = ctl->T;
  const int par = (int)(T & 1);
  const uint32_t tag = slice_tag(T);
  const uint32_t n = min(ctl->n_sampled, D.umax);
  const Win win = make_win<CellT>(ctl->tm, D.geo.P, D.geo.k);
  const CellT* re = static_cast<const CellT*>(D.re);
  const uint32_t idx = 2 * q;
  const bool two = idx + 1 < n;
  const uint32_t aip0 = D.ulist[idx];
  const uint32_t aip1 = two ? D.ulist[idx + 1] : aip0;
  const bool mine = (uint32_t)lane < D.geo.u;
  const uint32_t col0 = mine ? hash61(D.coef.a[lane], D.coef.b[lane], aip0) & D.geo.vmask : 0u;
  const uint32_t col1 = mine ? hash61(D.coef.a[lane], D.coef.b[lane], aip1) & D.geo.vmask : 0u;
  uint32_t cnt0, cnt1;
  union_count_atleast2<CellT>(re, D.geo.v, D.geo.g, D.geo.u, col0, col1, win, D.geo.rho_g, lane, cnt0, cnt1);
  if (lane == 0) {
    filter_admit(ctl, D.ctab[par], D.cflags[par], D.cmask, D.clist[par], D.cmax, par, tag, aip0, cnt0 >= D.geo.rho_g);
    if (two)
      filter_admit(ctl, D.ctab[par], D.cflags[par], D.cmask, D.clist[par], D.cmax, par, tag, aip1,
                   cnt1 >= D.geo.rho_g);
  }
}

// Host pairs per link for the flat filter: filt_off[l] = the pairs (two hosts each) of the
// active links before l, filt_off[n_links] the total.  One warp.
__global__ void kg_filter_offsets(const LinkDesc* __restrict__ descs, const GroupCtl* __restrict__ gctl,
                                  uint32_t* __restrict__ filt_off) {
  const unsigned nl = gctl->n_links;
  const int lane = threadIdx.x & 31;
  uint32_t run = 0;
  for (unsigned base = 0; base < nl; base += 32) {
    const unsigned l = base + (unsigned)lane;
    uint32_t c = 0;
    if (l < nl && descs[l].active) c = (min(descs[l].ctl->n_sampled, descs[l].umax) + 1u) / 2u;
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += t;
    }
    if (l < nl) filt_off[l] = run + incl - c;
    run += __shfl_sync(kFull, incl, 31);
  }
  if (lane == 0) filt_off[nl] = run;
}

// Every link's sampled hosts in one flat range of host pairs (prefixed by kg_filter_offsets).
__global__ void __launch_bounds__(256, 2) kg_filter(const LinkDesc* __restrict__ descs,
                                                    const GroupCtl* __restrict__ gctl,
                                                    const uint32_t* __restrict__ filt_off) {
  const int lane = threadIdx.x & 31;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const unsigned nl = gctl->n_links;
  const uint32_t total = filt_off[nl];
  for (uint32_t i = gw; i < total; i += nw) {
    const unsigned l = link_of(filt_off, nl, i);
    const LinkDesc& D = descs[l];
    with_cells(D.cell_bytes, [&](auto cell) { group_filter_pair<decltype(cell)>(D, i - filt_off[l], lane); });
  }
}

// ------------------------------------------------------------------------- sort
//
// Candidate lists of up to one tile: one block each (bitonic in shared memory).  Longer
// lists: all blocks together, one link after another (radix passes between grid barriers).

__device__ __forceinline__ bool group_barrier(GroupCtl* g, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &g->bar_gen;
    const unsigned gg = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&g->bar_count, 1u) == nblocks - 1u) {
      g->bar_count = 0;
      __threadfence();
      atomicAdd(&g->bar_gen, 1u);
    } else {
      unsigned it = 0;
      while (*gen == gg) {
        if (++it > kBarrierSpinLimit) {
          atomicOr(&g->overflow, 4u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(kSortThreads) kg_sort(const LinkDesc* __restrict__ descs, GroupCtl* __restrict__ gctl,
                                                        uint32_t* __restrict__ rep_off) {
  extern __shared__ uint32_t bsm[];
  __shared__ uint32_t wcnt[kSortWarps][kRadix];
  __shared__ uint32_t tot[kRadix];
  __shared__ uint32_t part[32];
  const unsigned nl = gctl->n_links;
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // where each link's entries go in the group report
    uint32_t run = 0;
    for (unsigned l = 0; l < nl; l++) {
      rep_off[l] = run;
      const LinkDesc& D = descs[l];
      if (D.active) run += min(D.ctl->cat_count[D.ctl->T & 1], D.cmax);
    }
    rep_off[nl] = run;
  }
  for (unsigned l = blockIdx.x; l < nl; l += gridDim.x) {
    const LinkDesc& D = descs[l];
    if (!D.active) continue;
    const unsigned long long T = D.ctl->T;
    const uint32_t n = min(D.ctl->cat_count[T & 1], D.cmax);
    if (n > 1 && n <= (uint32_t)kSortTile) bitonic_block(D.clist[T & 1], n, bsm);
    __syncthreads();
  }
  for (unsigned l = 0; l < nl; l++) {
    const LinkDesc& D = descs[l];
    if (!D.active) continue;
    const unsigned long long T = D.ctl->T;
    const uint32_t n = min(D.ctl->cat_count[T & 1], D.cmax);
    if (n <= (uint32_t)kSortTile) continue;
    uint32_t* list = D.clist[T & 1];
    const uint32_t ntiles = (n + kSortTile - 1) / kSortTile;
    for (int pass = 0; pass < 4; pass++) {
      const uint32_t* src = (pass & 1) ? D.sort_tmp : list;
      uint32_t* dst = (pass & 1) ? list : D.sort_tmp;
      radix_hist_tiles(src, n, ntiles, pass * 8, D.sort_hist, tot);
      if (!group_barrier(gctl, gridDim.x)) return;
      if (blockIdx.x == 0) radix_scan_block(D.sort_hist, ntiles * kRadix, part);
      if (!group_barrier(gctl, gridDim.x)) return;
      radix_scatter_tiles(src, dst, n, ntiles, pass * 8, D.sort_hist, wcnt, tot);
      if (!group_barrier(gctl, gridDim.x)) return;
    }
  }
}

// ------------------------------------------------------ estimate, carry, close

__device__ __forceinline__ bool grep_off_ok(uint32_t idx, uint32_t cap) { return idx < cap; }

// One task on one candidate of one link: the union SLE weight, Eq. 9 lookup and report
// entry (est), or the carry test on the post-slide union SRE (!est).
template <typename CellT>
__device__ __forceinline__ void group_estimate_one(const LinkDesc& D, uint32_t idx, bool est, int lane,
                                                   srla_entry* grep, uint32_t rep_cap, GroupCtl* gctl) {
  Ctl* ctl = D.ctl;
  const unsigned long long T = ctl->T;
  const int par = (int)(T & 1);
  const uint32_t aip = D.clist[par][idx];
  const uint32_t mycol = (uint32_t)lane < D.geo.u ? hash61(D.coef.a[lane], D.coef.b[lane], aip) & D.geo.vmask : 0u;
  // saturated sketches skip the gathers exactly (see k_estimate)
  bool le_full = true;
  unsigned long long min_census = ~0ull;
  for (uint32_t i = 0; i < D.geo.u; i++) {
    le_full &= ctl->census[i] == (unsigned long long)D.geo.v * D.geo.gl;
    min_census = min(min_census, ctl->census[i]);
  }
  const bool re_full = ctl->sre_post == (unsigned long long)D.geo.u * D.geo.v * D.geo.g;
  const uint32_t hint = ctl->sat_hint;
  const bool le_map = !le_full && D.le_spv && (hint & 1u) && 16ull * min_census >= 15ull * D.geo.v * D.geo.gl;
  const bool re_map = !re_full && D.re_spv && (hint & 2u) && !D.k_is_P &&
                      16ull * ctl->sre_post >= 15ull * D.geo.u * D.geo.v * D.geo.g;
  if (est) {
    uint32_t origin = 0;
    if (lane == 0) {  // issued before the gather, used after it
      const uint32_t s = set_find(D.ctab[par], D.cmask, slice_tag(T), aip);
      origin = (s != 0xFFFFFFFFu) ? D.cflags[par][s] : 0u;
    }
    const Win win = make_win<CellT>(ctl->tm, D.geo.P, D.geo.k);
    const bool sat = le_full || (le_map && host_saturated(D.le_sat, D.geo.v, D.geo.u, mycol, lane));
    const uint32_t w =
        sat ? D.geo.gl
            : union_count<CellT>(static_cast<const CellT*>(D.le), D.geo.v, D.geo.gl, D.geo.u, mycol, win, lane);
    if (lane == 0) {
      srla_entry e;
      e.aip = aip;
      e.w = w;
      e.est = D.lut_est[w];
      e.flags = origin | D.lut_flags[w];
      if (grep_off_ok(idx, rep_cap)) grep[idx] = e; else atomicOr(&gctl->overflow, 2u);
    }
    return;
  }
  const Win win_post = make_win<CellT>(ctl->tm, D.geo.P, D.geo.k - 1u);
  const bool sat = re_full || (re_map && host_saturated(D.re_sat, D.geo.v, D.geo.u, mycol, lane));
  const uint32_t cw =
      sat ? D.geo.g
          : union_count<CellT>(static_cast<const CellT*>(D.re), D.geo.v, D.geo.g, D.geo.u, mycol, win_post, lane);
  if (lane == 0 && cw >= D.geo.rho_g) {
    uint32_t slot;
    const int r = set_insert(D.ctab[par ^ 1], D.cmask, slice_tag(T + 1), aip, &slot);
    if (r == 1) {
      D.cflags[par ^ 1][slot] = SRLA_CARRIED;
      const unsigned at = atomicAdd(&ctl->cat_count[par ^ 1], 1u);
      if (at < D.cmax)
        D.clist[par ^ 1][at] = aip;
      else
        atomicOr(&ctl->overflow_next, 2u);
    } else if (r < 0) {
      atomicOr(&ctl->overflow_next, 2u);
    }
  }
}

// The last block closes every link's slice and gathers the links' statistics into one
// array (copied to the host with a single transfer), then resets the group counters.
__global__ void __launch_bounds__(256) kg_estimate(const LinkDesc* __restrict__ descs, GroupCtl* __restrict__ gctl,
                                                   srla_slice_stats* __restrict__ gstats,
                                                   const uint32_t* __restrict__ rep_off, srla_entry* __restrict__ grep) {
  __shared__ int s_last;
  const int lane = threadIdx.x & 31;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const unsigned nl = gctl->n_links;
  const uint32_t total = rep_off[nl];  // every link's candidates in one flat range
  // 2 * total tasks: the estimate of every candidate, then the carry test of every candidate
  for (uint32_t t = gw; t < 2 * total; t += nw) {
    const bool est = t < total;
    const uint32_t i = est ? t : t - total;
    const unsigned l = link_of(rep_off, nl, i);
    const LinkDesc& D = descs[l];
    const uint32_t off = rep_off[l];
    const uint32_t cap = gctl->rep_cap > off ? gctl->rep_cap - off : 0u;
    with_cells(D.cell_bytes,
               [&](auto cell) { group_estimate_one<decltype(cell)>(D, i - off, est, lane, grep + off, cap, gctl); });
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&gctl->blocks_done, 1u) == gridDim.x - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (unsigned l = threadIdx.x; l < nl; l += blockDim.x) {
    const LinkDesc& D = descs[l];
    if (!D.active) continue;
    const int par = (int)(D.ctl->T & 1);
    close_slice(D.geo, D.ctl, D.st[par], D.umax, D.cmax);
    gstats[l] = *D.st[par];
    gstats[l].overflow |= gctl->overflow & 6u;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    gctl->blocks_done = 0;
    gctl->next_task = 0;
    gctl->bar_count = 0;
    gctl->overflow = 0;
    __threadfence();
  }
}

}  // namespace srla
