// libsrla: the C-ABI of the SRLA hot path (declared in include/srla.h).
//
// Host code here only validates arguments, lays out the caller's workspace, enqueues the
// kernels of kernels.cuh / sort.cuh on the caller's stream and moves reports and
// checkpoints across PCIe.  Every step of the method runs on the GPU.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "host_layout.h"
#include "kernels.cuh"
#include "sort.cuh"

using namespace srla;
using namespace srla::host;

// Host batches go through a ring of kStageBufs staging parts, copied on kCopyStreams
// internal streams in turn.
constexpr int kStageBufs = 2;
constexpr int kCopyStreams = 2;

struct srla_s {
  srla_params p;
  Geo geo;
  Coef coef;
  Layout L;
  char* ws;
  cudaStream_t st;
  cudaStream_t st_copy;  // internal stream for report remainders and checkpoints
  cudaStream_t st_h2d[kCopyStreams];  // internal streams: host-to-device copies of host batches
  cudaStream_t st_side;  // internal stream: the estimator table beside filter and sort
  cudaStream_t st_d2h;   // internal stream: each slice's report header, after its slice end
  cudaEvent_t ev_fork, ev_join, ev_swept;
  cudaEvent_t ev_done[2];  // slice end complete, by slice parity
  cudaEvent_t ev_ready[kStageBufs], ev_free[kStageBufs];  // staging parts: copied / consumed by the scan
  bool free_pending[kStageBufs];
  int stage_cur;
  int sms;
  bool k_is_P;
  uint64_t T;             // open slice
  uint64_t n_pkts_open;   // packets pushed into the open slice
  uint64_t staging_used;  // staging packets used in the open slice
  uint64_t launches;      // kernels launched so far
  uint32_t scan_build;    // SRLA_SCAN_AUTO, _PLAIN, _READ_FIRST or _HEAVY
  uint64_t scans[3];      // scan launches of the plain, read-first and heavy builds
  int occ_scan[2];        // resident scan blocks per SM (unaligned, aligned batches)
  int occ_sweep;          // resident sweep blocks per SM
  int sort_grid;          // blocks of the cooperative sort
  cudaGraphExec_t graph[2];    // captured slice end, by slice parity
  uint64_t graph_launches;     // kernels per captured slice end
  struct Slot {
    uint64_t slice, n_pkts;
    bool valid;
    cudaEvent_t ev;
    srla_slice_stats* h_stats;
    srla_entry* h_entries;
  } slot[2];
  void* h_pinned;

  template <typename T>
  T* at(size_t off) const {
    return reinterpret_cast<T*>(ws + off);
  }
  Ctl* ctl() const { return at<Ctl>(L.ctl); }
};

namespace {

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return SRLA_OK;
  (void)cudaGetLastError();
  return SRLA_E_CUDA;
}

#define SRLA_TRY(x)                       \
  do {                                    \
    const int _r = cuda_err(x);           \
    if (_r != SRLA_OK) return _r;         \
  } while (0)

// Calls f with a value of the handle's recorder storage type (one-bit, 8-bit or 16-bit).
template <typename F>
int with_cells(uint32_t dr_bytes, F&& f) {
  if (dr_bytes == 1) return f(uint8_t{});
  if (dr_bytes == 2) return f(uint16_t{});
  return f(Bit{});
}

int grid_for(uint64_t items, int per_block, int cap) {
  const uint64_t b = (items + per_block - 1) / per_block;
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(b, (uint64_t)cap));
}

bool inline_mode(const srla_t* h) { return h->p.mode == SRLA_MODE_INLINE; }

// The pair table of slice T (none when the table is disabled).
unsigned long long* pair_table(const srla_t* h, uint64_t T) {
  if (!h->L.n_ptab) return nullptr;
  return h->at<unsigned long long>(h->L.ptab[h->L.n_ptab == 2 ? (int)(T & 1) : 0]);
}

// The candidate-set and indicator arrays the inline candidate test writes.
InlineArgs inline_args(const srla_t* h) {
  const Layout& L = h->L;
  InlineArgs a{};
  for (int q = 0; q < 2; q++) {
    a.si[q] = inline_mode(h) ? h->at<uint32_t>(L.si[q]) : nullptr;
    a.ctab[q] = h->at<unsigned long long>(L.ctab[q]);
    a.cflags[q] = h->at<uint32_t>(L.cflags[q]);
    a.clist[q] = h->at<uint32_t>(L.clist[q]);
  }
  a.cmask = L.cmask;
  a.cmax = h->p.max_candidates;
  return a;
}

// Read-first scan (8/16-bit recorders, order-free mode) when the newest slice whose report
// has reached the host ran with the pair table off: most pairs are then new, and a good share
// of their stores would repeat a stamp already in place.  The hint is one or two slices old
// and never waits; either scan gives the same recorders.
// The newest slice whose report copy has reached the host (one or two slices old; never
// waits), or null.
const srla_s::Slot* newest_reported(const srla_t* h) {
  for (uint64_t back = 1; back <= 2 && back <= h->T; back++) {
    const srla_s::Slot& s = h->slot[(h->T - back) & 1];
    if (!s.valid || s.slice != h->T - back) continue;
    if (cudaEventQuery(s.ev) != cudaSuccess) continue;
    return &s;
  }
  return nullptr;
}

bool read_first_hint(const srla_t* h) {
  const srla_s::Slot* s = newest_reported(h);
  if (!s) return false;
  const srla_slice_stats& st = *s->h_stats;
  return next_pair_mode(st.pair_table, st.n_claims, st.n_claim_repeats, st.slice) == 0;
}

// Heavy build (8/16-bit recorders, order-free rule, runs that fit the block's bitmaps) when
// the newest reported slice close switched heavy-host tracking on.
bool heavy_possible(const srla_t* h) {
  return h->p.dr_bytes != 0 && !inline_mode(h) && h->p.u * h->p.gl <= kHeavyLeBits && h->p.u * h->p.g <= kHeavyReBits;
}

bool heavy_hint(const srla_t* h) {
  const srla_s::Slot* s = newest_reported(h);
  return s && next_heavy_mode(s->h_stats->n_scanned, s->h_stats->n_heavy_events) != 0;
}

template <typename CellT>
int launch_scan(srla_t* h, const uint32_t* pairs, uint64_t n) {
  const bool vec = (reinterpret_cast<uintptr_t>(pairs) & 15u) == 0;
  const bool elide = !kIsBit<CellT> && !inline_mode(h) &&
                     (h->scan_build == SRLA_SCAN_READ_FIRST || (h->scan_build == SRLA_SCAN_AUTO && read_first_hint(h)));
  const bool heavy = !kIsBit<CellT> && !elide && heavy_possible(h) &&
                     (h->scan_build == SRLA_SCAN_HEAVY || (h->scan_build == SRLA_SCAN_AUTO && heavy_hint(h)));
  h->scans[elide ? 1 : heavy ? 2 : 0]++;
  auto kern = inline_mode(h) ? (vec ? k_scan<CellT, true, true> : k_scan<CellT, false, true>)
              : elide        ? (vec ? k_scan<CellT, true, false, true> : k_scan<CellT, false, false, true>)
              : heavy        ? (vec ? k_scan<CellT, true, false, false, true> : k_scan<CellT, false, false, false, true>)
                             : (vec ? k_scan<CellT, true> : k_scan<CellT, false>);
  const int threads = inline_mode(h) ? kScanThreadsInline : kScanThreads;
  const size_t smem = inline_mode(h) ? scan_smem_bytes<true>() : scan_smem_bytes<false>();
  const int grid = grid_for(n, threads * 4, h->sms * std::max(1, h->occ_scan[vec ? 1 : 0]));
  CellT* re = h->at<CellT>(h->L.re);
  CellT* le = h->at<CellT>(h->L.le);
  h->launches++;
  kern<<<grid, threads, smem, h->st>>>(pairs, n, h->geo, h->coef, re, le, h->ctl(),
                                         h->at<unsigned long long>(h->L.utab), h->L.umask,
                                         h->at<uint32_t>(h->L.ulist), h->p.max_sampled,
                                         pair_table(h, h->T), h->L.pmask,
                                         inline_args(h));
  return cuda_err(cudaGetLastError());
}

// One wave of resident blocks (sms * occupancy) in all, shared between the SLE and SRE rows
// in proportion to their lengths (at least one block per row, at most one per 1024 vectors);
// a second, partial wave would leave most SMs idle at its end.
template <typename CellT>
int launch_sweep(srla_t* h, int census, int reset, int after_close) {
  const srla_params& p = h->p;
  const double le_row = (double)cell_array_bytes<CellT>((size_t)p.v * p.gl) / 16;
  const double re_row = (double)cell_array_bytes<CellT>((size_t)p.v * p.g) / 16;
  const double target = (double)h->sms * h->occ_sweep / p.u;  // blocks per (SLE row + SRE row)
  const double share = reset ? le_row / (le_row + re_row) : 1.0;
  auto blocks = [](double want, double vecs) {
    return (uint32_t)std::max(1.0, std::min(std::floor(want), std::ceil(vecs / 1024)));
  };
  const uint32_t gx_le = blocks(target * share, le_row);
  const uint32_t gx_re = reset ? blocks(target * (1.0 - share), re_row) : 0u;
  const uint32_t grid = p.u * (gx_le + gx_re);
  h->launches++;
  k_sweep<CellT><<<grid, 256, 0, h->st>>>(h->geo, h->at<CellT>(h->L.re), h->at<CellT>(h->L.le), h->ctl(), census,
                                          reset, after_close, gx_le, gx_re, h->at<uint8_t>(h->L.le_sat),
                                          h->at<uint8_t>(h->L.re_sat), h->L.le_spv, h->L.re_spv);
  return cuda_err(cudaGetLastError());
}

int launch_sort(srla_t* h, cudaStream_t st) {
  const Layout& L = h->L;
  Ctl* ctl = h->ctl();
  uint32_t* l0 = h->at<uint32_t>(L.clist[0]);
  uint32_t* l1 = h->at<uint32_t>(L.clist[1]);
  uint32_t cmax = h->p.max_candidates;
  uint32_t* tmp = h->at<uint32_t>(L.sort_tmp);
  uint32_t* hist = h->at<uint32_t>(L.sort_hist);
  void* args[] = {&ctl, &l0, &l1, &tmp, &cmax, &hist};
  h->launches++;
  return cuda_err(cudaLaunchCooperativeKernel((const void*)k_sort, dim3(h->sort_grid), dim3(kSortThreads), args,
                                              kSortSmallSmem, st));
}

// The next slice starts with an empty pair table (all slots hold the empty key, ~0).
// Pair table q (of L.n_ptab) starts empty: every slot holds the empty key, ~0.
int clear_pairs(srla_t* h, int q, cudaStream_t st) {
  if (q >= h->L.n_ptab) return SRLA_OK;
  return cuda_err(cudaMemsetAsync(h->ws + h->L.ptab[q], 0xFF, ((size_t)h->L.pmask + 1) * 8, st));
}

int clear_pairs(srla_t* h) {
  int r = clear_pairs(h, 0, h->st);
  return r != SRLA_OK ? r : clear_pairs(h, 1, h->st);
}

// Recorder arrays up to this size are swept in about the time the candidate filter and sort
// take, so those two run beside the sweep; a longer sweep is not delayed by them.
constexpr size_t kOverlapSweepBytes = (size_t)128 << 20;

// The slice end of the open slice, whose index has parity q.
//
// Overlapped schedule (side stream, recorder arrays up to kOverlapSweepBytes): the candidate
// filter and sort run beside the sweep.  They read the SRE only through the window test, and
// the only SRE cells the sweep may change (when k < P) hold the alias stamp, which is outside
// the window; with k = P the census sweep changes nothing.  The Eq. 8/9 table follows the
// census on the main stream.  Otherwise the table runs beside the filter and sort, after the
// sweep.  Either way the next slice's pair table (used two slices ago; with two tables) is
// cleared on the side stream after the sweep, so that it is still in L2 when the next scan
// starts, and the estimate waits for everything; a single table is cleared at the end.
template <typename CellT>
int launch_end_slice(srla_t* h, int q) {
  const Layout& L = h->L;
  const bool inl = inline_mode(h);
  const bool two = h->L.n_ptab == 2;
  const bool overlap = h->st_side && L.le + cell_array_bytes<CellT>((size_t)h->p.u * h->p.v * h->p.gl) - L.re <=
                                         kOverlapSweepBytes;
  // one warp per 32 table entries, spread over the SMs (FP64 throughput is per SM)
  const int lut_grid = (int)std::min<uint32_t>((h->p.gl + 1 + 31) / 32, (uint32_t)h->sms * 8);
  int r;
  h->launches += inl ? 2 : 3;  // lut, (filter,) estimate
  auto filter_and_sort = [&](cudaStream_t st) -> int {
    if (!inl)  // the inline mode found its new candidates during the scan
      k_filter<CellT><<<h->sms * 4, 256, 0, st>>>(
          h->geo, h->coef, h->at<CellT>(L.re), h->ctl(), h->at<uint32_t>(L.ulist), h->p.max_sampled,
          h->at<unsigned long long>(L.ctab[0]), h->at<unsigned long long>(L.ctab[1]), h->at<uint32_t>(L.cflags[0]),
          h->at<uint32_t>(L.cflags[1]), L.cmask, h->at<uint32_t>(L.clist[0]), h->at<uint32_t>(L.clist[1]),
          h->p.max_candidates);
    return launch_sort(h, st);
  };
  auto lut = [&](cudaStream_t st) {
    k_lut<<<lut_grid, 32, 0, st>>>(h->geo, h->ctl(), h->at<float>(L.lut_est), h->at<uint32_t>(L.lut_flags));
  };
  if (overlap) {
    SRLA_TRY(cudaEventRecord(h->ev_fork, h->st));
    SRLA_TRY(cudaStreamWaitEvent(h->st_side, h->ev_fork, 0));
    if ((r = filter_and_sort(h->st_side)) != SRLA_OK) return r;
  }
  if ((r = launch_sweep<CellT>(h, 1, h->k_is_P ? 0 : 1, 0)) != SRLA_OK) return r;
  if (h->st_side) {
    SRLA_TRY(cudaEventRecord(h->ev_swept, h->st));
    SRLA_TRY(cudaStreamWaitEvent(h->st_side, h->ev_swept, 0));
    if (!overlap) lut(h->st_side);
    if (two && (r = clear_pairs(h, q ^ 1, h->st_side)) != SRLA_OK) return r;
    SRLA_TRY(cudaEventRecord(h->ev_join, h->st_side));
    if (overlap)
      lut(h->st);
    else if ((r = filter_and_sort(h->st)) != SRLA_OK)
      return r;
    SRLA_TRY(cudaStreamWaitEvent(h->st, h->ev_join, 0));
  } else {
    lut(h->st);
    if ((r = filter_and_sort(h->st)) != SRLA_OK) return r;
    if (two && (r = clear_pairs(h, q ^ 1, h->st)) != SRLA_OK) return r;
  }
  // Algorithm 3 clears every SI before the carried hosts set theirs for the next slice
  if (inl) SRLA_TRY(cudaMemsetAsync(h->ws + L.si[q ^ 1], 0, (size_t)h->p.u * h->p.v * 4, h->st));
  k_estimate<CellT><<<h->sms * 2, 256, 0, h->st>>>(
      h->geo, h->coef, h->at<CellT>(L.re), h->at<CellT>(L.le), h->ctl(), h->at<unsigned long long>(L.ctab[0]),
      h->at<unsigned long long>(L.ctab[1]), h->at<uint32_t>(L.cflags[0]), h->at<uint32_t>(L.cflags[1]), L.cmask,
      h->at<uint32_t>(L.clist[0]), h->at<uint32_t>(L.clist[1]), h->p.max_candidates,
      h->at<srla_entry>(L.rep_entries[0]), h->at<srla_entry>(L.rep_entries[1]),
      h->at<srla_slice_stats>(L.rep_stats[0]), h->at<srla_slice_stats>(L.rep_stats[1]), h->p.max_sampled,
      h->at<float>(L.lut_est), h->at<uint32_t>(L.lut_flags), inl ? h->at<uint32_t>(L.si[0]) : nullptr,
      inl ? h->at<uint32_t>(L.si[1]) : nullptr, h->at<uint8_t>(L.le_sat), h->at<uint8_t>(L.re_sat),
      (L.le_spv ? 1u : 0u) | (L.re_spv ? 2u : 0u));
  SRLA_TRY(cudaGetLastError());
  // with k = 2^z - 1 the recorders that saturate are still inside the window of the closed
  // slice, so they are cleared only after the slice was estimated and closed
  if (h->k_is_P && (r = launch_sweep<CellT>(h, 0, 1, 1)) != SRLA_OK) return r;
  return two ? SRLA_OK : clear_pairs(h, 0, h->st);
}

// The copy of slice q's statistics and first report entries into its pinned slot, on the
// report stream once the slice end is complete; the next slice's scan does not wait for it.
// The entries follow the statistics in the workspace (rep_entries[q] = rep_stats[q] +
// report_gap(L)) and in the slot alike, so one copy moves both.
int enqueue_report_copy(srla_t* h, int q) {
  srla_s::Slot& s = h->slot[q];
  SRLA_TRY(cudaEventRecord(h->ev_done[q], h->st));
  SRLA_TRY(cudaStreamWaitEvent(h->st_d2h, h->ev_done[q], 0));
  const uint32_t pre = std::min<uint32_t>(kPrefetch, h->p.max_candidates);
  SRLA_TRY(cudaMemcpyAsync(s.h_stats, h->ws + h->L.rep_stats[q], report_gap(h->L) + (size_t)pre * sizeof(srla_entry),
                           cudaMemcpyDeviceToHost, h->st_d2h));
  SRLA_TRY(cudaEventRecord(s.ev, h->st_d2h));
  return SRLA_OK;
}

// Capture the slice end once per parity into an executable graph: every kernel reads the
// open slice from the control block, so the same graph serves every slice of that parity.
int capture_graphs(srla_t* h) {
  cudaStream_t user = h->st;
  h->st = h->st_copy;
  int rc = SRLA_OK;
  for (int q = 0; q < 2 && rc == SRLA_OK; q++) {
    cudaGraph_t g = nullptr;
    const uint64_t before = h->launches;
    if (cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = SRLA_E_CUDA;
      break;
    }
    rc = with_cells(h->p.dr_bytes, [&](auto c) { return launch_end_slice<decltype(c)>(h, q); });
    const cudaError_t e = cudaStreamEndCapture(h->st, &g);
    if (rc == SRLA_OK && e != cudaSuccess) rc = SRLA_E_CUDA;
    if (rc == SRLA_OK && cudaGraphInstantiate(&h->graph[q], g, 0) != cudaSuccess) rc = SRLA_E_CUDA;
    if (g) cudaGraphDestroy(g);
    h->graph_launches = h->launches - before;
    h->launches = before;
  }
  h->st = user;
  if (rc != SRLA_OK) (void)cudaGetLastError();
  return rc;
}

// Zero the control block and both candidate/sampled set tables (fresh tags).
int reset_tables(srla_t* h, bool all) {
  const Layout& L = h->L;
  SRLA_TRY(cudaMemsetAsync(h->ws + L.utab, 0, ((size_t)L.umask + 1) * 8, h->st));
  for (int q = 0; q < 2; q++) SRLA_TRY(cudaMemsetAsync(h->ws + L.ctab[q], 0, ((size_t)L.cmask + 1) * 8, h->st));
  if (all) SRLA_TRY(cudaMemsetAsync(h->ws, 0, L.total, h->st));
  return clear_pairs(h);
}

// Resident blocks per SM of the scan and of the sweep, and the cooperative sort's grid (all
// co-resident).
int occupancy(srla_t* h) {
  int a = 0, b = 0, c = 0, sw = 0;
  const int rs = with_cells(h->p.dr_bytes, [&](auto cell) {
    using CellT = decltype(cell);
    const bool inl = inline_mode(h);
    auto k0 = inl ? k_scan<CellT, false, true> : k_scan<CellT, false>;
    auto k1 = inl ? k_scan<CellT, true, true> : k_scan<CellT, true>;
    const int threads = inl ? kScanThreadsInline : kScanThreads;
    const size_t smem = inl ? scan_smem_bytes<true>() : scan_smem_bytes<false>();
    if (cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_scan<CellT, false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)scan_smem_bytes<false>()) != cudaSuccess ||
        cudaFuncSetAttribute(k_scan<CellT, true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)scan_smem_bytes<false>()) != cudaSuccess ||
        cudaFuncSetAttribute(k_scan<CellT, false, false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)scan_smem_bytes<false>()) != cudaSuccess ||
        cudaFuncSetAttribute(k_scan<CellT, true, false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)scan_smem_bytes<false>()) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k0, threads, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k1, threads, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sw, k_sweep<CellT>, 256, 0) != cudaSuccess)
      return SRLA_E_CUDA;
    return SRLA_OK;
  });
  if (rs != SRLA_OK) return rs;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_sort, kSortThreads, kSortSmallSmem) != cudaSuccess || c < 1)
    return SRLA_E_CUDA;
  h->occ_scan[0] = std::max(1, a);
  h->occ_scan[1] = std::max(1, b);
  h->occ_sweep = std::max(1, sw);
  h->sort_grid = (int)std::max<uint32_t>(1, std::min<uint32_t>(h->L.ntiles, (uint32_t)(h->sms * c)));
  return SRLA_OK;
}

int init_ctl(srla_t* h, uint64_t T, uint32_t carried) {
  Ctl c{};
  c.T = T;
  c.tm = (uint32_t)(T % h->geo.P);
  c.w_star = h->geo.gl + 1;
  c.pair_mode = 1;
  c.cat_count[T & 1] = carried;
  SRLA_TRY(cudaMemcpyAsync(h->ctl(), &c, sizeof(Ctl), cudaMemcpyHostToDevice, h->st));
  return cudaStreamSynchronize(h->st) == cudaSuccess ? SRLA_OK : SRLA_E_CUDA;
}

}  // namespace

extern "C" {

int srla_check_params(const srla_params* p) { return check(p); }

size_t srla_workspace_bytes(const srla_params* p) {
  if (check(p) != SRLA_OK) return 0;
  return layout_of(p).total;
}

int srla_derived(const srla_params* p, uint32_t* tau, uint32_t* rho_g, uint32_t* stamp_mod) {
  if (check(p) != SRLA_OK) return SRLA_E_INVAL;
  if (tau) *tau = tau_of(p->theta, p->g);
  if (rho_g) *rho_g = rho_g_of(p->g);
  if (stamp_mod) *stamp_mod = (1u << p->z) - 1u;
  return SRLA_OK;
}

int srla_create(const srla_params* p, void* dev_workspace, size_t ws_bytes, void* stream, srla_t** out) {
  if (!out) return SRLA_E_INVAL;
  *out = nullptr;
  if (check(p) != SRLA_OK || !dev_workspace) return SRLA_E_INVAL;
  if (reinterpret_cast<uintptr_t>(dev_workspace) % kAlign) return SRLA_E_INVAL;
  const Layout L = layout_of(p);
  if (ws_bytes < L.total) return SRLA_E_NOMEM;
  srla_t* h = new (std::nothrow) srla_s();
  if (!h) return SRLA_E_NOMEM;
  h->p = *p;
  h->L = L;
  h->ws = static_cast<char*>(dev_workspace);
  h->st = static_cast<cudaStream_t>(stream);
  const uint32_t tau = tau_of(p->theta, p->g);
  h->geo = Geo{p->u, p->v, p->g, p->gl, p->v - 1, p->g - 1, p->gl - 1, p->k, (1u << p->z) - 1u,
               tau >= 32 ? 0xFFFFFFFFu : ((1u << tau) - 1u), rho_g_of(p->g), p->theta};
  for (int r = 0; r < SRLA_N_HASH; r++) {
    h->coef.a[r] = p->hash_a[r];
    h->coef.b[r] = p->hash_b[r];
  }
  h->k_is_P = (p->k == h->geo.P);
  h->T = p->start_slice;
  int dev = 0, rc = SRLA_OK;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete h;
    return cuda_err(cudaErrorUnknown);
  }
  const size_t per_slot = report_gap(h->L) + (size_t)kPrefetch * sizeof(srla_entry);
  if (cudaHostAlloc(&h->h_pinned, 2 * per_slot, cudaHostAllocDefault) != cudaSuccess) {
    delete h;
    return cuda_err(cudaErrorMemoryAllocation);
  }
  if (cudaStreamCreateWithFlags(&h->st_copy, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFreeHost(h->h_pinned);
    delete h;
    return SRLA_E_CUDA;
  }
  for (cudaStream_t& cs : h->st_h2d)
    if (rc == SRLA_OK && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) rc = SRLA_E_CUDA;
  if (rc == SRLA_OK && (cudaStreamCreateWithFlags(&h->st_side, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaStreamCreateWithFlags(&h->st_d2h, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
                        cudaEventCreateWithFlags(&h->ev_swept, cudaEventDisableTiming) != cudaSuccess ||
                        cudaEventCreateWithFlags(&h->ev_done[0], cudaEventDisableTiming) != cudaSuccess ||
                        cudaEventCreateWithFlags(&h->ev_done[1], cudaEventDisableTiming) != cudaSuccess))
    rc = SRLA_E_CUDA;
  for (int q = 0; q < kStageBufs && rc == SRLA_OK; q++) {
    if (cudaEventCreateWithFlags(&h->ev_ready[q], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_free[q], cudaEventDisableTiming) != cudaSuccess)
      rc = SRLA_E_CUDA;
  }
  for (int q = 0; q < 2; q++) {
    h->slot[q].valid = false;
    h->slot[q].h_stats = reinterpret_cast<srla_slice_stats*>(static_cast<char*>(h->h_pinned) + q * per_slot);
    h->slot[q].h_entries = reinterpret_cast<srla_entry*>(reinterpret_cast<char*>(h->slot[q].h_stats) +
                                                         report_gap(h->L));
    if (cudaEventCreateWithFlags(&h->slot[q].ev, cudaEventDisableTiming) != cudaSuccess) rc = SRLA_E_CUDA;
  }
  if (rc == SRLA_OK) {
    cudaFuncSetAttribute(k_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSortSmallSmem);
    rc = occupancy(h);
  }
  if (rc == SRLA_OK) rc = reset_tables(h, true);
  if (rc == SRLA_OK) rc = init_ctl(h, h->T, 0);
  if (rc == SRLA_OK && capture_graphs(h) != SRLA_OK) {
    // the slice end then runs as individual launches on the caller's stream
    for (int q = 0; q < 2; q++) {
      if (h->graph[q]) cudaGraphExecDestroy(h->graph[q]);
      h->graph[q] = nullptr;
    }
  }
  if (rc != SRLA_OK) {
    srla_destroy(h);
    return rc;
  }
  *out = h;
  return SRLA_OK;
}

int srla_push_packets(srla_t* h, const uint32_t* pairs, uint64_t n_pairs, int on_device) {
  if (!h || (!pairs && n_pairs)) return SRLA_E_INVAL;
  if (n_pairs == 0) return SRLA_OK;
  auto scan = [&](const uint32_t* src, uint64_t n) {
    return with_cells(h->p.dr_bytes, [&](auto c) { return launch_scan<decltype(c)>(h, src, n); });
  };
  if (on_device) {
    const int r = scan(pairs, n_pairs);
    if (r == SRLA_OK) h->n_pkts_open += n_pairs;
    return r;
  }
  // Staging ring: the copies of the parts run back to back on the internal copy stream(s),
  // while the caller's stream scans each part once it has arrived; a part is copied into
  // again only after its last scan (events order the reuse), so the copy of the next parts
  // never waits on the scans of the previous ones.
  uint32_t* staging = h->at<uint32_t>(h->L.staging);
  const uint64_t part = std::max<uint64_t>(2, (h->L.staging_pkts / kStageBufs) & ~1ull);
  while (n_pairs) {
    const int x = h->stage_cur;
    h->stage_cur = (x + 1) % kStageBufs;
    const uint64_t m = std::min<uint64_t>(n_pairs, part);
    uint32_t* dst = staging + 2 * part * (uint64_t)x;
    cudaStream_t cs = h->st_h2d[x % kCopyStreams];
    if (h->free_pending[x]) SRLA_TRY(cudaStreamWaitEvent(cs, h->ev_free[x], 0));
    SRLA_TRY(cudaMemcpyAsync(dst, pairs, m * 8, cudaMemcpyHostToDevice, cs));
    SRLA_TRY(cudaEventRecord(h->ev_ready[x], cs));
    SRLA_TRY(cudaStreamWaitEvent(h->st, h->ev_ready[x], 0));
    const int r = scan(dst, m);
    if (r != SRLA_OK) return r;
    SRLA_TRY(cudaEventRecord(h->ev_free[x], h->st));
    h->free_pending[x] = true;
    h->n_pkts_open += m;
    pairs += 2 * m;
    n_pairs -= m;
  }
  return SRLA_OK;
}

int srla_end_slice(srla_t* h, uint64_t* slice_id) {
  if (!h) return SRLA_E_INVAL;
  const int q = (int)(h->T & 1);
  srla_s::Slot& s = h->slot[q];
  if (h->graph[q]) {
    SRLA_TRY(cudaGraphLaunch(h->graph[q], h->st));
    h->launches += h->graph_launches;
  } else {
    const int r = with_cells(h->p.dr_bytes, [&](auto c) { return launch_end_slice<decltype(c)>(h, q); });
    if (r != SRLA_OK) return r;
  }
  if (const int r = enqueue_report_copy(h, q); r != SRLA_OK) return r;
  s.slice = h->T;
  s.n_pkts = h->n_pkts_open;
  s.valid = true;
  if (slice_id) *slice_id = h->T;
  h->T++;
  h->n_pkts_open = 0;
  h->staging_used = 0;
  if ((h->T & 0x7FFFFFFFull) == 0) {
    // The 31-bit set tag wraps: start the new slice on cleared tables.  The carried list of
    // the new slice sits in the table being cleared, so re-insert it from its list.
    SRLA_TRY(cudaStreamSynchronize(h->st));
    Ctl c;
    SRLA_TRY(cudaMemcpy(&c, h->ctl(), sizeof(Ctl), cudaMemcpyDeviceToHost));
    const uint32_t nc = std::min<uint32_t>(c.cat_count[h->T & 1], h->p.max_candidates);
    int rr = reset_tables(h, false);
    if (rr != SRLA_OK) return rr;
    c.cat_count[h->T & 1] = 0;
    SRLA_TRY(cudaMemcpyAsync(h->ctl(), &c, sizeof(Ctl), cudaMemcpyHostToDevice, h->st));
    const Layout& L = h->L;
    if (nc) {
      // copy the list aside (into the sort scratch) before re-inserting it into its own table
      SRLA_TRY(cudaMemcpyAsync(h->ws + L.sort_tmp, h->ws + L.clist[h->T & 1], (size_t)nc * 4,
                               cudaMemcpyDeviceToDevice, h->st));
      h->launches++;
      k_insert_carried<<<grid_for(nc, 256, h->sms * 4), 256, 0, h->st>>>(
          h->at<uint32_t>(L.sort_tmp), nc, h->ctl(), h->at<unsigned long long>(L.ctab[0]),
          h->at<unsigned long long>(L.ctab[1]), h->at<uint32_t>(L.cflags[0]), h->at<uint32_t>(L.cflags[1]),
          L.cmask, h->at<uint32_t>(L.clist[0]), h->at<uint32_t>(L.clist[1]), h->p.max_candidates, h->geo, h->coef,
          nullptr);  // the SI bits of the carried hosts are already set
      SRLA_TRY(cudaGetLastError());
    }
  }
  return SRLA_OK;
}

int srla_report(srla_t* h, uint64_t slice_id, srla_entry* out, size_t cap, size_t* n_out,
                srla_slice_stats* stats) {
  if (!h || (cap && !out)) return SRLA_E_INVAL;
  const int q = (int)(slice_id & 1);
  srla_s::Slot& s = h->slot[q];
  if (!s.valid || s.slice != slice_id) return SRLA_E_ORDER;
  SRLA_TRY(cudaEventSynchronize(s.ev));
  srla_slice_stats st = *s.h_stats;
  st.n_pkts = s.n_pkts;
  const size_t n = st.n_candidates;
  if (n_out) *n_out = n;
  if (stats) *stats = st;
  const size_t take = std::min(n, cap);
  const size_t pre = std::min<size_t>(take, std::min<uint32_t>(kPrefetch, h->p.max_candidates));
  if (pre) std::memcpy(out, s.h_entries, pre * sizeof(srla_entry));
  if (take > pre) {
    SRLA_TRY(cudaMemcpyAsync(out + pre, h->ws + h->L.rep_entries[q] + pre * sizeof(srla_entry),
                             (take - pre) * sizeof(srla_entry), cudaMemcpyDeviceToHost, h->st_copy));
    SRLA_TRY(cudaStreamSynchronize(h->st_copy));
  }
  if (st.overflow & 4u) return SRLA_E_TIMEOUT;
  if (st.overflow) return SRLA_E_CAPACITY;
  if (cap < n) return SRLA_E_NOMEM;
  return SRLA_OK;
}

int srla_sync(srla_t* h) {
  if (!h) return SRLA_E_INVAL;
  return cuda_err(cudaStreamSynchronize(h->st));
}

size_t srla_state_bytes(const srla_t* h) {
  if (!h) return 0;
  return state_bytes_of(&h->p, h->p.max_candidates);
}

}  // extern "C"

namespace {

template <typename CellT>
int export_cells(srla_t* h, size_t off, size_t n, uint16_t* dst) {
  // decode through the staging area, one chunk (a multiple of 32 recorders) at a time
  const size_t chunk = (h->L.staging_pkts * 8 / 2) & ~(size_t)31;  // uint16 per chunk
  uint16_t* stage = h->at<uint16_t>(h->L.staging);
  for (size_t x = 0; x < n; x += chunk) {
    const size_t m = std::min(chunk, n - x);
    h->launches++;
    k_decode<CellT><<<grid_for(m, 256, h->sms * 8), 256, 0, h->st>>>(cells_from(h->at<CellT>(off), x), stage, m,
                                                                      h->ctl(), h->geo.P);
    SRLA_TRY(cudaGetLastError());
    SRLA_TRY(cudaMemcpyAsync(dst + x, stage, m * 2, cudaMemcpyDeviceToHost, h->st));
    SRLA_TRY(cudaStreamSynchronize(h->st));
  }
  return SRLA_OK;
}

template <typename CellT>
int import_cells(srla_t* h, size_t off, size_t n, const uint16_t* src, uint32_t tm) {
  const size_t chunk = (h->L.staging_pkts * 8 / 2) & ~(size_t)31;
  uint16_t* stage = h->at<uint16_t>(h->L.staging);
  for (size_t x = 0; x < n; x += chunk) {
    const size_t m = std::min(chunk, n - x);
    SRLA_TRY(cudaMemcpyAsync(stage, src + x, m * 2, cudaMemcpyHostToDevice, h->st));
    h->launches++;
    k_encode<CellT><<<grid_for(m, 256, h->sms * 8), 256, 0, h->st>>>(stage, cells_from(h->at<CellT>(off), x), m,
                                                                      tm, h->geo.P);
    SRLA_TRY(cudaGetLastError());
    SRLA_TRY(cudaStreamSynchronize(h->st));
  }
  return SRLA_OK;
}

}  // namespace

extern "C" {

int srla_export_state(srla_t* h, void* host_buf, size_t cap) {
  if (!h || !host_buf) return SRLA_E_INVAL;
  if (h->n_pkts_open) return SRLA_E_ORDER;
  const srla_params& p = h->p;
  SRLA_TRY(cudaStreamSynchronize(h->st));
  Ctl c;
  SRLA_TRY(cudaMemcpy(&c, h->ctl(), sizeof(Ctl), cudaMemcpyDeviceToHost));
  const uint32_t nc = std::min<uint32_t>(c.cat_count[h->T & 1], p.max_candidates);
  const size_t nre = (size_t)p.u * p.v * p.g, nle = (size_t)p.u * p.v * p.gl;
  const size_t need = sizeof(StateHeader) + (nre + nle) * 2 + (size_t)nc * 4;
  if (cap < need) return SRLA_E_NOMEM;
  StateHeader hd{kStateMagic, kStateVersion, p.u, p.v, p.g, p.gl, p.dr_bytes, p.z, p.k, p.theta, h->T, nc, 0};
  char* b = static_cast<char*>(host_buf);
  std::memcpy(b, &hd, sizeof(hd));
  uint16_t* dre = reinterpret_cast<uint16_t*>(b + sizeof(hd));
  uint16_t* dle = dre + nre;
  int r = with_cells(p.dr_bytes, [&](auto c) { return export_cells<decltype(c)>(h, h->L.re, nre, dre); });
  if (r != SRLA_OK) return r;
  r = with_cells(p.dr_bytes, [&](auto c) { return export_cells<decltype(c)>(h, h->L.le, nle, dle); });
  if (r != SRLA_OK) return r;
  uint32_t* carry = reinterpret_cast<uint32_t*>(dle + nle);
  if (nc) {
    SRLA_TRY(cudaMemcpy(carry, h->ws + h->L.clist[h->T & 1], (size_t)nc * 4, cudaMemcpyDeviceToHost));
    std::sort(carry, carry + nc);
  }
  return SRLA_OK;
}

int srla_import_state(srla_t* h, const void* host_buf, size_t len) {
  if (!h || !host_buf || len < sizeof(StateHeader)) return SRLA_E_INVAL;
  if (h->n_pkts_open) return SRLA_E_ORDER;
  const srla_params& p = h->p;
  StateHeader hd;
  std::memcpy(&hd, host_buf, sizeof(hd));
  if (hd.magic != kStateMagic || hd.version != kStateVersion || hd.u != p.u || hd.v != p.v || hd.g != p.g ||
      hd.gl != p.gl || hd.z != p.z || hd.k != p.k)
    return SRLA_E_INVAL;
  const size_t nre = (size_t)p.u * p.v * p.g, nle = (size_t)p.u * p.v * p.gl;
  if (len < sizeof(StateHeader) + (nre + nle) * 2 + (size_t)hd.n_carry * 4) return SRLA_E_INVAL;
  if (hd.n_carry > p.max_candidates) return SRLA_E_CAPACITY;
  SRLA_TRY(cudaStreamSynchronize(h->st));
  int r = reset_tables(h, false);
  if (r != SRLA_OK) return r;
  for (int q = 0; q < 2; q++) h->slot[q].valid = false;
  h->T = hd.slice;
  h->staging_used = 0;
  if ((r = init_ctl(h, h->T, 0)) != SRLA_OK) return r;
  const uint32_t tm = (uint32_t)(h->T % h->geo.P);
  const uint16_t* sre = reinterpret_cast<const uint16_t*>(static_cast<const char*>(host_buf) + sizeof(hd));
  const uint16_t* sle = sre + nre;
  r = with_cells(p.dr_bytes, [&](auto c) { return import_cells<decltype(c)>(h, h->L.re, nre, sre, tm); });
  if (r != SRLA_OK) return r;
  r = with_cells(p.dr_bytes, [&](auto c) { return import_cells<decltype(c)>(h, h->L.le, nle, sle, tm); });
  if (r != SRLA_OK) return r;
  uint32_t* si_open = inline_mode(h) ? h->at<uint32_t>(h->L.si[h->T & 1]) : nullptr;
  if (si_open) SRLA_TRY(cudaMemsetAsync(si_open, 0, (size_t)p.u * p.v * 4, h->st));
  if (hd.n_carry) {
    const uint32_t* carry = reinterpret_cast<const uint32_t*>(sle + nle);
    uint32_t* stage = h->at<uint32_t>(h->L.sort_tmp);
    SRLA_TRY(cudaMemcpyAsync(stage, carry, (size_t)hd.n_carry * 4, cudaMemcpyHostToDevice, h->st));
    const Layout& L = h->L;
    h->launches++;
    k_insert_carried<<<grid_for(hd.n_carry, 256, h->sms * 4), 256, 0, h->st>>>(
        stage, hd.n_carry, h->ctl(), h->at<unsigned long long>(L.ctab[0]), h->at<unsigned long long>(L.ctab[1]),
        h->at<uint32_t>(L.cflags[0]), h->at<uint32_t>(L.cflags[1]), L.cmask, h->at<uint32_t>(L.clist[0]),
        h->at<uint32_t>(L.clist[1]), p.max_candidates, h->geo, h->coef, si_open);
    SRLA_TRY(cudaGetLastError());
  }
  return cuda_err(cudaStreamSynchronize(h->st));
}

uint64_t srla_kernel_launches(const srla_t* h) { return h ? h->launches : 0; }

int srla_set_scan_build(srla_t* h, uint32_t build) {
  if (!h || build > SRLA_SCAN_HEAVY) return SRLA_E_INVAL;
  // the read-first build exists for 8- and 16-bit recorders under the order-free rule; the
  // heavy build, in addition, for runs that fit its bitmaps
  if (build == SRLA_SCAN_READ_FIRST && (h->p.dr_bytes == 0 || inline_mode(h))) return SRLA_E_INVAL;
  if (build == SRLA_SCAN_HEAVY && !heavy_possible(h)) return SRLA_E_INVAL;
  h->scan_build = build;
  return SRLA_OK;
}

int srla_scan_builds(const srla_t* h, uint64_t* plain, uint64_t* read_first, uint64_t* heavy) {
  if (!h) return SRLA_E_INVAL;
  if (plain) *plain = h->scans[0];
  if (read_first) *read_first = h->scans[1];
  if (heavy) *heavy = h->scans[2];
  return SRLA_OK;
}

int srla_uses_graph(const srla_t* h) { return h && h->graph[0] && h->graph[1] ? 1 : 0; }

void srla_destroy(srla_t* h) {
  if (!h) return;
  if (h->st_copy) {
    cudaStreamSynchronize(h->st);
    cudaStreamDestroy(h->st_copy);
  }
  for (cudaStream_t cs : h->st_h2d)
    if (cs) cudaStreamDestroy(cs);
  if (h->st_d2h) {
    cudaStreamSynchronize(h->st_d2h);
    cudaStreamDestroy(h->st_d2h);
  }
  if (h->st_side) cudaStreamDestroy(h->st_side);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_swept) cudaEventDestroy(h->ev_swept);
  for (int q = 0; q < 2; q++) {
    if (h->ev_done[q]) cudaEventDestroy(h->ev_done[q]);
    if (h->slot[q].ev) cudaEventDestroy(h->slot[q].ev);
    if (h->graph[q]) cudaGraphExecDestroy(h->graph[q]);
  }
  for (int q = 0; q < kStageBufs; q++) {
    if (h->ev_ready[q]) cudaEventDestroy(h->ev_ready[q]);
    if (h->ev_free[q]) cudaEventDestroy(h->ev_free[q]);
  }
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  delete h;
}

const char* srla_strerror(int code) {
  switch (code) {
    case SRLA_OK: return "ok";
    case SRLA_E_INVAL: return "invalid argument";
    case SRLA_E_NOMEM: return "insufficient memory or buffer";
    case SRLA_E_CAPACITY: return "per-slice capacity exceeded; results incomplete";
    case SRLA_E_CUDA: return "CUDA runtime error";
    case SRLA_E_ORDER: return "call out of order";
    case SRLA_E_TIMEOUT: return "device wait timed out";
    default: return "unknown error";
  }
}

}  // extern "C"

// ------------------------------------------------------ allocation-free batch report
//
// Some callers cannot allocate device memory at all: a capture thread with real-time
// deadlines (cudaMalloc and cudaFree may synchronize the whole device), or a plugin whose
// host framework owns every device buffer and hands out only fixed input/output slots.  For
// them, srla_batch_report_static runs the
// scan and the slice end of a fresh estimator over one device batch with its workspace
// carved out of a fixed scratch array compiled into this library, instead of a caller
// workspace.  Every GPU that loads the library holds the array until the process exits.

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[SRLA_STATIC_SCRATCH_BYTES];

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kStaticMaxDevices];  // device address of g_static_scratch, per device

// Once per device, with that device current: the device address of the scratch array (in
// host code the array's name is only a host-side stand-in) and the shared-memory opt-in of
// the single-block sort.
int static_scratch_setup(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_static_scratch) != cudaSuccess || !addr) return cuda_err(cudaErrorUnknown);
    if (cudaFuncSetAttribute(k_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSortSmallSmem) !=
        cudaSuccess)
      return cuda_err(cudaErrorUnknown);
    g_static_addr[dev] = addr;
  }
  *out = g_static_addr[dev];
  return SRLA_OK;
}

template <typename CellT>
int static_batch(srla_s* h, const uint32_t* d_pairs, uint64_t n_pairs) {
  int r = SRLA_OK;
  if (n_pairs && (r = launch_scan<CellT>(h, d_pairs, n_pairs)) != SRLA_OK) return r;
  return launch_end_slice<CellT>(h, (int)(h->T & 1));
}

}  // namespace

extern "C" int srla_batch_report_static(const srla_params* p, const uint32_t* d_pairs, uint64_t n_pairs,
                                        void* stream, srla_entry* out, size_t cap, size_t* n_out,
                                        srla_slice_stats* stats) {
  if (check(p) != SRLA_OK || (n_pairs && !d_pairs) || (cap && !out)) return SRLA_E_INVAL;
  // the call synchronizes the stream, which a stream being captured must not do (it would
  // end the caller's capture with an error): refuse before any other CUDA call
  cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
  SRLA_TRY(cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &capturing));
  if (capturing != cudaStreamCaptureStatusNone) return SRLA_E_INVAL;
  srla_params q = *p;
  q.staging_pkts = 2;  // the batch is already on the device: no host staging area
  const Layout L = layout_of(&q, 1);  // one slice: one pair table
  if (L.total > (size_t)SRLA_STATIC_SCRATCH_BYTES) return SRLA_E_NOMEM;
  int dev = 0;
  SRLA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kStaticMaxDevices) return SRLA_E_INVAL;
  void* base = nullptr;
  int r = static_scratch_setup(dev, &base);
  if (r != SRLA_OK) return r;

  srla_s h{};  // lives on this stack frame; no events, pinned buffers or streams are made
  h.p = q;
  h.L = L;
  h.ws = static_cast<char*>(base);
  h.st = static_cast<cudaStream_t>(stream);
  const uint32_t tau = tau_of(q.theta, q.g);
  h.geo = Geo{q.u, q.v, q.g, q.gl, q.v - 1, q.g - 1, q.gl - 1, q.k, (1u << q.z) - 1u,
              tau >= 32 ? 0xFFFFFFFFu : ((1u << tau) - 1u), rho_g_of(q.g), q.theta};
  for (int x = 0; x < SRLA_N_HASH; x++) {
    h.coef.a[x] = q.hash_a[x];
    h.coef.b[x] = q.hash_b[x];
  }
  h.k_is_P = (q.k == h.geo.P);
  h.T = q.start_slice;
  SRLA_TRY(cudaDeviceGetAttribute(&h.sms, cudaDevAttrMultiProcessorCount, dev));
  if ((r = occupancy(&h)) != SRLA_OK) return r;

  // The array keeps the previous call's contents: the recorders, the sets and the control
  // block must start at zero, so the whole used part is cleared first.
  SRLA_TRY(cudaMemsetAsync(h.ws, 0, L.total, h.st));
  if ((r = clear_pairs(&h)) != SRLA_OK) return r;
  Ctl c{};
  c.T = h.T;
  c.tm = (uint32_t)(h.T % h.geo.P);
  c.w_star = h.geo.gl + 1;
  c.pair_mode = 1;
  SRLA_TRY(cudaMemcpyAsync(h.ctl(), &c, sizeof(Ctl), cudaMemcpyHostToDevice, h.st));
  r = with_cells(q.dr_bytes, [&](auto c) { return static_batch<decltype(c)>(&h, d_pairs, n_pairs); });
  if (r != SRLA_OK) return r;

  const int par = (int)(h.T & 1);
  srla_slice_stats st;
  SRLA_TRY(cudaMemcpyAsync(&st, h.ws + L.rep_stats[par], sizeof(st), cudaMemcpyDeviceToHost, h.st));
  SRLA_TRY(cudaStreamSynchronize(h.st));
  st.n_pkts = n_pairs;
  const size_t n = st.n_candidates;
  if (n_out) *n_out = n;
  if (stats) *stats = st;
  const size_t take = std::min(n, cap);
  if (take) {
    SRLA_TRY(cudaMemcpyAsync(out, h.ws + L.rep_entries[par], take * sizeof(srla_entry), cudaMemcpyDeviceToHost,
                             h.st));
    SRLA_TRY(cudaStreamSynchronize(h.st));
  }
  if (st.overflow & 4u) return SRLA_E_TIMEOUT;
  if (st.overflow) return SRLA_E_CAPACITY;
  if (cap < n) return SRLA_E_NOMEM;
  return SRLA_OK;
}

extern "C" int srla_wait_selftest(void* dev_scratch, size_t bytes, void* stream, uint32_t blocks, uint32_t absent,
                                  uint32_t spin_limit) {
  if (!dev_scratch || bytes < 256 || (reinterpret_cast<uintptr_t>(dev_scratch) & 15u) || blocks < 2 || blocks > 64 ||
      absent >= blocks)
    return SRLA_E_INVAL;
  static_assert(sizeof(Ctl) <= 256, "control block fits the self-test scratch");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Ctl* ctl = static_cast<Ctl*>(dev_scratch);
  SRLA_TRY(cudaMemsetAsync(ctl, 0, sizeof(Ctl), st));
  k_wait_selftest<<<blocks, 32, 0, st>>>(ctl, absent, spin_limit);
  SRLA_TRY(cudaGetLastError());
  unsigned overflow = 0;
  SRLA_TRY(cudaMemcpyAsync(&overflow, &ctl->overflow, sizeof(overflow), cudaMemcpyDeviceToHost, st));
  SRLA_TRY(cudaStreamSynchronize(st));
  return (overflow & 4u) ? SRLA_E_TIMEOUT : SRLA_OK;
}

template <typename CellT>
static void launch_probe(uint32_t policy, int grid, cudaStream_t st, void* buf, uint64_t cells, uint64_t n,
                         uint64_t seed) {
  CellT* b = static_cast<CellT*>(buf);
  if constexpr (sizeof(CellT) == 8) {
    if (policy == kProbeCas)
      k_scatter_probe<CellT, kProbeCas><<<grid, 256, 0, st>>>(b, cells, n, seed);
    else
      k_scatter_probe<CellT, kProbeLoad><<<grid, 256, 0, st>>>(b, cells, n, seed);
  } else {
    if (policy == kProbeStore)
      k_scatter_probe<CellT, kProbeStore><<<grid, 256, 0, st>>>(b, cells, n, seed);
    else if (policy == kProbeAtomicMax)
      k_scatter_probe<CellT, kProbeAtomicMax><<<grid, 256, 0, st>>>(b, cells, n, seed);
    else if (policy == kProbeReadFirst)
      k_scatter_probe<CellT, kProbeReadFirst><<<grid, 256, 0, st>>>(b, cells, n, seed);
    else
      k_scatter_probe<CellT, kProbeLoad><<<grid, 256, 0, st>>>(b, cells, n, seed);
  }
}

extern "C" int srla_scatter_probe(void* dev_buf, size_t bytes, uint32_t cell_bytes, uint64_t n_stores, uint64_t seed,
                                  uint32_t policy, void* stream) {
  if (!dev_buf || policy > kProbeLoad) return SRLA_E_INVAL;
  // 1-, 2- and 4-byte cells for stores, maxima and read-first writes; 8-byte slots for the
  // compare-and-swap; any of them for loads
  const bool cell_ok = policy == kProbeCas    ? cell_bytes == 8
                       : policy == kProbeLoad ? (cell_bytes == 1 || cell_bytes == 2 || cell_bytes == 4 || cell_bytes == 8)
                                              : (cell_bytes == 1 || cell_bytes == 2 || cell_bytes == 4);
  if (!cell_ok) return SRLA_E_INVAL;
  if (reinterpret_cast<uintptr_t>(dev_buf) & (cell_bytes == 8 ? 7u : 3u)) return SRLA_E_INVAL;  // word-aligned
  // the CAS loop of the atomic maximum reads and writes whole 32-bit words: only cells of
  // whole words of the buffer are used
  const uint64_t cells = (policy == kProbeAtomicMax ? bytes & ~(size_t)3 : bytes) / cell_bytes;
  if (!cells) return SRLA_E_INVAL;
  int dev = 0, sms = 0;
  SRLA_TRY(cudaGetDevice(&dev));
  SRLA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int grid = grid_for(n_stores, 256, sms * 8);
  if (cell_bytes == 1)
    launch_probe<uint8_t>(policy, grid, st, dev_buf, cells, n_stores, seed);
  else if (cell_bytes == 2)
    launch_probe<uint16_t>(policy, grid, st, dev_buf, cells, n_stores, seed);
  else if (cell_bytes == 4)
    launch_probe<uint32_t>(policy, grid, st, dev_buf, cells, n_stores, seed);
  else
    launch_probe<unsigned long long>(policy, grid, st, dev_buf, cells, n_stores, seed);
  return cuda_err(cudaGetLastError());
}
