// libsrla groups: many links advanced together, one CUDA graph launch per slice
// (declared in include/srla.h).  Host code lays out the caller's workspace, carves link
// regions out of its arena, keeps the device link table and work lists current, builds the
// per-slice task table, and replays one captured graph per slice parity.
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <new>
#include <vector>

#include "group.cuh"
#include "host_layout.h"

using namespace srla;
using namespace srla::host;

namespace {

constexpr uint64_t kChunkVecs = 1ull << 14;  // 256 KB of recorders per sweep chunk
constexpr int kGroupScanThreads = 256;       // default scan block size (the tuner may change it)

int gerr(cudaError_t e) {
  if (e == cudaSuccess) return SRLA_OK;
  (void)cudaGetLastError();
  return SRLA_E_CUDA;
}

#define G_TRY(x)                   \
  do {                             \
    const int _r = gerr(x);        \
    if (_r != SRLA_OK) return _r;  \
  } while (0)

constexpr uint32_t kMinTaskPkts = 1u << 14;  // the smallest task size the tuner tries

uint64_t max_tasks_for(uint32_t max_links, uint64_t max_pkts) {
  // every push may leave one partial task behind
  return max_pkts / kMinTaskPkts + 8ull * max_links + 64;
}

// Recorders decoded per step of a state export (through the fixed part's export area).
constexpr size_t kExportChunk = (size_t)1 << 21;

struct Fixed {
  size_t gctl, descs, tasks, filt_off, gstats[2], rep_off[2], grep[2], stage[2], xstage, total;
  uint64_t max_tasks;
};

Fixed fixed_layout(uint32_t max_links, uint64_t max_pkts, uint64_t max_host_pkts, uint32_t max_report) {
  Fixed F{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  F.max_tasks = max_tasks_for(max_links, max_pkts);
  F.gctl = take(sizeof(GroupCtl));
  F.descs = take(sizeof(LinkDesc) * max_links);
  F.tasks = take(sizeof(TaskHeader) + sizeof(ScanTask) * F.max_tasks);
  F.filt_off = take(sizeof(uint32_t) * (max_links + 1));
  for (int q = 0; q < 2; q++) {
    F.gstats[q] = take(sizeof(srla_slice_stats) * max_links);
    F.rep_off[q] = take(sizeof(uint32_t) * (max_links + 1));
    F.grep[q] = take(sizeof(srla_entry) * (size_t)max_report);
    F.stage[q] = take(8 * (size_t)max_host_pkts);
  }
  F.xstage = take(kExportChunk * sizeof(uint16_t));
  F.total = off;
  return F;
}

srla_params link_params(const srla_params& p) {
  srla_params q = p;
  q.staging_pkts = 4;  // host batches of a group go through the group's staging area
  return q;
}

struct Slot {
  bool active = false;
  srla_params p{};
  Layout L{};
  size_t off = 0, bytes = 0;  // arena region
  uint64_t T = 0;             // open slice of the link
  uint64_t pkts_open = 0;
  uint64_t attached_at = 0;   // first group slice of the link
  uint64_t pkts_slice[2] = {0, 0};
  uint32_t policy = SRLA_SCAN_POLICY_ADAPTIVE_RF;  // aggregation policy of its scan
};

struct Region {
  size_t off, bytes;
};

}  // namespace

struct srla_group_s {
  uint32_t max_links = 0;
  uint64_t max_pkts = 0, max_host_pkts = 0;
  uint32_t max_report = 0;
  Fixed F{};
  char* ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t st = nullptr, st_copy = nullptr, st_side = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr}, ev_fork = nullptr, ev_join = nullptr;
  int sms = 0, sort_grid = 0;
  int filt_grid = 0, est_grid = 0, sweep_grid = 0;  // one wave of resident blocks
  void* h_pinned = nullptr;
  TaskHeader* h_tasks[2] = {nullptr, nullptr};
  srla_slice_stats* h_stats[2] = {nullptr, nullptr};
  uint32_t* h_off[2] = {nullptr, nullptr};
  std::vector<Slot> slots;
  std::vector<Region> free_list;
  size_t chunk_off = 0, chunk_bytes = 0;  // arena region of the sweep work lists
  cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [slice parity][read-first scan]
  uint64_t G = 0;
  bool valid[2] = {false, false};
  uint64_t G_of[2] = {0, 0};
  std::vector<ScanTask> pending;
  uint64_t n_tasks_open = 0;
  uint64_t stage_used = 0;
  bool stage_waited = false;
  uint64_t launches = 0, graph_launches = 0;
  uint64_t scan_builds[2] = {0, 0};  // slice ends that ran the lean / the read-first scan
  // policy of links attached from now on: the one the autotuner chose for the class of
  // links with fewer packets (a new link's rate is not known yet)
  uint32_t new_policy = SRLA_SCAN_POLICY_ADAPTIVE_RF;
  int scan_threads = kGroupScanThreads;  // scan block size: 128, 256 or 512
  uint32_t task_pkts = kTaskPkts;        // packets per scan task
  int scan_grid_of[2][3] = {{0, 0, 0}, {0, 0, 0}};  // resident blocks of each scan build and block size
  int capture_rf = -1;                   // the scan build a capture records (-1: from the policies)
  struct Segment {
    uint32_t link;
    const uint32_t* ptr;
    uint64_t n;
  };
  std::vector<Segment> segments;  // the open slice's batches, before splitting into tasks

  GroupCtl* gctl() const { return reinterpret_cast<GroupCtl*>(ws + F.gctl); }
  LinkDesc* descs() const { return reinterpret_cast<LinkDesc*>(ws + F.descs); }
};

namespace {

// ------------------------------------------------------------------ arena allocator

bool arena_alloc(srla_group_t* g, size_t bytes, size_t* off) {
  bytes = align_up(bytes);
  for (size_t i = 0; i < g->free_list.size(); i++) {
    Region& r = g->free_list[i];
    if (r.bytes >= bytes) {
      *off = r.off;
      r.off += bytes;
      r.bytes -= bytes;
      if (r.bytes == 0) g->free_list.erase(g->free_list.begin() + (long)i);
      return true;
    }
  }
  return false;
}

// The same from the top of the arena: the sweep work lists, rebuilt at every membership
// change, then never leave holes between link regions (which are taken from the bottom).
bool arena_alloc_top(srla_group_t* g, size_t bytes, size_t* off) {
  bytes = align_up(bytes);
  for (size_t i = g->free_list.size(); i-- > 0;) {
    Region& r = g->free_list[i];
    if (r.bytes >= bytes) {
      r.bytes -= bytes;
      *off = r.off + r.bytes;
      if (r.bytes == 0) g->free_list.erase(g->free_list.begin() + (long)i);
      return true;
    }
  }
  return false;
}

void arena_free(srla_group_t* g, size_t off, size_t bytes) {
  bytes = align_up(bytes);
  if (!bytes) return;
  auto it = std::lower_bound(g->free_list.begin(), g->free_list.end(), off,
                             [](const Region& r, size_t o) { return r.off < o; });
  it = g->free_list.insert(it, Region{off, bytes});
  // coalesce with the neighbours
  if (it + 1 != g->free_list.end() && it->off + it->bytes == (it + 1)->off) {
    it->bytes += (it + 1)->bytes;
    g->free_list.erase(it + 1);
  }
  if (it != g->free_list.begin() && (it - 1)->off + (it - 1)->bytes == it->off) {
    (it - 1)->bytes += it->bytes;
    g->free_list.erase(it);
  }
}

// -------------------------------------------------------------- device link table

LinkDesc make_desc(srla_group_t* g, const Slot& s) {
  LinkDesc D{};
  const srla_params& p = s.p;
  const Layout& L = s.L;
  char* base = g->ws + s.off;
  const uint32_t tau = tau_of(p.theta, p.g);
  D.geo = Geo{p.u, p.v, p.g, p.gl, p.v - 1, p.g - 1, p.gl - 1, p.k, (1u << p.z) - 1u,
              tau >= 32 ? 0xFFFFFFFFu : ((1u << tau) - 1u), rho_g_of(p.g), p.theta};
  for (int r = 0; r < SRLA_N_HASH; r++) {
    D.coef.a[r] = p.hash_a[r];
    D.coef.b[r] = p.hash_b[r];
  }
  D.active = 1;
  D.scan_policy = s.policy;
  D.cell_bytes = p.dr_bytes;
  D.k_is_P = p.k == D.geo.P;
  D.umask = L.umask;
  D.umax = p.max_sampled;
  D.cmask = L.cmask;
  D.cmax = p.max_candidates;
  D.ntiles = L.ntiles;
  D.pmask = L.pmask;
  D.ctl = reinterpret_cast<Ctl*>(base + L.ctl);
  D.re = base + L.re;
  D.le = base + L.le;
  D.utab = reinterpret_cast<unsigned long long*>(base + L.utab);
  D.ulist = reinterpret_cast<uint32_t*>(base + L.ulist);
  for (int q = 0; q < 2; q++) {
    D.ctab[q] = reinterpret_cast<unsigned long long*>(base + L.ctab[q]);
    D.cflags[q] = reinterpret_cast<uint32_t*>(base + L.cflags[q]);
    D.clist[q] = reinterpret_cast<uint32_t*>(base + L.clist[q]);
    D.st[q] = reinterpret_cast<srla_slice_stats*>(base + L.rep_stats[q]);
  }
  D.sort_tmp = reinterpret_cast<uint32_t*>(base + L.sort_tmp);
  D.sort_hist = reinterpret_cast<uint32_t*>(base + L.sort_hist);
  D.lut_est = reinterpret_cast<float*>(base + L.lut_est);
  D.lut_flags = reinterpret_cast<uint32_t*>(base + L.lut_flags);
  D.ptab = L.pairs ? reinterpret_cast<unsigned long long*>(base + L.ptab[0]) : nullptr;
  D.le_spv = L.le_spv;
  D.re_spv = L.re_spv;
  D.le_sat = L.le_spv ? reinterpret_cast<uint8_t*>(base + L.le_sat) : nullptr;
  D.re_sat = L.re_spv ? reinterpret_cast<uint8_t*>(base + L.re_sat) : nullptr;
  return D;
}

void add_rows(std::vector<SweepChunk>& out, uint32_t link, uint32_t kind, uint32_t rows, uint64_t vecs_per_row) {
  for (uint32_t r = 0; r < rows; r++)
    for (uint64_t b = 0; b < vecs_per_row; b += kChunkVecs)
      out.push_back(SweepChunk{link, kind, r, 0, b, std::min(kChunkVecs, vecs_per_row - b)});
}

// Rebuild the sweep work lists and the group counters (n_links, n_chunks, n_post) after a
// membership change.  The lists live in the arena; the copies are ordered on the stream
// after every slice end already enqueued, so no running graph sees a half-written list.
int rebuild_work(srla_group_t* g) {
  std::vector<SweepChunk> chunks, post;
  uint32_t n_links = 0;
  for (uint32_t l = 0; l < g->max_links; l++) {
    const Slot& s = g->slots[l];
    if (!s.active) continue;
    n_links = l + 1;
    const srla_params& p = s.p;
    const uint64_t le_vecs = recorder_bytes(&p, (uint64_t)p.v * p.gl) / 16,
                   re_vecs = recorder_bytes(&p, (uint64_t)p.v * p.g) / 16;
    const bool kP = p.k == (1u << p.z) - 1u;
    add_rows(chunks, l, 0, p.u, le_vecs);
    if (!kP) add_rows(chunks, l, 1, p.u, re_vecs);
    if (s.L.pairs) add_rows(chunks, l, 2, 1, ((uint64_t)s.L.pmask + 1) * 8 / 16);
    if (kP) {
      add_rows(post, l, 0, p.u, le_vecs);
      add_rows(post, l, 1, p.u, re_vecs);
    }
  }
  const size_t need = (chunks.size() + post.size()) * sizeof(SweepChunk);
  // the new list is placed before the old one is given back, so that a failure leaves the
  // old list (and the counters that point to it) in place; only when both do not fit at
  // once is the old one freed first (a shrinking list then always fits)
  size_t off = 0;
  if (need && !arena_alloc_top(g, need, &off)) {
    if (!g->chunk_bytes) return SRLA_E_NOMEM;
    for (int q = 0; q < 2; q++) G_TRY(cudaEventSynchronize(g->ev[q]));
    arena_free(g, g->chunk_off, g->chunk_bytes);
    g->chunk_bytes = 0;
    if (!arena_alloc_top(g, need, &off)) {
      const unsigned zero[3] = {0, 0, 0};  // n_links, n_chunks, n_post: no sweep until the next rebuild
      G_TRY(cudaMemcpyAsync(&g->gctl()->n_links, zero, sizeof(zero), cudaMemcpyHostToDevice, g->st));
      return SRLA_E_NOMEM;
    }
  } else if (g->chunk_bytes) {
    arena_free(g, g->chunk_off, g->chunk_bytes);
  }
  g->chunk_off = off;
  g->chunk_bytes = need;
  SweepChunk* dchunks = reinterpret_cast<SweepChunk*>(g->ws + off);
  if (!chunks.empty())
    G_TRY(cudaMemcpyAsync(dchunks, chunks.data(), chunks.size() * sizeof(SweepChunk), cudaMemcpyHostToDevice, g->st));
  if (!post.empty())
    G_TRY(cudaMemcpyAsync(dchunks + chunks.size(), post.data(), post.size() * sizeof(SweepChunk),
                          cudaMemcpyHostToDevice, g->st));
  struct {
    const SweepChunk* chunks;
    const SweepChunk* post;
    unsigned next_task, blocks_done, bar_count, bar_gen, n_links, n_chunks, n_post;
  } head{dchunks, dchunks + chunks.size(), 0, 0, 0, 0, n_links, (unsigned)chunks.size(), (unsigned)post.size()};
  constexpr size_t kHead = offsetof(GroupCtl, n_post) + sizeof(unsigned);  // fields up to n_post
  static_assert(offsetof(decltype(head), n_post) + sizeof(unsigned) == kHead, "GroupCtl head layout");
  G_TRY(cudaMemcpyAsync(g->gctl(), &head, kHead, cudaMemcpyHostToDevice, g->st));
  return cudaStreamSynchronize(g->st) == cudaSuccess ? SRLA_OK : SRLA_E_CUDA;
}

// ------------------------------------------------------------------ the slice end

int scan_grid_index(int threads) { return threads == 128 ? 0 : threads == 256 ? 1 : 2; }

// Whether an attached link's policy may choose the read-first scan (8/16-bit recorders only).
bool any_read_first(const srla_group_t* g) {
  for (const Slot& s : g->slots)
    if (s.active && s.p.dr_bytes &&
        (s.policy == SRLA_SCAN_POLICY_ADAPTIVE_RF || s.policy == SRLA_SCAN_POLICY_OFF_RF))
      return true;
  return false;
}

template <bool kReadFirst>
void launch_group_scan_build(srla_group_t* g, int threads, const TaskHeader* tasks) {
  const int grid = g->scan_grid_of[kReadFirst][scan_grid_index(threads)];
  if (threads == 128)
    kg_scan<128, kReadFirst><<<grid, 128, 0, g->st>>>(g->descs(), tasks, g->gctl());
  else if (threads == 512)
    kg_scan<512, kReadFirst><<<grid, 512, 0, g->st>>>(g->descs(), tasks, g->gctl());
  else
    kg_scan<256, kReadFirst><<<grid, 256, 0, g->st>>>(g->descs(), tasks, g->gctl());
}

// One wave of resident blocks of each block size of a scan build.
template <bool kReadFirst>
cudaError_t scan_occupancy(srla_group_t* g) {
  const int threads[3] = {128, 256, 512};
  const void* fn[3] = {reinterpret_cast<const void*>(kg_scan<128, kReadFirst>),
                       reinterpret_cast<const void*>(kg_scan<256, kReadFirst>),
                       reinterpret_cast<const void*>(kg_scan<512, kReadFirst>)};
  for (int i = 0; i < 3; i++) {
    int occ = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn[i], threads[i], 0);
    if (e != cudaSuccess) return e;
    g->scan_grid_of[kReadFirst][i] = g->sms * std::max(1, occ);
  }
  return cudaSuccess;
}

void launch_group_scan(srla_group_t* g, int threads, const TaskHeader* tasks) {
  const bool rf = g->capture_rf >= 0 ? g->capture_rf != 0 : any_read_first(g);
  if (rf)
    launch_group_scan_build<true>(g, threads, tasks);
  else
    launch_group_scan_build<false>(g, threads, tasks);
}

// Split the open slice's batches into scan tasks of at most task_pkts packets.
int split_tasks(srla_group_t* g) {
  g->pending.clear();
  for (const auto& sg : g->segments)
    for (uint64_t x = 0; x < sg.n; x += g->task_pkts)
      g->pending.push_back(ScanTask{reinterpret_cast<unsigned long long>(sg.ptr + 2 * x),
                                    (uint32_t)std::min<uint64_t>(g->task_pkts, sg.n - x), sg.link});
  if (g->pending.size() > g->F.max_tasks) return SRLA_E_CAPACITY;
  // longest first, so that the persistent scan blocks finish together
  std::stable_sort(g->pending.begin(), g->pending.end(), [](const ScanTask& a, const ScanTask& b) { return a.n > b.n; });
  return SRLA_OK;
}

int enqueue_slice(srla_group_t* g, int q) {
  const Fixed& F = g->F;
  LinkDesc* descs = g->descs();
  GroupCtl* gctl = g->gctl();
  G_TRY(cudaMemcpyAsync(g->ws + F.tasks, g->h_tasks[q], sizeof(TaskHeader) + sizeof(ScanTask) * F.max_tasks,
                        cudaMemcpyHostToDevice, g->st));
  g->launches += 7;  // scan, filter offsets, filter, sort, sweep, lut, estimate, (post sweep below)
  launch_group_scan(g, g->scan_threads, reinterpret_cast<const TaskHeader*>(g->ws + F.tasks));
  // the candidate filter and sort run beside the sweep (they read the SRE only through the
  // window test; the sweep changes only SRE cells outside the window); the Eq. 8/9 tables
  // follow the census
  uint32_t* filt_off = reinterpret_cast<uint32_t*>(g->ws + F.filt_off);
  uint32_t* rep_off = reinterpret_cast<uint32_t*>(g->ws + F.rep_off[q]);
  G_TRY(cudaEventRecord(g->ev_fork, g->st));
  G_TRY(cudaStreamWaitEvent(g->st_side, g->ev_fork, 0));
  kg_filter_offsets<<<1, 32, 0, g->st_side>>>(descs, gctl, filt_off);
  kg_filter<<<g->filt_grid, 256, 0, g->st_side>>>(descs, gctl, filt_off);
  void* args[] = {&descs, &gctl, &rep_off};
  G_TRY(cudaLaunchCooperativeKernel((const void*)kg_sort, dim3(g->sort_grid), dim3(kSortThreads), args,
                                    kSortSmallSmem, g->st_side));
  G_TRY(cudaEventRecord(g->ev_join, g->st_side));
  kg_sweep<<<g->sweep_grid, 256, 0, g->st>>>(descs, gctl, 0);
  kg_lut<<<std::max(1, std::min<int>((int)g->max_links, g->sms * 4)), 256, 0, g->st>>>(descs, gctl);
  G_TRY(cudaStreamWaitEvent(g->st, g->ev_join, 0));
  kg_estimate<<<g->est_grid, 256, 0, g->st>>>(descs, gctl, reinterpret_cast<srla_slice_stats*>(g->ws + F.gstats[q]),
                                             rep_off, reinterpret_cast<srla_entry*>(g->ws + F.grep[q]));
  g->launches += 1;
  kg_sweep<<<g->sweep_grid, 256, 0, g->st>>>(descs, gctl, 1);
  G_TRY(cudaGetLastError());
  G_TRY(cudaMemcpyAsync(g->h_stats[q], g->ws + F.gstats[q], sizeof(srla_slice_stats) * g->max_links,
                        cudaMemcpyDeviceToHost, g->st));
  G_TRY(cudaMemcpyAsync(g->h_off[q], rep_off, sizeof(uint32_t) * (g->max_links + 1), cudaMemcpyDeviceToHost, g->st));
  return SRLA_OK;
}

int capture(srla_group_t* g) {
  cudaStream_t user = g->st;
  g->st = g->st_copy;
  int rc = SRLA_OK;
  for (int x = 0; x < 4 && rc == SRLA_OK; x++) {
    const int q = x & 1, rf = x >> 1;
    cudaGraph_t graph = nullptr;
    const uint64_t before = g->launches;
    if (cudaStreamBeginCapture(g->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = SRLA_E_CUDA;
      break;
    }
    g->capture_rf = rf;
    rc = enqueue_slice(g, q);
    g->capture_rf = -1;
    const cudaError_t e = cudaStreamEndCapture(g->st, &graph);
    if (rc == SRLA_OK && e != cudaSuccess) rc = SRLA_E_CUDA;
    if (rc == SRLA_OK && cudaGraphInstantiate(&g->graph[q][rf], graph, 0) != cudaSuccess) rc = SRLA_E_CUDA;
    if (graph) cudaGraphDestroy(graph);
    g->graph_launches = g->launches - before;
    g->launches = before;
  }
  g->st = user;
  if (rc != SRLA_OK) (void)cudaGetLastError();
  return rc;
}

// Before reusing the parity-q task table and staging half, the slice that used them last
// (two slices ago) must be past its copies.
int wait_parity(srla_group_t* g, int q) {
  if (g->valid[q]) G_TRY(cudaEventSynchronize(g->ev[q]));
  return SRLA_OK;
}

bool slot_was_attached(const srla_group_t* g, uint32_t link, uint64_t gs) {
  const Slot& s = g->slots[link];
  return s.active && s.attached_at <= gs;
}

}  // namespace

extern "C" {

size_t srla_group_fixed_bytes(uint32_t max_links, uint64_t max_pkts, uint64_t max_host_pkts, uint32_t max_report) {
  if (max_links < 1 || max_links > (1u << 16) || max_report < 1) return 0;
  return fixed_layout(max_links, max_pkts, max_host_pkts, max_report).total;
}

size_t srla_group_link_bytes(const srla_params* p) {
  // groups run the order-free candidate rule only (the inline test is a single-link mode)
  if (check(p) != SRLA_OK || p->mode != SRLA_MODE_ORDER_FREE) return 0;
  const srla_params q = link_params(*p);
  return align_up(layout_of(&q, 1).total);
}

int srla_group_create(uint32_t max_links, uint64_t max_pkts, uint64_t max_host_pkts, uint32_t max_report,
                      void* dev_workspace, size_t ws_bytes, void* stream, srla_group_t** out) {
  if (!out) return SRLA_E_INVAL;
  *out = nullptr;
  const size_t fixed = srla_group_fixed_bytes(max_links, max_pkts, max_host_pkts, max_report);
  if (!fixed || !dev_workspace || reinterpret_cast<uintptr_t>(dev_workspace) % kAlign) return SRLA_E_INVAL;
  if (ws_bytes < fixed) return SRLA_E_NOMEM;
  srla_group_t* g = new (std::nothrow) srla_group_s();
  if (!g) return SRLA_E_NOMEM;
  g->max_links = max_links;
  g->max_pkts = max_pkts;
  g->max_host_pkts = max_host_pkts;
  g->max_report = max_report;
  g->F = fixed_layout(max_links, max_pkts, max_host_pkts, max_report);
  g->ws = static_cast<char*>(dev_workspace);
  g->ws_bytes = ws_bytes;
  g->st = static_cast<cudaStream_t>(stream);
  g->slots.resize(max_links);
  g->free_list.push_back(Region{g->F.total, (ws_bytes - g->F.total) & ~(kAlign - 1)});
  int rc = SRLA_OK;
  int dev = 0, occ_sort = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    rc = SRLA_E_CUDA;
  if (rc == SRLA_OK &&
      (cudaStreamCreateWithFlags(&g->st_copy, cudaStreamNonBlocking) != cudaSuccess ||
       cudaStreamCreateWithFlags(&g->st_side, cudaStreamNonBlocking) != cudaSuccess ||
       cudaEventCreateWithFlags(&g->ev[0], cudaEventDisableTiming) != cudaSuccess ||
       cudaEventCreateWithFlags(&g->ev[1], cudaEventDisableTiming) != cudaSuccess ||
       cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
       cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming) != cudaSuccess))
    rc = SRLA_E_CUDA;
  const size_t tbytes = sizeof(TaskHeader) + sizeof(ScanTask) * g->F.max_tasks;
  const size_t sbytes = sizeof(srla_slice_stats) * max_links, obytes = sizeof(uint32_t) * (max_links + 1);
  if (rc == SRLA_OK && cudaHostAlloc(&g->h_pinned, 2 * (tbytes + sbytes + obytes) + 64, cudaHostAllocDefault) != cudaSuccess)
    rc = SRLA_E_NOMEM;
  if (rc == SRLA_OK) {
    char* h = static_cast<char*>(g->h_pinned);
    for (int q = 0; q < 2; q++) {
      g->h_tasks[q] = reinterpret_cast<TaskHeader*>(h);
      h += tbytes;
      g->h_stats[q] = reinterpret_cast<srla_slice_stats*>(h);
      h += sbytes;
      g->h_off[q] = reinterpret_cast<uint32_t*>(h);
      h += obytes;
      std::memset(g->h_tasks[q], 0, tbytes);
    }
    cudaFuncSetAttribute(kg_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSortSmallSmem);
    int o_filt = 0, o_est = 0, o_sweep = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o_filt, kg_filter, 256, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o_est, kg_estimate, 256, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o_sweep, kg_sweep, 256, 0) != cudaSuccess ||
        scan_occupancy<false>(g) != cudaSuccess || scan_occupancy<true>(g) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_sort, kg_sort, kSortThreads, kSortSmallSmem) != cudaSuccess ||
        occ_sort < 1)
      rc = SRLA_E_CUDA;
    g->sort_grid = g->sms * occ_sort;
    g->filt_grid = g->sms * std::max(1, o_filt);
    g->est_grid = g->sms * std::max(1, o_est);
    g->sweep_grid = g->sms * std::max(1, o_sweep);
  }
  if (rc == SRLA_OK) rc = gerr(cudaMemsetAsync(g->ws, 0, g->F.total, g->st));
  if (rc == SRLA_OK) {
    GroupCtl c{};
    c.rep_cap = max_report;
    rc = gerr(cudaMemcpyAsync(g->gctl(), &c, sizeof(c), cudaMemcpyHostToDevice, g->st));
  }
  if (rc == SRLA_OK) rc = rebuild_work(g);
  if (rc == SRLA_OK) rc = capture(g);
  if (rc != SRLA_OK) {
    srla_group_destroy(g);
    return rc;
  }
  *out = g;
  return SRLA_OK;
}

int srla_group_attach(srla_group_t* g, const srla_params* p, uint32_t* link) {
  if (!g || !link || check(p) != SRLA_OK || p->mode != SRLA_MODE_ORDER_FREE) return SRLA_E_INVAL;
  if (!g->segments.empty()) return SRLA_E_ORDER;
  uint32_t l = 0;
  while (l < g->max_links && g->slots[l].active) l++;
  if (l == g->max_links) return SRLA_E_CAPACITY;
  // the slot's previous occupant may still be referenced by an enqueued slice end
  for (int q = 0; q < 2; q++) G_TRY(cudaEventSynchronize(g->ev[q]));
  const srla_params lp = link_params(*p);
  const Layout L = layout_of(&lp, 1);
  size_t off = 0;
  if (!arena_alloc(g, L.total, &off)) return SRLA_E_NOMEM;
  Slot& s = g->slots[l];
  s = Slot{};
  s.policy = g->new_policy;
  s.active = true;
  s.p = lp;
  s.L = L;
  s.off = off;
  s.bytes = L.total;
  s.T = p->start_slice;
  s.attached_at = g->G;
  char* base = g->ws + off;
  G_TRY(cudaMemsetAsync(base, 0, L.total, g->st));
  if (L.pairs) G_TRY(cudaMemsetAsync(base + L.ptab[0], 0xFF, ((size_t)L.pmask + 1) * 8, g->st));
  Ctl c{};
  c.T = s.T;
  c.tm = (uint32_t)(s.T % ((1u << lp.z) - 1u));
  c.w_star = lp.gl + 1;
  c.pair_mode = 1;
  G_TRY(cudaMemcpyAsync(base + L.ctl, &c, sizeof(c), cudaMemcpyHostToDevice, g->st));
  const LinkDesc D = make_desc(g, s);
  G_TRY(cudaMemcpyAsync(g->descs() + l, &D, sizeof(D), cudaMemcpyHostToDevice, g->st));
  const int rc = rebuild_work(g);
  if (rc != SRLA_OK) {  // undo: the slot and its device entry are free again, the old links' lists rebuilt
    s.active = false;
    const LinkDesc none{};
    G_TRY(cudaMemcpyAsync(g->descs() + l, &none, sizeof(none), cudaMemcpyHostToDevice, g->st));
    G_TRY(cudaStreamSynchronize(g->st));
    arena_free(g, off, L.total);
    const int r2 = rebuild_work(g);
    return r2 != SRLA_OK ? r2 : rc;
  }
  *link = l;
  return SRLA_OK;
}

int srla_group_detach(srla_group_t* g, uint32_t link) {
  if (!g || link >= g->max_links || !g->slots[link].active) return SRLA_E_INVAL;
  if (!g->segments.empty()) return SRLA_E_ORDER;
  for (int q = 0; q < 2; q++) G_TRY(cudaEventSynchronize(g->ev[q]));
  Slot& s = g->slots[link];
  s.active = false;
  LinkDesc D{};
  G_TRY(cudaMemcpyAsync(g->descs() + link, &D, sizeof(D), cudaMemcpyHostToDevice, g->st));
  arena_free(g, s.off, s.bytes);
  return rebuild_work(g);
}

int srla_group_push(srla_group_t* g, uint32_t link, const uint32_t* pairs, uint64_t n_pairs, int on_device) {
  if (!g || link >= g->max_links || !g->slots[link].active || (!pairs && n_pairs)) return SRLA_E_INVAL;
  if (n_pairs == 0) return SRLA_OK;
  const int q = (int)(g->G & 1);
  const uint32_t* src = pairs;
  if (!on_device) {
    if (g->stage_used + n_pairs > g->max_host_pkts) return SRLA_E_CAPACITY;
    if (!g->stage_waited) {
      const int r = wait_parity(g, q);
      if (r != SRLA_OK) return r;
      g->stage_waited = true;
    }
    uint32_t* dst = reinterpret_cast<uint32_t*>(g->ws + g->F.stage[q]) + 2 * g->stage_used;
    G_TRY(cudaMemcpyAsync(dst, pairs, n_pairs * 8, cudaMemcpyHostToDevice, g->st));
    src = dst;
    g->stage_used += n_pairs;
  }
  g->n_tasks_open += (n_pairs + g->task_pkts - 1) / g->task_pkts;
  if (g->n_tasks_open > g->F.max_tasks) {
    g->n_tasks_open -= (n_pairs + g->task_pkts - 1) / g->task_pkts;
    return SRLA_E_CAPACITY;
  }
  g->segments.push_back(srla_group_s::Segment{link, src, n_pairs});
  g->slots[link].pkts_open += n_pairs;
  return SRLA_OK;
}

int srla_group_end_slice(srla_group_t* g, uint64_t* group_slice) {
  if (!g) return SRLA_E_INVAL;
  const int q = (int)(g->G & 1);
  int r = wait_parity(g, q);
  if (r != SRLA_OK) return r;
  if ((r = split_tasks(g)) != SRLA_OK) return r;
  g->h_tasks[q]->n_tasks = (unsigned)g->pending.size();
  if (!g->pending.empty())
    std::memcpy(reinterpret_cast<ScanTask*>(g->h_tasks[q] + 1), g->pending.data(), g->pending.size() * sizeof(ScanTask));
  const int rf = any_read_first(g) ? 1 : 0;
  G_TRY(cudaGraphLaunch(g->graph[q][rf], g->st));
  g->scan_builds[rf]++;
  g->launches += g->graph_launches;
  G_TRY(cudaEventRecord(g->ev[q], g->st));
  for (Slot& s : g->slots) {
    if (!s.active) continue;
    s.pkts_slice[q] = s.pkts_open;
    s.pkts_open = 0;
    s.T++;
  }
  g->valid[q] = true;
  g->G_of[q] = g->G;
  if (group_slice) *group_slice = g->G;
  g->G++;
  g->pending.clear();
  g->segments.clear();
  g->n_tasks_open = 0;
  g->stage_used = 0;
  g->stage_waited = false;
  return SRLA_OK;
}

int srla_group_report_all(srla_group_t* g, uint64_t gs, srla_entry* out, size_t cap, size_t* n_out, uint32_t* offsets,
                          srla_slice_stats* stats) {
  if (!g || (cap && !out)) return SRLA_E_INVAL;
  const int q = (int)(gs & 1);
  if (!g->valid[q] || g->G_of[q] != gs) return SRLA_E_ORDER;
  G_TRY(cudaEventSynchronize(g->ev[q]));
  const uint32_t* off = g->h_off[q];
  uint32_t n_links = 0;
  for (uint32_t l = 0; l < g->max_links; l++)
    if (g->slots[l].active) n_links = l + 1;
  const size_t total = std::min<size_t>(off[n_links], g->max_report);
  uint32_t ovf = 0;
  for (uint32_t l = 0; l < g->max_links; l++) {
    const bool live = l < n_links && slot_was_attached(g, l, gs);
    if (offsets) offsets[l] = l < n_links ? std::min<uint32_t>(off[l], (uint32_t)total) : (uint32_t)total;
    if (stats) {
      if (live) {
        stats[l] = g->h_stats[q][l];
        stats[l].n_pkts = g->slots[l].pkts_slice[q];
      } else {
        std::memset(&stats[l], 0, sizeof(srla_slice_stats));
      }
    }
    if (live) ovf |= g->h_stats[q][l].overflow;
  }
  if (offsets) offsets[g->max_links] = (uint32_t)total;
  if (n_out) *n_out = total;
  const size_t take = std::min(total, cap);
  if (take) {
    G_TRY(cudaMemcpyAsync(out, g->ws + g->F.grep[q], take * sizeof(srla_entry), cudaMemcpyDeviceToHost, g->st_copy));
    G_TRY(cudaStreamSynchronize(g->st_copy));
  }
  if (ovf & 4u) return SRLA_E_TIMEOUT;
  if (ovf || off[n_links] > g->max_report) return SRLA_E_CAPACITY;
  if (cap < total) return SRLA_E_NOMEM;
  return SRLA_OK;
}

int srla_group_report(srla_group_t* g, uint32_t link, uint64_t gs, srla_entry* out, size_t cap, size_t* n_out,
                      srla_slice_stats* stats) {
  if (!g || link >= g->max_links || (cap && !out)) return SRLA_E_INVAL;
  const int q = (int)(gs & 1);
  if (!g->valid[q] || g->G_of[q] != gs || !slot_was_attached(g, link, gs)) return SRLA_E_ORDER;
  G_TRY(cudaEventSynchronize(g->ev[q]));
  const uint32_t a = std::min<uint32_t>(g->h_off[q][link], g->max_report);
  const uint32_t b = std::min<uint32_t>(g->h_off[q][link + 1], g->max_report);
  srla_slice_stats st = g->h_stats[q][link];
  st.n_pkts = g->slots[link].pkts_slice[q];
  const size_t n = st.n_candidates;
  if (n_out) *n_out = n;
  if (stats) *stats = st;
  const size_t have = b > a ? b - a : 0;
  const size_t take = std::min(std::min(n, cap), have);
  if (take) {
    G_TRY(cudaMemcpyAsync(out, g->ws + g->F.grep[q] + (size_t)a * sizeof(srla_entry), take * sizeof(srla_entry),
                          cudaMemcpyDeviceToHost, g->st_copy));
    G_TRY(cudaStreamSynchronize(g->st_copy));
  }
  if (st.overflow & 4u) return SRLA_E_TIMEOUT;
  if (st.overflow || have < n) return SRLA_E_CAPACITY;
  if (cap < n) return SRLA_E_NOMEM;
  return SRLA_OK;
}

int srla_group_set_scan_policy(srla_group_t* g, uint32_t link, uint32_t policy) {
  if (!g || link >= g->max_links || !g->slots[link].active || policy > SRLA_SCAN_POLICY_OFF_RF) return SRLA_E_INVAL;
  g->slots[link].policy = policy;
  // stream-ordered after every slice end already enqueued, before the next one
  G_TRY(cudaMemcpyAsync(reinterpret_cast<char*>(g->descs() + link) + offsetof(LinkDesc, scan_policy),
                        &g->slots[link].policy, sizeof(uint32_t), cudaMemcpyHostToDevice, g->st));
  return gerr(cudaStreamSynchronize(g->st));
}

int srla_group_scan_policy(const srla_group_t* g, uint32_t link, uint32_t* policy) {
  if (!g || !policy || link >= g->max_links || !g->slots[link].active) return SRLA_E_INVAL;
  *policy = g->slots[link].policy;
  return SRLA_OK;
}

int srla_group_autotune(srla_group_t* g, int reps, uint32_t* best_threads, uint32_t* best_task_pkts) {
  if (!g || reps < 1) return SRLA_E_INVAL;
  if (g->segments.empty()) return SRLA_E_ORDER;
  const int threads[3] = {128, 256, 512};
  const uint32_t tasks[3] = {1u << 14, 1u << 16, 1u << 18};
  const int q = (int)(g->G & 1);
  int r = wait_parity(g, q);
  if (r != SRLA_OK) return r;
  G_TRY(cudaStreamSynchronize(g->st));
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return SRLA_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return SRLA_E_CUDA;
  }
  // Each trial starts from empty pair tables and a zero task counter; the recorder stores and
  // sampled-host inserts repeat the slice's own, so the state after tuning is unchanged.
  auto trial = [&](int nthreads, float* ms) -> int {
    int rr = split_tasks(g);
    if (rr != SRLA_OK) return rr;
    g->h_tasks[q]->n_tasks = (unsigned)g->pending.size();
    std::memcpy(reinterpret_cast<ScanTask*>(g->h_tasks[q] + 1), g->pending.data(), g->pending.size() * sizeof(ScanTask));
    for (const Slot& s : g->slots)
      if (s.active && s.L.pairs)
        rr = rr ? rr : gerr(cudaMemsetAsync(g->ws + s.off + s.L.ptab[0], 0xFF, ((size_t)s.L.pmask + 1) * 8, g->st));
    rr = rr ? rr : gerr(cudaMemsetAsync(&g->gctl()->next_task, 0, sizeof(unsigned), g->st));
    rr = rr ? rr : gerr(cudaMemcpyAsync(g->ws + g->F.tasks, g->h_tasks[q], sizeof(TaskHeader) + sizeof(ScanTask) * g->pending.size(),
                                        cudaMemcpyHostToDevice, g->st));
    rr = rr ? rr : gerr(cudaEventRecord(e0, g->st));
    if (rr == SRLA_OK) {
      g->launches++;
      launch_group_scan(g, nthreads, reinterpret_cast<const TaskHeader*>(g->ws + g->F.tasks));
    }
    rr = rr ? rr : gerr(cudaEventRecord(e1, g->st));
    rr = rr ? rr : gerr(cudaEventSynchronize(e1));
    if (rr == SRLA_OK && cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) rr = SRLA_E_CUDA;
    return rr;
  };
  auto median = [](std::vector<float>& v) {
    std::sort(v.begin(), v.end());
    return v.empty() ? 1e30f : v[v.size() / 2];
  };
  // 1. launch shape: block size x packets per task
  std::vector<std::vector<float>> ms(9);
  for (int rep = 0; rep < reps && r == SRLA_OK; rep++) {
    for (int c = 0; c < 9 && r == SRLA_OK; c++) {
      g->task_pkts = tasks[c % 3];
      float t = 0;
      if ((r = trial(threads[c / 3], &t)) == SRLA_OK) ms[c].push_back(t);
    }
  }
  int best = 4;  // 256 threads, 64K packets
  float best_ms = 1e30f;
  for (int c = 0; c < 9; c++) {
    const float med = median(ms[c]);
    if (med < best_ms) {
      best_ms = med;
      best = c;
    }
  }
  g->scan_threads = threads[best / 3];
  g->task_pkts = tasks[best % 3];
  // 2. aggregation policy per link class (by packets in the open slice), one class at a time
  constexpr uint64_t kHeavyPkts = 1ull << 18;
  auto set_class = [&](int cls, uint32_t pol) -> int {
    for (uint32_t l = 0; l < g->max_links; l++) {
      Slot& s = g->slots[l];
      if (!s.active || (int)(s.pkts_open >= kHeavyPkts) != cls) continue;
      s.policy = pol;
      G_TRY(cudaMemcpyAsync(reinterpret_cast<char*>(g->descs() + l) + offsetof(LinkDesc, scan_policy), &s.policy,
                            sizeof(uint32_t), cudaMemcpyHostToDevice, g->st));
      G_TRY(cudaStreamSynchronize(g->st));  // the host value is reused before the copy would run
    }
    return SRLA_OK;
  };
  // The search starts from the plain build on every link, so that each class's trials see
  // the lean scan instantiation (one link that may choose the read-first build selects the
  // other for the whole group).
  for (int cls = 0; cls < 2 && r == SRLA_OK; cls++) r = set_class(cls, SRLA_SCAN_POLICY_ADAPTIVE);
  bool light_tuned = false;  // the class of links with fewer packets had links to tune
  for (int cls = 0; cls < 2 && r == SRLA_OK; cls++) {
    bool any = false;
    for (const Slot& s : g->slots) any |= s.active && s.pkts_open && (int)(s.pkts_open >= kHeavyPkts) == cls;
    if (!any) continue;
    std::vector<float> pm[4];
    for (int rep = 0; rep < reps && r == SRLA_OK; rep++) {
      for (uint32_t pol = 0; pol < 4 && r == SRLA_OK; pol++) {
        float t = 0;
        if ((r = set_class(cls, pol)) == SRLA_OK && (r = trial(g->scan_threads, &t)) == SRLA_OK) pm[pol].push_back(t);
      }
    }
    uint32_t best_pol = SRLA_SCAN_POLICY_ADAPTIVE_RF;
    float best_pol_ms = median(pm[best_pol]);
    for (uint32_t pol = 0; pol < 4; pol++) {
      const float med = median(pm[pol]);
      if (med < best_pol_ms) {
        best_pol_ms = med;
        best_pol = pol;
      }
    }
    r = r ? r : set_class(cls, best_pol);
    if (r == SRLA_OK && (cls == 0 || !light_tuned)) g->new_policy = best_pol;
    light_tuned |= cls == 0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the slice end starts from empty pair tables, zero scan counters and a zero task counter,
  // as without tuning
  for (const Slot& s : g->slots) {
    if (!s.active) continue;
    if (s.L.pairs)
      r = r ? r : gerr(cudaMemsetAsync(g->ws + s.off + s.L.ptab[0], 0xFF, ((size_t)s.L.pmask + 1) * 8, g->st));
    char* c = g->ws + s.off + s.L.ctl;
    r = r ? r : gerr(cudaMemsetAsync(c + offsetof(Ctl, n_miss), 0, 2 * sizeof(unsigned), g->st));
    r = r ? r : gerr(cudaMemsetAsync(c + offsetof(Ctl, n_scan), 0, 4 * sizeof(unsigned long long), g->st));
  }
  r = r ? r : gerr(cudaMemsetAsync(&g->gctl()->next_task, 0, sizeof(unsigned), g->st));
  g->pending.clear();
  // the captured slice ends must launch the chosen scan
  for (int x = 0; x < 2; x++) {
    for (cudaGraphExec_t& e : g->graph[x]) {
      if (e) cudaGraphExecDestroy(e);
      e = nullptr;
    }
  }
  r = r ? r : capture(g);
  if (best_threads) *best_threads = (uint32_t)g->scan_threads;
  if (best_task_pkts) *best_task_pkts = g->task_pkts;
  return r;
}

size_t srla_group_state_bytes(const srla_group_t* g, uint32_t link) {
  if (!g || link >= g->max_links || !g->slots[link].active) return 0;
  return state_bytes_of(&g->slots[link].p, g->slots[link].p.max_candidates);
}

int srla_group_export_state(srla_group_t* g, uint32_t link, void* host_buf, size_t cap) {
  if (!g || !host_buf || link >= g->max_links || !g->slots[link].active) return SRLA_E_INVAL;
  if (!g->segments.empty()) return SRLA_E_ORDER;  // only at a slice boundary
  const Slot& s = g->slots[link];
  const srla_params& p = s.p;
  char* base = g->ws + s.off;
  G_TRY(cudaStreamSynchronize(g->st));
  Ctl c;
  G_TRY(cudaMemcpy(&c, base + s.L.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  const uint32_t nc = std::min<uint32_t>(c.cat_count[c.T & 1], p.max_candidates);
  const size_t nre = (size_t)p.u * p.v * p.g, nle = (size_t)p.u * p.v * p.gl;
  if (cap < state_bytes_of(&p, nc)) return SRLA_E_NOMEM;
  StateHeader hd{kStateMagic, kStateVersion, p.u, p.v, p.g, p.gl, p.dr_bytes, p.z, p.k, p.theta, c.T, nc, 0};
  char* b = static_cast<char*>(host_buf);
  std::memcpy(b, &hd, sizeof(hd));
  uint16_t* dst = reinterpret_cast<uint16_t*>(b + sizeof(hd));
  uint16_t* stage = reinterpret_cast<uint16_t*>(g->ws + g->F.xstage);
  const uint32_t P = (1u << p.z) - 1u;
  const Ctl* dctl = reinterpret_cast<const Ctl*>(base + s.L.ctl);
  // SRE then SLE, decoded to the paper's distances one chunk (a multiple of 32 recorders) at a time
  const size_t arr_off[2] = {s.L.re, s.L.le}, arr_n[2] = {nre, nle};
  for (int a = 0; a < 2; a++) {
    for (size_t x = 0; x < arr_n[a]; x += kExportChunk) {
      const size_t m = std::min(kExportChunk, arr_n[a] - x);
      const int grid = (int)std::min<size_t>((m + 255) / 256, (size_t)g->sms * 8);
      g->launches++;
      auto run = [&](auto cell) {
        using CellT = decltype(cell);
        k_decode<CellT><<<grid, 256, 0, g->st>>>(cells_from(reinterpret_cast<CellT*>(base + arr_off[a]), x), stage,
                                                  m, dctl, P);
      };
      if (p.dr_bytes == 1)
        run(uint8_t{});
      else if (p.dr_bytes == 2)
        run(uint16_t{});
      else
        run(Bit{});
      G_TRY(cudaGetLastError());
      G_TRY(cudaMemcpyAsync(dst + x, stage, m * 2, cudaMemcpyDeviceToHost, g->st));
      G_TRY(cudaStreamSynchronize(g->st));
    }
    dst += arr_n[a];
  }
  uint32_t* carry = reinterpret_cast<uint32_t*>(dst);
  if (nc) {
    G_TRY(cudaMemcpy(carry, base + s.L.clist[c.T & 1], (size_t)nc * 4, cudaMemcpyDeviceToHost));
    std::sort(carry, carry + nc);
  }
  return SRLA_OK;
}

int srla_group_sync(srla_group_t* g) {
  if (!g) return SRLA_E_INVAL;
  return gerr(cudaStreamSynchronize(g->st));
}

uint64_t srla_group_kernel_launches(const srla_group_t* g) { return g ? g->launches : 0; }

int srla_group_scan_builds(const srla_group_t* g, uint64_t* lean, uint64_t* read_first) {
  if (!g) return SRLA_E_INVAL;
  if (lean) *lean = g->scan_builds[0];
  if (read_first) *read_first = g->scan_builds[1];
  return SRLA_OK;
}

void srla_group_destroy(srla_group_t* g) {
  if (!g) return;
  if (g->st) cudaStreamSynchronize(g->st);
  for (int q = 0; q < 2; q++) {
    for (cudaGraphExec_t e : g->graph[q])
      if (e) cudaGraphExecDestroy(e);
    if (g->ev[q]) cudaEventDestroy(g->ev[q]);
  }
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  if (g->ev_join) cudaEventDestroy(g->ev_join);
  if (g->st_copy) cudaStreamDestroy(g->st_copy);
  if (g->st_side) cudaStreamDestroy(g->st_side);
  if (g->h_pinned) cudaFreeHost(g->h_pinned);
  delete g;
}

}  // extern "C"
