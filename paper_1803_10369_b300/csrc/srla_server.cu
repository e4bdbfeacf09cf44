// libsrla serving: a request loop over one link group (declared in include/srla.h).
//
// Clients open, close and feed links from any host thread; their requests queue under one
// mutex.  The tick thread's srla_server_tick takes the queues, retires departed links, admits waiting
// links in arrival order while the byte budget and the group's arena and slots allow, pushes
// the batches of admitted links, and closes the slice of all of them with one graph launch.
// Only the tick thread touches the group, so the GPU work of every admitted link runs in
// the same launches while new requests keep arriving.
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "srla.h"

namespace {

struct Open {
  uint64_t key;
  srla_params p;
  uint64_t bytes;
};

struct Batch {
  uint64_t key;
  const uint32_t* pairs;
  uint64_t n;
  int on_device;
};

struct Member {
  uint64_t key;
  uint32_t link;
};

}  // namespace

struct srla_server_s {
  srla_group_t* g = nullptr;
  srla_server_config cfg{};
  std::mutex mu;  // guards the request queues and the key tables below
  std::deque<Open> waiting;
  std::vector<uint64_t> closes;
  std::vector<Batch> batches;
  std::unordered_map<uint64_t, uint32_t> link_of;  // admitted key -> group link
  std::unordered_map<uint64_t, uint64_t> bytes_of;  // admitted key -> arena bytes
  uint64_t used = 0;
  std::vector<Member> members[2];  // links of the two most recent slices, by parity
  uint64_t slice_of[2] = {~0ull, ~0ull};
  int tune_reps = 0;               // autotune the scan at the next tick
  std::vector<srla_entry> all;     // scratch for report_all
  std::vector<uint32_t> offs;
  std::vector<srla_slice_stats> stats;
};

extern "C" {

size_t srla_server_workspace_bytes(const srla_server_config* c, uint64_t arena_bytes) {
  if (!c) return 0;
  const size_t f = srla_group_fixed_bytes(c->max_links, c->max_pkts, c->max_host_pkts, c->max_report);
  return f ? f + arena_bytes : 0;
}

int srla_server_create(const srla_server_config* c, void* dev_workspace, size_t ws_bytes, void* stream,
                       srla_server_t** out) {
  if (!c || !out) return SRLA_E_INVAL;
  *out = nullptr;
  srla_server_t* s = new (std::nothrow) srla_server_s();
  if (!s) return SRLA_E_NOMEM;
  s->cfg = *c;
  const int r =
      srla_group_create(c->max_links, c->max_pkts, c->max_host_pkts, c->max_report, dev_workspace, ws_bytes, stream, &s->g);
  if (r != SRLA_OK) {
    delete s;
    return r;
  }
  s->all.resize(c->max_report);
  s->offs.resize((size_t)c->max_links + 1);
  s->stats.resize(c->max_links);
  *out = s;
  return SRLA_OK;
}

int srla_server_open(srla_server_t* s, uint64_t key, const srla_params* p) {
  if (!s || !p) return SRLA_E_INVAL;
  const uint64_t bytes = srla_group_link_bytes(p);
  if (bytes == 0) return SRLA_E_INVAL;
  if (bytes > s->cfg.budget_bytes) return SRLA_E_NOMEM;
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->link_of.count(key)) return SRLA_E_INVAL;
  for (const Open& o : s->waiting)
    if (o.key == key) return SRLA_E_INVAL;
  s->waiting.push_back(Open{key, *p, bytes});
  return SRLA_OK;
}

int srla_server_close(srla_server_t* s, uint64_t key) {
  if (!s) return SRLA_E_INVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  for (auto it = s->waiting.begin(); it != s->waiting.end(); ++it)
    if (it->key == key) {
      s->waiting.erase(it);
      return SRLA_OK;
    }
  if (!s->link_of.count(key)) return SRLA_E_INVAL;
  s->closes.push_back(key);
  return SRLA_OK;
}

int srla_server_submit(srla_server_t* s, uint64_t key, const uint32_t* pairs, uint64_t n_pairs, int on_device) {
  if (!s || (!pairs && n_pairs)) return SRLA_E_INVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if (!s->link_of.count(key)) return SRLA_E_ORDER;
  if (n_pairs) s->batches.push_back(Batch{key, pairs, n_pairs, on_device});
  return SRLA_OK;
}

int srla_server_submit_many(srla_server_t* s, uint32_t n, const uint64_t* keys, const uint32_t* const* pairs,
                            const uint64_t* n_pairs, int on_device, uint32_t* taken) {
  if (!s || (n && (!keys || !pairs || !n_pairs))) return SRLA_E_INVAL;
  uint32_t k = 0;
  std::lock_guard<std::mutex> lock(s->mu);
  for (uint32_t i = 0; i < n; i++) {
    if (!pairs[i] && n_pairs[i]) return SRLA_E_INVAL;
    if (!s->link_of.count(keys[i])) continue;
    if (n_pairs[i]) s->batches.push_back(Batch{keys[i], pairs[i], n_pairs[i], on_device});
    k++;
  }
  if (taken) *taken = k;
  return SRLA_OK;
}

int srla_server_autotune(srla_server_t* s, int reps) {
  if (!s || reps < 1) return SRLA_E_INVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  s->tune_reps = reps;
  return SRLA_OK;
}

int srla_server_tick(srla_server_t* s, uint64_t* slice, uint32_t* admitted, uint32_t* waiting) {
  if (!s) return SRLA_E_INVAL;
  std::vector<uint64_t> closes;
  std::vector<Batch> batches;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    closes.swap(s->closes);
    batches.swap(s->batches);
  }
  int r = SRLA_OK;
  // departures first: their memory and slots serve the waiting links
  for (uint64_t key : closes) {
    uint32_t link;
    uint64_t bytes;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      auto it = s->link_of.find(key);
      if (it == s->link_of.end()) continue;
      link = it->second;
      bytes = s->bytes_of[key];
      s->link_of.erase(it);
      s->bytes_of.erase(key);
    }
    if ((r = srla_group_detach(s->g, link)) != SRLA_OK) return r;
    s->used -= bytes;
  }
  // admissions in arrival order while the budget, the arena and the slots allow
  for (;;) {
    Open o;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      if (s->waiting.empty() || s->used + s->waiting.front().bytes > s->cfg.budget_bytes) break;
      o = s->waiting.front();
    }
    uint32_t link;
    r = srla_group_attach(s->g, &o.p, &link);
    if (r == SRLA_E_NOMEM || r == SRLA_E_CAPACITY) break;  // waits for more departures
    if (r != SRLA_OK) return r;
    std::lock_guard<std::mutex> lock(s->mu);
    s->waiting.pop_front();
    s->link_of[o.key] = link;
    s->bytes_of[o.key] = o.bytes;
    s->used += o.bytes;
  }
  // the batches of links that are (still) admitted
  for (const Batch& b : batches) {
    uint32_t link;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      auto it = s->link_of.find(b.key);
      if (it == s->link_of.end()) continue;  // the link departed before its batch was pushed
      link = it->second;
    }
    if ((r = srla_group_push(s->g, link, b.pairs, b.n, b.on_device)) != SRLA_OK) return r;
  }
  int reps = 0;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    reps = s->tune_reps;
    s->tune_reps = 0;
  }
  if (reps && !batches.empty()) {
    r = srla_group_autotune(s->g, reps, nullptr, nullptr);
    if (r != SRLA_OK) return r;
  }
  uint64_t gs = 0;
  if ((r = srla_group_end_slice(s->g, &gs)) != SRLA_OK) return r;
  const int q = (int)(gs & 1);
  std::lock_guard<std::mutex> lock(s->mu);
  s->members[q].clear();
  for (const auto& kv : s->link_of) s->members[q].push_back(Member{kv.first, kv.second});
  s->slice_of[q] = gs;
  if (slice) *slice = gs;
  if (admitted) *admitted = (uint32_t)s->link_of.size();
  if (waiting) *waiting = (uint32_t)s->waiting.size();
  return SRLA_OK;
}

int srla_server_poll(srla_server_t* s, uint64_t slice, srla_server_result* results, size_t result_cap,
                     size_t* n_results, srla_entry* entries, size_t entry_cap, size_t* n_entries) {
  if (!s || (result_cap && !results) || (entry_cap && !entries)) return SRLA_E_INVAL;
  const int q = (int)(slice & 1);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->slice_of[q] != slice) return SRLA_E_ORDER;
  }
  size_t n = 0;
  const int rc = srla_group_report_all(s->g, slice, s->all.data(), s->all.size(), &n, s->offs.data(), s->stats.data());
  if (rc != SRLA_OK && rc != SRLA_E_CAPACITY) return rc;
  std::vector<Member> mem;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    mem = s->members[q];
  }
  size_t nr = 0, ne = 0;
  int out_rc = rc;
  for (const Member& m : mem) {
    const uint32_t a = s->offs[m.link], b = s->offs[m.link + 1];
    if (nr < result_cap) {
      srla_server_result& res = results[nr];
      res.key = m.key;
      res.first = (uint32_t)ne;
      res.count = b - a;
      res.stats = s->stats[m.link];
      if (ne + (b - a) <= entry_cap)
        std::memcpy(entries + ne, s->all.data() + a, (size_t)(b - a) * sizeof(srla_entry));
      else
        out_rc = out_rc == SRLA_OK ? SRLA_E_NOMEM : out_rc;
    } else {
      out_rc = out_rc == SRLA_OK ? SRLA_E_NOMEM : out_rc;
    }
    nr++;
    ne += b - a;
  }
  if (n_results) *n_results = nr;
  if (n_entries) *n_entries = ne;
  return out_rc;
}

uint64_t srla_server_used_bytes(const srla_server_t* s) { return s ? s->used : 0; }

// The state of an admitted link between ticks (tick thread): the group link's export.
static int server_link(srla_server_t* s, uint64_t key, uint32_t* link) {
  std::lock_guard<std::mutex> lock(s->mu);
  const auto it = s->link_of.find(key);
  if (it == s->link_of.end()) return SRLA_E_ORDER;
  *link = it->second;
  return SRLA_OK;
}

size_t srla_server_state_bytes(srla_server_t* s, uint64_t key) {
  uint32_t link = 0;
  if (!s || server_link(s, key, &link) != SRLA_OK) return 0;
  return srla_group_state_bytes(s->g, link);
}

int srla_server_export_state(srla_server_t* s, uint64_t key, void* host_buf, size_t cap) {
  if (!s || !host_buf) return SRLA_E_INVAL;
  uint32_t link = 0;
  const int r = server_link(s, key, &link);
  return r != SRLA_OK ? r : srla_group_export_state(s->g, link, host_buf, cap);
}

void srla_server_destroy(srla_server_t* s) {
  if (!s) return;
  srla_group_destroy(s->g);
  delete s;
}

}  // extern "C"
