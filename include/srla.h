/*
 * libsrla -- sliding-window super point cardinality estimation (SRLA, arXiv 1803.10369)
 * on one B300 GPU (sm_103a).  C ABI: plain pointers and sizes, no C++ or torch types.
 *
 * One handle estimates one monitored link (one sliding estimator array, Section 4.1).
 * The caller pushes the link's IP pairs slice by slice and closes every slice; the library
 * answers with the sorted list of candidate super points of the window that ends with that
 * slice, each with its union-SLE weight, its cardinality estimate (Eq. 9) and flags.
 *
 * Conventions for every entry point:
 *   - the return value is 0 on success or a negative SRLA_E_* code; nothing aborts, traps
 *     or throws across the ABI;
 *   - the library never allocates device memory: the caller provides one workspace of
 *     srla_workspace_bytes() bytes (for instance a torch tensor) that holds the sketches,
 *     the per-slice buffers and all scratch space, and keeps it alive until srla_destroy;
 *   - all device work is enqueued on the CUDA stream given to srla_create, in order;
 *   - a handle is used by one host thread at a time.
 */
#ifndef SRLA_H
#define SRLA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SRLA_MAX_ROWS 16            /* u <= 16 */
#define SRLA_N_HASH (SRLA_MAX_ROWS + 3)

/* Error codes. */
#define SRLA_OK 0
#define SRLA_E_INVAL (-1)           /* invalid parameter or argument */
#define SRLA_E_NOMEM (-2)           /* workspace too small, or host memory exhausted */
#define SRLA_E_CAPACITY (-3)        /* a per-slice capacity was exceeded; results incomplete */
#define SRLA_E_CUDA (-4)            /* a CUDA runtime call failed */
#define SRLA_E_ORDER (-5)           /* call out of order (see each entry point) */
#define SRLA_E_TIMEOUT (-6)         /* a bounded device wait gave up; results invalid */

/* Report flags. */
#define SRLA_SUPER 1u               /* estimate >= theta (Definition 2), or saturated */
#define SRLA_SATURATED 2u           /* every union SLE cell in the window: estimate is +inf */
#define SRLA_CARRIED 4u             /* carried from the previous slice end (Algorithm 3) */
#define SRLA_NEW 8u                 /* sampled in this slice and passing the union SRE test */

/* Candidate rules (srla_params.mode). */
#define SRLA_MODE_ORDER_FREE 0u     /* a host sampled in the slice is a new candidate iff its
                                       union SRE passes at the end of the slice; exact,
                                       independent of packet order */
#define SRLA_MODE_INLINE 1u         /* Algorithm 2 as printed: the union SRE test runs at packet
                                       time and the 16 super point indicator bits of Section 4.1
                                       suppress repeats; depends on packet order (parallel
                                       threads race), single links only */

/*
 * Parameters (Sections 3.2, 4.1, 5).  v, g and gl must be powers of two.
 *   u, v        rows and columns of the sliding estimator array (u <= SRLA_MAX_ROWS)
 *   g, gl       distance recorders per SRE and per SLE (the paper's g and g')
 *   dr_bytes    bytes that hold one recorder: 1 or 2; 0 packs one-bit recorders 32 to a word
 *               (then z = 1, so k = 1: the discrete window of Section 3.1; 8x less memory
 *               than 1-byte recorders)
 *   z           recorder bits, 1 <= z <= 8 * dr_bytes (z = 1 when dr_bytes = 0); the largest
 *               distance is 2^z - 1
 *   k           window length in slices, 1 <= k <= 2^z - 1 (Section 3.2)
 *   theta       super point threshold, >= 1 (Definition 2)
 *   start_slice index of the first open slice
 *   staging_pkts  packets the host-input staging area holds (0: 2^20)
 *   max_sampled   distinct hosts sampled into the SRE per slice
 *   max_candidates  candidate list entries per slice (new + carried)
 *   pair_slots_log2 size of the per-slice table of scanned pairs that lets the scan skip a
 *               pair already scanned in the open slice (it writes the same stamps): 0 gives
 *               2^21 slots, -1 disables the table, 10..28 choose 2^value slots (8 bytes each;
 *               a link's workspace holds two such tables, one per slice parity, so that the
 *               next slice's is cleared while the current slice is closed)
 *   mode        SRLA_MODE_ORDER_FREE (0) or SRLA_MODE_INLINE (1).  In the inline mode the SI
 *               bit of a host is bits 28..31 of the sampling-role hash applied to aip, the
 *               SI bits are cleared at each slice end and set again for the carried hosts
 *               (Algorithm 3), pairs are not de-duplicated within the slice (each packet
 *               runs the test), and the slice statistics count no sampled hosts.
 *   hash_a, hash_b  coefficients of the hash family h(x) = (a*x + b) mod (2^61 - 1), one
 *               pair per role: rows 0..u-1 (column of aip in row i), u (SLE cell of bip),
 *               u+1 (SRE cell of bip), u+2 (sampling hash of bip); a in [1, 2^61-2],
 *               b in [0, 2^61-2].  The paper leaves the family open (Section 3.2).
 * Sizes: a row of SRE (v*g recorders) and of SLE (v*gl) recorders takes at least 16 bytes;
 * g*dr_bytes and gl*dr_bytes are at least 4 (g, gl >= 4 for one-bit recorders).
 */
typedef struct srla_params {
  uint32_t u, v, g, gl;
  uint32_t dr_bytes, z, k, theta;
  uint64_t start_slice;
  uint64_t staging_pkts;
  uint32_t max_sampled, max_candidates;
  int32_t pair_slots_log2;
  uint32_t mode;
  uint64_t hash_a[SRLA_N_HASH];
  uint64_t hash_b[SRLA_N_HASH];
} srla_params;

/* One report line: a candidate super point of the window ending with the reported slice. */
typedef struct srla_entry {
  uint32_t aip;    /* the host */
  uint32_t w;      /* |ULE(aip)|^k: union SLE recorders inside the window (Algorithm 1) */
  float est;       /* Eq. 9 estimate of |OP(aip, t, k)|, FP32 (+inf when saturated) */
  uint32_t flags;  /* SRLA_SUPER | SRLA_SATURATED | SRLA_CARRIED | SRLA_NEW */
} srla_entry;

/* Per-slice figures returned with a report. */
typedef struct srla_slice_stats {
  uint64_t slice;            /* index of the reported slice */
  uint64_t n_pkts;           /* packets pushed into it */
  uint32_t n_sampled;        /* distinct hosts with a pair sampled into the SRE */
  uint32_t n_new;            /* of which passed the union SRE test */
  uint32_t n_candidates;     /* report length (new and carried, de-duplicated) */
  uint32_t n_carry_out;      /* hosts carried into the next slice (Algorithm 3) */
  uint32_t w_star;           /* least w whose estimate is >= theta (gl + 1 if none) */
  uint32_t overflow;         /* bit 0: max_sampled exceeded; bit 1: max_candidates exceeded;
                                bit 2: a device-side wait timed out */
  double up;                 /* UP of Eq. 8 */
  uint64_t census[SRLA_MAX_ROWS]; /* |LDR(i)|^k of Section 4.2, per row */
  /* Work of the slice's scan (Algorithm 2), for measurement; these counts depend on thread
   * timing (which of the repeats of a pair are skipped), the results above do not.         */
  uint32_t pair_table;       /* 1: the scans consulted the per-slice table of scanned pairs
                                (when the link has one); 0: it was switched off this slice */
  uint32_t heavy_hosts;      /* 1: the previous slice close saw heavy hosts, which selects the
                                heavy scan build for this slice (groups; single links take it
                                from the newest reported slice, see srla_set_scan_build) */
  uint64_t n_claims;         /* pairs that missed their block's table of recent pairs and
                                claimed a slot of the pair table (one compare-and-swap each) */
  uint64_t n_claim_repeats;  /* of which the pair table had seen already (not scanned again) */
  uint64_t n_scanned;        /* pairs scanned: their u SLE recorders set */
  uint64_t n_scanned_sampled; /* of which sampled: their u SRE recorders set as well */
  uint64_t n_set_probes;     /* insertions tried into the slice's set of sampled hosts (one
                                per distinct host of a warp's sampled pairs) */
  uint64_t n_heavy_events;   /* of which hosts with three or more sampled pairs in one
                                warp's batch of 32 scanned pairs (heavy hosts: the next slice
                                takes the heavy build when they occur in at least 1/8 of the
                                batches) */
} srla_slice_stats;

typedef struct srla_s srla_t;

/* Validate parameters: 0 or SRLA_E_INVAL.  No GPU needed. */
int srla_check_params(const srla_params *p);

/* Workspace bytes needed for p (0 when p is invalid).  No GPU needed. */
size_t srla_workspace_bytes(const srla_params *p);

/* Values derived from p by the paper's formulas (no GPU needed): tau of Eq. 1,
 * ceil(rho*g) with rho = 0.99 (1 - e^{-1/3}) (Section 3.2), and the stamp modulus 2^z - 1. */
int srla_derived(const srla_params *p, uint32_t *tau, uint32_t *rho_g, uint32_t *stamp_mod);

/*
 * Create an estimator on the current CUDA device.
 *   dev_workspace: device pointer, 256-byte aligned, ws_bytes >= srla_workspace_bytes(p);
 *                  owned by the caller, must outlive the handle.
 *   stream: a cudaStream_t (NULL = legacy default stream).
 * All recorders start empty (DRinit, Section 3.2).  Errors: INVAL, NOMEM, CUDA.
 */
int srla_create(const srla_params *p, void *dev_workspace, size_t ws_bytes, void *stream,
                srla_t **out);

/*
 * Scan n_pairs IP pairs into the open slice (Algorithm 2).  pairs holds 2*n_pairs uint32,
 * interleaved aip, bip.  on_device = 1: pairs is device memory, read by kernels on the
 * stream; the caller keeps it unchanged until the stream passes this call (for instance
 * until srla_report or srla_sync returns).  on_device = 0: pairs is host memory (pinned
 * memory gives an asynchronous copy); it is copied through the staging area and must stay
 * unchanged until srla_sync or the next srla_report returns.  n_pairs = 0 is a no-op.
 * Errors: INVAL, CUDA.
 */
int srla_push_packets(srla_t *h, const uint32_t *pairs, uint64_t n_pairs, int on_device);

/*
 * Close the open slice: row census (Section 4.2), Eq. 8, candidate list, Eq. 9 estimates,
 * the slide and carry of Algorithm 3.  Asynchronous; *slice_id receives the closed slice's
 * index and the next slice opens.  Errors: CUDA.
 */
int srla_end_slice(srla_t *h, uint64_t *slice_id);

/*
 * Wait for the report of slice_id and copy it: entries sorted by ascending aip.  The two
 * most recently closed slices can be reported; older ones give SRLA_E_ORDER.  Up to cap
 * entries are written to out (out may be NULL when cap is 0); *n_out receives the full
 * count.  stats may be NULL.  Returns SRLA_E_CAPACITY when a per-slice capacity overflowed
 * (the entries are then those that fit), SRLA_E_NOMEM when cap < *n_out, SRLA_E_TIMEOUT when
 * a bounded device-side wait of the slice end gave up (stats.overflow bit 2).
 */
int srla_report(srla_t *h, uint64_t slice_id, srla_entry *out, size_t cap, size_t *n_out,
                srla_slice_stats *stats);

/* Block until all work enqueued by this handle has finished. */
int srla_sync(srla_t *h);

/*
 * Checkpoint.  The state is the recorder distances (uint16 each, the paper's DR values,
 * 2^z - 1 = empty), the open slice index and the carried host list, in a self-describing
 * host buffer of srla_state_bytes() bytes.  Export and import are only allowed at a slice
 * boundary (no packets pushed into the open slice), else SRLA_E_ORDER.  Import checks that
 * the geometry matches (SRLA_E_INVAL otherwise).
 */
size_t srla_state_bytes(const srla_t *h);
int srla_export_state(srla_t *h, void *host_buf, size_t cap);
int srla_import_state(srla_t *h, const void *host_buf, size_t len);

/* Number of CUDA kernels this handle has launched since srla_create (all entry points). */
uint64_t srla_kernel_launches(const srla_t *h);

/*
 * The scan (Algorithm 2) has three builds that leave the same recorders: the plain build
 * stores every recorder of a scanned pair; the read-first build (8- and 16-bit recorders,
 * order-free rule) reads the recorders first and skips those already holding the open
 * slice's stamp, which pays when most pairs are new; the heavy build (the same recorders,
 * and u*g' <= 4096, u*g <= 2048) is the plain build in which every block keeps a bitmap of
 * the recorders it has stamped for one heavy host (a host filling at least 4 of a warp's 32
 * scanned pairs) and stores each of them once, which pays when one host talks to very many
 * destinations.  SRLA_SCAN_AUTO (the default) takes the newest slice whose report reached
 * the host: the read-first build if its pair table was switched off, else the heavy build if
 * its close saw heavy hosts (slice statistics heavy_hosts / n_heavy_events), else the plain
 * build.  The other values force one build (a tuning and testing aid).  srla_set_scan_build
 * returns SRLA_E_INVAL for an unknown value or a build the link cannot run.
 * srla_scan_builds counts the scan launches of each build since srla_create (any pointer
 * may be NULL).
 */
#define SRLA_SCAN_AUTO 0u
#define SRLA_SCAN_PLAIN 1u
#define SRLA_SCAN_READ_FIRST 2u
#define SRLA_SCAN_HEAVY 3u
int srla_set_scan_build(srla_t *h, uint32_t build);
int srla_scan_builds(const srla_t *h, uint64_t *plain, uint64_t *read_first, uint64_t *heavy);

/* 1 if srla_end_slice replays a CUDA graph captured at srla_create (one per slice parity),
 * 0 if it launches its kernels one by one (capture was not possible on this device). */
int srla_uses_graph(const srla_t *h);

void srla_destroy(srla_t *h);

/*
 * Allocation-free batch report (the paper has no counterpart; this is a service for callers).
 *
 * Some callers cannot allocate device memory: a packet-capture thread with real-time
 * deadlines (cudaMalloc and cudaFree may synchronize the whole device and stall it), or a
 * plugin whose host framework owns all device memory and hands it only fixed input and
 * output buffers.  This entry point needs no workspace and makes no device or host
 * allocation: it runs the scan and the slice end of a fresh estimator over one device batch
 * d_pairs (n_pairs interleaved aip, bip) on `stream`, i.e. the report that srla_create +
 * srla_push_packets + srla_end_slice + srla_report give for a first slice holding exactly
 * this batch, and copies it (sorted by aip) to the host buffer out (cap entries; *n_out =
 * full count; stats may be NULL).  It synchronizes `stream` and returns when the report is
 * on the host; while `stream` is being captured it returns SRLA_E_INVAL before any other
 * CUDA call, leaving the capture intact.
 *
 * Scratch: a fixed array of SRLA_STATIC_SCRATCH_BYTES compiled into the library, present on
 * every GPU that loads the library until the process exits.  Parameters whose one-slice
 * layout (the workspace layout with one pair table and no host staging, a little less than
 * srla_workspace_bytes) exceeds it are rejected with SRLA_E_NOMEM before any GPU work.  The first call on a device looks up the array's device
 * address (and sets a kernel attribute) for that device; make that first call before any
 * stream capture.  Every call clears and reuses the same array, so calls that overlap on the
 * GPU (other streams, other host threads) race and corrupt each other: serialize them.
 * Errors: INVAL, NOMEM, CAPACITY (as srla_report), CUDA.
 */
#define SRLA_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
int srla_batch_report_static(const srla_params *p, const uint32_t *d_pairs, uint64_t n_pairs,
                             void *stream, srla_entry *out, size_t cap, size_t *n_out,
                             srla_slice_stats *stats);

/* Self-test of the bounded device waits (the grid barrier of the cooperative candidate
 * sort; the group sort uses the same pattern).  Launches `blocks` (2..64) blocks on `stream`
 * that meet at one barrier, of which the last `absent` (< blocks) never arrive; the others
 * poll at most spin_limit times (each poll sleeps about 64 ns), then give up and flag the
 * timeout.  dev_scratch: caller-owned device memory of at least 256 bytes, 16-byte aligned
 * (cleared and used as a control block).  Returns SRLA_E_TIMEOUT when the wait gave up,
 * SRLA_OK when every block arrived; the CUDA context stays usable either way (no trap, no
 * fault).  Errors: INVAL, CUDA. */
int srla_wait_selftest(void *dev_scratch, size_t bytes, void *stream, uint32_t blocks, uint32_t absent,
                       uint32_t spin_limit);

/* Store roofline probe (a measurement aid, not part of the method): enqueues on `stream`
 * n_stores accesses of cell_bytes each to pseudo-random cells of the caller's device buffer
 * dev_buf of `bytes` bytes (at least one cell, aligned to 4 bytes, to 8 for 8-byte cells):
 * the access shape of the scan's recorder updates (Algorithm 2) without their hashing,
 * de-duplication or sampling.  All writes carry the same value, as all writers of a slice
 * write the same stamp.  policy: how an access is made,
 *   SRLA_PROBE_STORE       a plain store (the scan's choice; cell_bytes 1, 2 or 4);
 *   SRLA_PROBE_ATOMIC_MAX  an atomic maximum (native on 4-byte cells; on 1- and 2-byte
 *                          cells a compare-and-swap loop on the enclosing 32-bit word,
 *                          at most 64 tries; only the cells of whole words of the buffer
 *                          are used);
 *   SRLA_PROBE_READ_FIRST  a load through L2, then a store only if the cell differs;
 *   SRLA_PROBE_CAS         a 64-bit compare-and-swap from the all-ones key (cell_bytes 8):
 *                          the scan's claims in its table of scanned pairs;
 *   SRLA_PROBE_LOAD        a plain load through L2 (cell_bytes 1, 2, 4 or 8): the scan's
 *                          probes of its sampled-host set.
 * Time it with events on the same stream.  Overwrites the buffer.  Errors: INVAL, CUDA. */
#define SRLA_PROBE_STORE 0u
#define SRLA_PROBE_ATOMIC_MAX 1u
#define SRLA_PROBE_READ_FIRST 2u
#define SRLA_PROBE_CAS 3u
#define SRLA_PROBE_LOAD 4u
int srla_scatter_probe(void *dev_buf, size_t bytes, uint32_t cell_bytes, uint64_t n_stores, uint64_t seed,
                       uint32_t policy, void *stream);
const char *srla_strerror(int code);


/* ======================================================================================
 * Groups: many monitored links advanced together (one CUDA graph launch per slice).
 *
 * Each link is an independent estimator array (one per edge router, Section 3.1) with its
 * own parameters, window and slice index.  A group owns one caller-provided workspace: a
 * fixed part (link table, task table, report buffer, staging) and an arena from which link
 * regions are carved when links attach.  Between two slice ends the caller pushes packets of
 * any attached link; srla_group_end_slice then scans all of them and closes the slice of
 * every attached link with one graph launch (kernels over all links, not one launch per
 * link).  Attach and detach are allowed at slice boundaries (no packets pushed yet), which
 * is how a serving loop admits and retires links while others keep running.
 * ====================================================================================== */
typedef struct srla_group_s srla_group_t;

/* Fixed workspace part of a group (0 on invalid arguments).  The arena for links is the
 * rest of the workspace given to srla_group_create.
 *   max_links        link slots
 *   max_pkts         packets per slice over all links (device and host batches)
 *   max_host_pkts    packets per slice pushed from host memory (staged, double-buffered)
 *   max_report       report entries per slice over all links                                */
size_t srla_group_fixed_bytes(uint32_t max_links, uint64_t max_pkts, uint64_t max_host_pkts,
                              uint32_t max_report);

/* Arena bytes one link with parameters p occupies (0 if p is invalid); for admission.    */
size_t srla_group_link_bytes(const srla_params *p);

int srla_group_create(uint32_t max_links, uint64_t max_pkts, uint64_t max_host_pkts,
                      uint32_t max_report, void *dev_workspace, size_t ws_bytes, void *stream,
                      srla_group_t **out);

/* Attach a link (fresh, empty recorders, slice index p->start_slice); *link receives its
 * slot.  SRLA_E_NOMEM when the arena has no room, SRLA_E_CAPACITY when all slots are used,
 * SRLA_E_ORDER when packets were already pushed in the open slice.                        */
int srla_group_attach(srla_group_t *g, const srla_params *p, uint32_t *link);
/* Detach a link; its arena region is reused by later attaches.  Reports of its past slices
 * are no longer available.  SRLA_E_ORDER when packets were already pushed in the slice.  */
int srla_group_detach(srla_group_t *g, uint32_t link);

/* Packets of one link for the open slice (as srla_push_packets).  Device batches must stay
 * unchanged until the slice end's work completes (srla_group_report / srla_group_sync).  */
int srla_group_push(srla_group_t *g, uint32_t link, const uint32_t *pairs, uint64_t n_pairs,
                    int on_device);

/* Scan and close the open slice of every attached link; *group_slice receives the group
 * slice counter (0, 1, 2, ...).                                                          */
int srla_group_end_slice(srla_group_t *g, uint64_t *group_slice);

/* All reports of a group slice (one of the two most recent ones): the entries of every link
 * that was attached at that slice, concatenated in slot order, each link's sorted by aip.
 * offsets[l] .. offsets[l+1] are link l's entries (max_links + 1 values); stats[l] its
 * statistics (zeroed for free slots); either may be NULL.  Returns like srla_report.     */
int srla_group_report_all(srla_group_t *g, uint64_t group_slice, srla_entry *out, size_t cap,
                          size_t *n_out, uint32_t *offsets, srla_slice_stats *stats);
/* One link's report of a group slice.                                                   */
int srla_group_report(srla_group_t *g, uint32_t link, uint64_t group_slice, srla_entry *out,
                      size_t cap, size_t *n_out, srla_slice_stats *stats);

/* Aggregation policy of a link's scan (the pair table of scanned pairs and the scan build):
 *   SRLA_SCAN_POLICY_ADAPTIVE     pair table switched per slice by the previous slice close
 *                                 (off while fewer than a quarter of its claims find repeats),
 *                                 plain build;
 *   SRLA_SCAN_POLICY_ADAPTIVE_RF  the same table rule, and the read-first build (8/16-bit
 *                                 recorders) in the slices where the table is off (default);
 *   SRLA_SCAN_POLICY_OFF          no pair table, plain build;
 *   SRLA_SCAN_POLICY_OFF_RF       no pair table, read-first build (8/16-bit recorders).
 * All four leave the same recorders; they differ in speed only.  srla_group_set_scan_policy
 * takes effect from the next scan; INVAL for a free slot or an unknown policy.            */
#define SRLA_SCAN_POLICY_ADAPTIVE 0u
#define SRLA_SCAN_POLICY_ADAPTIVE_RF 1u
#define SRLA_SCAN_POLICY_OFF 2u
#define SRLA_SCAN_POLICY_OFF_RF 3u
int srla_group_set_scan_policy(srla_group_t *g, uint32_t link, uint32_t policy);
int srla_group_scan_policy(const srla_group_t *g, uint32_t link, uint32_t *policy);

/* The group scan is compiled twice: a lean kernel, and one that adds the read-first build
 * (it needs more registers).  A slice end runs the second when some attached link's policy
 * may choose the read-first build (SRLA_SCAN_POLICY_ADAPTIVE_RF or _OFF_RF on 8/16-bit
 * recorders), else the first.  srla_group_scan_builds counts the slice ends that ran each
 * since srla_group_create (either pointer may be NULL); INVAL for g = NULL.               */
int srla_group_scan_builds(const srla_group_t *g, uint64_t *lean, uint64_t *read_first);

/* Scan autotuner: with the open slice's packets pushed, time the group scan with block sizes
 * 128/256/512 and tasks of 2^14/2^16/2^18 packets (reps runs each, on empty pair tables) and
 * keep the fastest (median); then, starting from SRLA_SCAN_POLICY_ADAPTIVE on every link,
 * per link class (links with fewer than 2^18 packets in the open slice, then links with more)
 * time the four aggregation policies above for that class's links and keep the fastest.  The choices hold for all later slices (srla_group_scan_policy
 * reads a link's); the slice's results are unchanged (the trial scans repeat the slice's own
 * idempotent recorder stores and set insertions).  Links attached after the tuning start on
 * the policy chosen for the class of links with fewer packets (or, when that class had no
 * links, for the other); before any tuning, on SRLA_SCAN_POLICY_ADAPTIVE_RF.  Errors: ORDER
 * when nothing was pushed, CUDA.                                                         */
int srla_group_autotune(srla_group_t *g, int reps, uint32_t *best_threads, uint32_t *best_task_pkts);

/* Checkpoint of one attached link at a slice boundary (no packets pushed in the open group
 * slice, else SRLA_E_ORDER), in the format of srla_export_state: the recorder distances, the
 * link's open slice and its carried hosts.  srla_group_state_bytes gives the buffer size (0
 * for a free slot).  Synchronizes the group's stream.                                     */
size_t srla_group_state_bytes(const srla_group_t *g, uint32_t link);
int srla_group_export_state(srla_group_t *g, uint32_t link, void *host_buf, size_t cap);

int srla_group_sync(srla_group_t *g);
uint64_t srla_group_kernel_launches(const srla_group_t *g);
void srla_group_destroy(srla_group_t *g);


/* ======================================================================================
 * Serving: a request loop over one group.  Links arrive (open), depart (close) and send
 * packet batches (submit) from any host thread; one tick thread calls srla_server_tick
 * once per slice.  A tick applies the departures, admits waiting links in arrival order
 * while their arena bytes fit the HBM budget and a slot is free (continuous batching: a link
 * that arrives while slices are running joins at the next tick), pushes the batches that
 * arrived for admitted links, and closes the slice of every admitted link with one graph
 * launch.  Links are named by the caller's 64-bit keys.
 * ====================================================================================== */
typedef struct srla_server_s srla_server_t;

typedef struct srla_server_config {
  uint32_t max_links;      /* group slots */
  uint32_t max_report;     /* report entries per slice over all links */
  uint64_t max_pkts;       /* packets per slice over all links */
  uint64_t max_host_pkts;  /* of which from host memory */
  uint64_t budget_bytes;   /* admission budget for link regions (at most the arena) */
} srla_server_config;

/* One admitted link's result of a closed slice. */
typedef struct srla_server_result {
  uint64_t key;
  uint32_t first, count;   /* its entries: entries[first .. first + count) */
  srla_slice_stats stats;
} srla_server_result;

/* Workspace bytes: the group's fixed part plus `arena_bytes` for link regions. */
size_t srla_server_workspace_bytes(const srla_server_config *c, uint64_t arena_bytes);
int srla_server_create(const srla_server_config *c, void *dev_workspace, size_t ws_bytes,
                       void *stream, srla_server_t **out);

/* A link arrives with parameters p (queued until admitted).  INVAL: bad p or key in use;
 * NOMEM: the link alone exceeds the budget.                                               */
int srla_server_open(srla_server_t *s, uint64_t key, const srla_params *p);
/* A link departs at the next tick (or leaves the admission queue).                      */
int srla_server_close(srla_server_t *s, uint64_t key);
/* A batch for the link's open slice, pushed at the next tick.  Device or host memory (see
 * srla_push_packets); it must stay unchanged until the tick that pushes it has returned
 * and, for device memory, until that slice's results are polled.  ORDER: the link is not
 * admitted (the batch is not taken).                                                     */
int srla_server_submit(srla_server_t *s, uint64_t key, const uint32_t *pairs, uint64_t n_pairs,
                       int on_device);

/* n batches at once (keys[i], pairs[i], n_pairs[i], all in device or all in host memory).
 * *taken receives how many were queued; batches of links not admitted are skipped.       */
int srla_server_submit_many(srla_server_t *s, uint32_t n, const uint64_t *keys,
                            const uint32_t *const *pairs, const uint64_t *n_pairs, int on_device,
                            uint32_t *taken);

/* Ask the next tick to autotune the group scan on its own batches (srla_group_autotune with
 * reps runs per configuration) before closing the slice.                                 */
int srla_server_autotune(srla_server_t *s, int reps);

/* Close a slice (tick thread).  *slice receives its index; *admitted / *waiting (may be
 * NULL) the links in it and the links still queued for admission.                       */
int srla_server_tick(srla_server_t *s, uint64_t *slice, uint32_t *admitted, uint32_t *waiting);

/* Results of one of the two most recent slices: per admitted link, its key, statistics and
 * entry range in `entries` (sorted by aip within a link).  Driver thread (like tick).     */
int srla_server_poll(srla_server_t *s, uint64_t slice, srla_server_result *results,
                     size_t result_cap, size_t *n_results, srla_entry *entries,
                     size_t entry_cap, size_t *n_entries);

/* Bytes of the budget in use by admitted links (tick thread). */
uint64_t srla_server_used_bytes(const srla_server_t *s);

/* Checkpoint of an admitted link between ticks (tick thread), as srla_group_export_state;
 * SRLA_E_ORDER when the key is not admitted.  srla_server_state_bytes is 0 for such a key. */
size_t srla_server_state_bytes(srla_server_t *s, uint64_t key);
int srla_server_export_state(srla_server_t *s, uint64_t key, void *host_buf, size_t cap);
void srla_server_destroy(srla_server_t *s);

#ifdef __cplusplus
}
#endif

#endif /* SRLA_H */
