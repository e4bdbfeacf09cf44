"""Thin Python binding of libsrla (include/srla.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels.  PyTorch provides the device
workspace and the stream.  There is no fallback: if the library cannot be built or loaded,
or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

MAX_ROWS = 16
N_HASH = MAX_ROWS + 3

OK, E_INVAL, E_NOMEM, E_CAPACITY, E_CUDA, E_ORDER, E_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
SUPER, SATURATED, CARRIED, NEW = 1, 2, 4, 8
MODE_ORDER_FREE, MODE_INLINE = 0, 1
SCAN_AUTO, SCAN_PLAIN, SCAN_READ_FIRST, SCAN_HEAVY = 0, 1, 2, 3
SCAN_POLICY_ADAPTIVE, SCAN_POLICY_ADAPTIVE_RF, SCAN_POLICY_OFF, SCAN_POLICY_OFF_RF = 0, 1, 2, 3
SCAN_POLICY_NAMES = {0: "adaptive-table/plain", 1: "adaptive-table/read-first-when-off", 2: "table-off/plain",
                     3: "table-off/read-first"}


class srla_params(ctypes.Structure):
    _fields_ = [
        ("u", ctypes.c_uint32), ("v", ctypes.c_uint32), ("g", ctypes.c_uint32), ("gl", ctypes.c_uint32),
        ("dr_bytes", ctypes.c_uint32), ("z", ctypes.c_uint32), ("k", ctypes.c_uint32), ("theta", ctypes.c_uint32),
        ("start_slice", ctypes.c_uint64), ("staging_pkts", ctypes.c_uint64),
        ("max_sampled", ctypes.c_uint32), ("max_candidates", ctypes.c_uint32),
        ("pair_slots_log2", ctypes.c_int32), ("mode", ctypes.c_uint32),
        ("hash_a", ctypes.c_uint64 * N_HASH), ("hash_b", ctypes.c_uint64 * N_HASH),
    ]


class srla_entry(ctypes.Structure):
    _fields_ = [("aip", ctypes.c_uint32), ("w", ctypes.c_uint32), ("est", ctypes.c_float), ("flags", ctypes.c_uint32)]


class srla_slice_stats(ctypes.Structure):
    _fields_ = [
        ("slice", ctypes.c_uint64), ("n_pkts", ctypes.c_uint64),
        ("n_sampled", ctypes.c_uint32), ("n_new", ctypes.c_uint32), ("n_candidates", ctypes.c_uint32),
        ("n_carry_out", ctypes.c_uint32), ("w_star", ctypes.c_uint32), ("overflow", ctypes.c_uint32),
        ("up", ctypes.c_double), ("census", ctypes.c_uint64 * MAX_ROWS),
        ("pair_table", ctypes.c_uint32), ("heavy_hosts", ctypes.c_uint32),
        ("n_claims", ctypes.c_uint64), ("n_claim_repeats", ctypes.c_uint64),
        ("n_scanned", ctypes.c_uint64), ("n_scanned_sampled", ctypes.c_uint64),
        ("n_set_probes", ctypes.c_uint64), ("n_heavy_events", ctypes.c_uint64),
    ]


ENTRY_DTYPE = np.dtype([("aip", "<u4"), ("w", "<u4"), ("est", "<f4"), ("flags", "<u4")])
assert ENTRY_DTYPE.itemsize == ctypes.sizeof(srla_entry)

_lock = threading.Lock()
_lib = None

# Every symbol declared in include/srla.h, with its ctypes signature.
_P = ctypes.c_void_p
SIGNATURES = {
    "srla_check_params": (ctypes.c_int, [_P]),
    "srla_workspace_bytes": (ctypes.c_size_t, [_P]),
    "srla_derived": (ctypes.c_int, [_P, _P, _P, _P]),
    "srla_create": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P, _P]),
    "srla_push_packets": (ctypes.c_int, [_P, _P, ctypes.c_uint64, ctypes.c_int]),
    "srla_end_slice": (ctypes.c_int, [_P, _P]),
    "srla_report": (ctypes.c_int, [_P, ctypes.c_uint64, _P, ctypes.c_size_t, _P, _P]),
    "srla_sync": (ctypes.c_int, [_P]),
    "srla_state_bytes": (ctypes.c_size_t, [_P]),
    "srla_export_state": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "srla_import_state": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "srla_kernel_launches": (ctypes.c_uint64, [_P]),
    "srla_set_scan_build": (ctypes.c_int, [_P, ctypes.c_uint32]),
    "srla_scan_builds": (ctypes.c_int, [_P, _P, _P, _P]),
    "srla_uses_graph": (ctypes.c_int, [_P]),
    "srla_destroy": (None, [_P]),
    "srla_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "srla_batch_report_static": (ctypes.c_int, [_P, _P, ctypes.c_uint64, _P, _P, ctypes.c_size_t, _P, _P]),
    "srla_wait_selftest": (ctypes.c_int, [_P, ctypes.c_size_t, _P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]),
    "srla_scatter_probe": (ctypes.c_int, [_P, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.c_uint32, _P]),
    "srla_group_fixed_bytes": (ctypes.c_size_t, [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]),
    "srla_group_link_bytes": (ctypes.c_size_t, [_P]),
    "srla_group_create": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, _P,
                                         ctypes.c_size_t, _P, _P]),
    "srla_group_attach": (ctypes.c_int, [_P, _P, _P]),
    "srla_group_detach": (ctypes.c_int, [_P, ctypes.c_uint32]),
    "srla_group_push": (ctypes.c_int, [_P, ctypes.c_uint32, _P, ctypes.c_uint64, ctypes.c_int]),
    "srla_group_end_slice": (ctypes.c_int, [_P, _P]),
    "srla_group_report_all": (ctypes.c_int, [_P, ctypes.c_uint64, _P, ctypes.c_size_t, _P, _P, _P]),
    "srla_group_report": (ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint64, _P, ctypes.c_size_t, _P, _P]),
    "srla_group_autotune": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "srla_group_set_scan_policy": (ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint32]),
    "srla_group_scan_policy": (ctypes.c_int, [_P, ctypes.c_uint32, _P]),
    "srla_group_state_bytes": (ctypes.c_size_t, [_P, ctypes.c_uint32]),
    "srla_group_export_state": (ctypes.c_int, [_P, ctypes.c_uint32, _P, ctypes.c_size_t]),
    "srla_group_sync": (ctypes.c_int, [_P]),
    "srla_group_kernel_launches": (ctypes.c_uint64, [_P]),
    "srla_group_scan_builds": (ctypes.c_int, [_P, _P, _P]),
    "srla_group_destroy": (None, [_P]),
    "srla_server_workspace_bytes": (ctypes.c_size_t, [_P, ctypes.c_uint64]),
    "srla_server_create": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P, _P]),
    "srla_server_open": (ctypes.c_int, [_P, ctypes.c_uint64, _P]),
    "srla_server_close": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "srla_server_submit": (ctypes.c_int, [_P, ctypes.c_uint64, _P, ctypes.c_uint64, ctypes.c_int]),
    "srla_server_submit_many": (ctypes.c_int, [_P, ctypes.c_uint32, _P, _P, _P, ctypes.c_int, _P]),
    "srla_server_autotune": (ctypes.c_int, [_P, ctypes.c_int]),
    "srla_server_tick": (ctypes.c_int, [_P, _P, _P, _P]),
    "srla_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, _P, ctypes.c_size_t, _P, _P, ctypes.c_size_t, _P]),
    "srla_server_used_bytes": (ctypes.c_uint64, [_P]),
    "srla_server_state_bytes": (ctypes.c_size_t, [_P, ctypes.c_uint64]),
    "srla_server_export_state": (ctypes.c_int, [_P, ctypes.c_uint64, _P, ctypes.c_size_t]),
    "srla_server_destroy": (None, [_P]),
}

STATIC_SCRATCH_BYTES = 32 * 1024 * 1024


def lib():
    """Load (building first if needed) the in-tree libsrla.so."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def library_path() -> str:
    return _build.LIB


class SRLAError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = lib().srla_strerror(code).decode()
        super().__init__(f"{what}: {msg} ({code})")


def _ck(code: int, what: str):
    if code != OK:
        raise SRLAError(code, what)


def make_params(u, v, g, gl, dr_bytes, z, k, theta, hash_a, hash_b, start_slice=0, staging_pkts=0,
                max_sampled=1 << 16, max_candidates=1 << 14, pair_slots_log2=0, mode=MODE_ORDER_FREE) -> srla_params:
    p = srla_params()
    p.pair_slots_log2 = pair_slots_log2
    p.mode = mode
    p.u, p.v, p.g, p.gl = u, v, g, gl
    p.dr_bytes, p.z, p.k, p.theta = dr_bytes, z, k, theta
    p.start_slice, p.staging_pkts = start_slice, staging_pkts
    p.max_sampled, p.max_candidates = max_sampled, max_candidates
    ha = np.asarray(hash_a, dtype=np.uint64).ravel()
    hb = np.asarray(hash_b, dtype=np.uint64).ravel()
    for r in range(min(N_HASH, ha.size)):
        p.hash_a[r] = int(ha[r])
        p.hash_b[r] = int(hb[r])
    return p


def wait_selftest(blocks=2, absent=1, spin_limit=10000, device="cuda") -> int:
    """Run the bounded-wait self-test (srla_wait_selftest); returns its status code."""
    import torch

    scratch = torch.zeros(256, dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream(scratch.device)
    return lib().srla_wait_selftest(ctypes.c_void_p(scratch.data_ptr()), 256, ctypes.c_void_p(stream.cuda_stream),
                                    blocks, absent, spin_limit)


PROBE_STORE, PROBE_ATOMIC_MAX, PROBE_READ_FIRST, PROBE_CAS, PROBE_LOAD = 0, 1, 2, 3, 4


def scatter_probe(buf, cell_bytes: int, n_stores: int, seed: int = 1, stream=None, policy: int = PROBE_STORE):
    """Enqueue the store roofline probe (srla_scatter_probe) on `stream` over the torch buffer
    `buf`; `policy` is PROBE_STORE, PROBE_ATOMIC_MAX, PROBE_READ_FIRST, PROBE_CAS (8-byte
    cells) or PROBE_LOAD."""
    import torch

    st = stream if stream is not None else torch.cuda.current_stream(buf.device)
    _ck(lib().srla_scatter_probe(ctypes.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size(), cell_bytes,
                                 n_stores, seed, policy, ctypes.c_void_p(st.cuda_stream)), "srla_scatter_probe")


def _pinned_entries(n: int):
    """A reusable report buffer of n entries in page-locked host memory (device-to-host copies
    into it run at the link's full rate; into pageable memory they are several times slower).
    Returns the numpy view and the torch tensor that owns the memory."""
    import torch

    mem = torch.empty(max(1, n) * ENTRY_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
    return mem.numpy().view(ENTRY_DTYPE)[:n], mem


def params_for(w, hash_a, hash_b, **over) -> srla_params:
    """Parameters of a synth.Workload-like object (fields u, v, g, gl, dr_bytes, z, k, theta...)."""
    kw = dict(u=w.u, v=w.v, g=w.g, gl=w.gl, dr_bytes=w.dr_bytes, z=w.z, k=w.k, theta=w.theta,
              start_slice=w.start_slice, max_sampled=w.max_sampled, max_candidates=w.max_candidates)
    kw.update(over)
    return make_params(hash_a=hash_a, hash_b=hash_b, **kw)


def check_params(p: srla_params) -> int:
    return lib().srla_check_params(ctypes.byref(p))


def workspace_bytes(p: srla_params) -> int:
    return lib().srla_workspace_bytes(ctypes.byref(p))


def derived(p: srla_params):
    tau, rg, pm = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _ck(lib().srla_derived(ctypes.byref(p), ctypes.byref(tau), ctypes.byref(rg), ctypes.byref(pm)), "srla_derived")
    return tau.value, rg.value, pm.value


class Link:
    """One monitored link: a sliding estimator array resident in a torch-owned workspace."""

    def __init__(self, params: srla_params, device="cuda", stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libsrla needs a CUDA device")
        self.params = params
        self.L = lib()
        nbytes = workspace_bytes(params)
        if nbytes == 0:
            raise SRLAError(E_INVAL, "srla_workspace_bytes")
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            h = ctypes.c_void_p()
            _ck(self.L.srla_create(ctypes.byref(params), ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                   ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), "srla_create")
        self._h = h
        self._last = None
        self._out, self._out_mem = _pinned_entries(params.max_candidates)  # reused report buffer

    # -- packets ---------------------------------------------------------------
    def push(self, pairs):
        """pairs: (n, 2) uint32 packets: a CUDA tensor (read in place), or host memory (numpy
        array or CPU tensor; pinned tensors give an asynchronous copy)."""
        import torch

        if isinstance(pairs, torch.Tensor):
            if pairs.dtype not in (torch.int32, torch.uint32) or not pairs.is_contiguous():
                raise ValueError("pairs must be a contiguous int32/uint32 tensor of shape (n, 2)")
            n = pairs.numel() // 2
            on_dev = 1 if pairs.is_cuda else 0
            ptr = pairs.data_ptr()
            self._keep = pairs
        else:
            arr = np.ascontiguousarray(pairs, dtype=np.uint32)
            n = arr.size // 2
            on_dev = 0
            ptr = arr.ctypes.data
            self._keep = arr
        _ck(self.L.srla_push_packets(self._h, ctypes.c_void_p(ptr), n, on_dev), "srla_push_packets")

    def end_slice(self) -> int:
        sid = ctypes.c_uint64()
        _ck(self.L.srla_end_slice(self._h, ctypes.byref(sid)), "srla_end_slice")
        self._last = sid.value
        return sid.value

    def report(self, slice_id=None, cap=None, allow_overflow=False):
        """Sorted report of a closed slice: dict of numpy arrays (aip, w, est, flags) + stats."""
        if slice_id is None:
            slice_id = self._last
        if cap is None:
            cap = self.params.max_candidates
            out = self._out
        else:
            out = np.empty(cap, dtype=ENTRY_DTYPE)
        n = ctypes.c_size_t()
        st = srla_slice_stats()
        rc = self.L.srla_report(self._h, slice_id, ctypes.c_void_p(out.ctypes.data), cap, ctypes.byref(n),
                                ctypes.byref(st))
        if rc != OK and not (allow_overflow and rc == E_CAPACITY):
            raise SRLAError(rc, "srla_report")
        m = min(n.value, cap)
        e = out[:m].copy()  # one contiguous copy out of the reused buffer; the fields view it
        stats = {f: getattr(st, f) for f, _ in srla_slice_stats._fields_ if f != "census"}
        stats["census"] = np.array(st.census[: self.params.u], dtype=np.uint64)
        return {"aip": e["aip"], "w": e["w"], "est": e["est"], "flags": e["flags"], "stats": stats, "rc": rc}

    def kernel_launches(self) -> int:
        return self.L.srla_kernel_launches(self._h)

    def set_scan_build(self, build: int):
        """SCAN_AUTO, SCAN_PLAIN, SCAN_READ_FIRST or SCAN_HEAVY (srla_set_scan_build)."""
        _ck(self.L.srla_set_scan_build(self._h, build), "srla_set_scan_build")

    def scan_builds(self):
        """Scan launches so far of the plain, read-first and heavy builds."""
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _ck(self.L.srla_scan_builds(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "srla_scan_builds")
        return a.value, b.value, c.value

    def uses_graph(self) -> bool:
        return bool(self.L.srla_uses_graph(self._h))

    def sync(self):
        _ck(self.L.srla_sync(self._h), "srla_sync")

    # -- checkpoint --------------------------------------------------------------
    def export_state(self) -> bytes:
        n = self.L.srla_state_bytes(self._h)
        buf = ctypes.create_string_buffer(n)
        _ck(self.L.srla_export_state(self._h, buf, n), "srla_export_state")
        return buf.raw

    def import_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _ck(self.L.srla_import_state(self._h, buf, len(blob)), "srla_import_state")

    def state_arrays(self):
        """Exported state as (re[u, v, g], le[u, v, gl], slice, carried hosts), distances uint16."""
        return state_arrays_of(self.params, self.export_state())

    def close(self):
        if getattr(self, "_h", None):
            self.L.srla_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def state_arrays_of(p: srla_params, b: bytes):
    """Split an exported state (srla_export_state format) into (re[u, v, g], le[u, v, gl],
    open slice, carried hosts); distances are uint16."""
    hdr = np.frombuffer(b[:56], dtype=np.uint32)
    slice_ = int(np.frombuffer(b[40:48], dtype=np.uint64)[0])
    n_carry = int(hdr[12])
    nre, nle = p.u * p.v * p.g, p.u * p.v * p.gl
    d = np.frombuffer(b[56:56 + 2 * (nre + nle)], dtype=np.uint16)
    re = d[:nre].reshape(p.u, p.v, p.g).copy()
    le = d[nre:].reshape(p.u, p.v, p.gl).copy()
    carry = np.frombuffer(b[56 + 2 * (nre + nle):56 + 2 * (nre + nle) + 4 * n_carry], dtype=np.uint32).copy()
    return re, le, slice_, carry


def _stats_dict(st, u):
    d = {f: getattr(st, f) for f, _ in srla_slice_stats._fields_ if f != "census"}
    d["census"] = np.array(st.census[:u], dtype=np.uint64)
    return d


def _pairs_arg(pairs):
    """(pointer, n, on_device, keep-alive object) of a batch of (n, 2) uint32 pairs."""
    import torch

    if isinstance(pairs, torch.Tensor):
        if pairs.dtype not in (torch.int32, torch.uint32) or not pairs.is_contiguous():
            raise ValueError("pairs must be a contiguous int32/uint32 tensor of shape (n, 2)")
        return pairs.data_ptr(), pairs.numel() // 2, 1 if pairs.is_cuda else 0, pairs
    arr = np.ascontiguousarray(pairs, dtype=np.uint32)
    return arr.ctypes.data, arr.size // 2, 0, arr


class Group:
    """Many links advanced together: one CUDA graph launch scans and closes every link's slice.

    The workspace is one torch tensor: a fixed part plus an arena for link regions
    (``arena_bytes``).  Links attach and detach between slices."""

    def __init__(self, max_links, max_pkts, arena_bytes, max_host_pkts=0, max_report=1 << 16, device="cuda",
                 stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libsrla needs a CUDA device")
        self.L = lib()
        self.max_links, self.max_report = max_links, max_report
        fixed = self.L.srla_group_fixed_bytes(max_links, max_pkts, max_host_pkts, max_report)
        if fixed == 0:
            raise SRLAError(E_INVAL, "srla_group_fixed_bytes")
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(fixed + int(arena_bytes), dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            h = ctypes.c_void_p()
            _ck(self.L.srla_group_create(max_links, max_pkts, max_host_pkts, max_report,
                                         ctypes.c_void_p(self.workspace.data_ptr()), self.workspace.numel(),
                                         ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
                "srla_group_create")
        self._h = h
        self.params = {}
        self._keep = []
        self._out, self._out_mem = _pinned_entries(max_report)

    @staticmethod
    def link_bytes(params: srla_params) -> int:
        return lib().srla_group_link_bytes(ctypes.byref(params))

    def attach(self, params: srla_params) -> int:
        link = ctypes.c_uint32()
        _ck(self.L.srla_group_attach(self._h, ctypes.byref(params), ctypes.byref(link)), "srla_group_attach")
        self.params[link.value] = params
        return link.value

    def detach(self, link: int):
        _ck(self.L.srla_group_detach(self._h, link), "srla_group_detach")
        self.params.pop(link, None)

    def push(self, link: int, pairs):
        ptr, n, on_dev, keep = _pairs_arg(pairs)
        self._keep.append(keep)
        _ck(self.L.srla_group_push(self._h, link, ctypes.c_void_p(ptr), n, on_dev), "srla_group_push")

    def end_slice(self) -> int:
        gs = ctypes.c_uint64()
        _ck(self.L.srla_group_end_slice(self._h, ctypes.byref(gs)), "srla_group_end_slice")
        self._last = gs.value
        self._keep = self._keep[-4096:]
        return gs.value

    def report_all(self, gs=None, allow_overflow=False):
        """{link: report dict} for every link attached at group slice gs."""
        if gs is None:
            gs = self._last
        n = ctypes.c_size_t()
        offs = (ctypes.c_uint32 * (self.max_links + 1))()
        stats = (srla_slice_stats * self.max_links)()
        rc = self.L.srla_group_report_all(self._h, gs, ctypes.c_void_p(self._out.ctypes.data), self.max_report,
                                          ctypes.byref(n), offs, stats)
        if rc != OK and not (allow_overflow and rc == E_CAPACITY):
            raise SRLAError(rc, "srla_group_report_all")
        out = {}
        for link, p in self.params.items():
            e = self._out[offs[link]:offs[link + 1]]
            out[link] = {"aip": e["aip"].copy(), "w": e["w"].copy(), "est": e["est"].copy(),
                         "flags": e["flags"].copy(), "stats": _stats_dict(stats[link], p.u), "rc": rc}
        return out

    def report(self, link: int, gs=None, allow_overflow=False):
        if gs is None:
            gs = self._last
        p = self.params[link]
        out = np.empty(p.max_candidates, dtype=ENTRY_DTYPE)
        n = ctypes.c_size_t()
        st = srla_slice_stats()
        rc = self.L.srla_group_report(self._h, link, gs, ctypes.c_void_p(out.ctypes.data), p.max_candidates,
                                      ctypes.byref(n), ctypes.byref(st))
        if rc != OK and not (allow_overflow and rc == E_CAPACITY):
            raise SRLAError(rc, "srla_group_report")
        e = out[:min(n.value, p.max_candidates)]
        return {"aip": e["aip"].copy(), "w": e["w"].copy(), "est": e["est"].copy(), "flags": e["flags"].copy(),
                "stats": _stats_dict(st, p.u), "rc": rc}

    def autotune(self, reps=3):
        """Pick the scan block size, task size and per-class aggregation policies on the open
        slice's packets; returns (block size, packets per task)."""
        t, k = ctypes.c_uint32(), ctypes.c_uint32()
        _ck(self.L.srla_group_autotune(self._h, reps, ctypes.byref(t), ctypes.byref(k)), "srla_group_autotune")
        return t.value, k.value

    def set_scan_policy(self, link: int, policy: int):
        _ck(self.L.srla_group_set_scan_policy(self._h, link, policy), "srla_group_set_scan_policy")

    def scan_policy(self, link: int) -> int:
        p = ctypes.c_uint32()
        _ck(self.L.srla_group_scan_policy(self._h, link, ctypes.byref(p)), "srla_group_scan_policy")
        return p.value

    def state_arrays(self, link: int):
        """One link's exported state (srla_group_export_state), as Link.state_arrays."""
        n = self.L.srla_group_state_bytes(self._h, link)
        if n == 0:
            raise SRLAError(E_INVAL, "srla_group_state_bytes")
        buf = ctypes.create_string_buffer(n)
        _ck(self.L.srla_group_export_state(self._h, link, buf, n), "srla_group_export_state")
        return state_arrays_of(self.params[link], buf.raw)

    def sync(self):
        _ck(self.L.srla_group_sync(self._h), "srla_group_sync")

    def kernel_launches(self) -> int:
        return self.L.srla_group_kernel_launches(self._h)

    def scan_builds(self):
        """(lean, read_first): slice ends that ran each group scan instantiation."""
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        _ck(self.L.srla_group_scan_builds(self._h, ctypes.byref(a), ctypes.byref(b)), "srla_group_scan_builds")
        return a.value, b.value

    def close(self):
        if getattr(self, "_h", None):
            self.L.srla_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class srla_server_config(ctypes.Structure):
    _fields_ = [("max_links", ctypes.c_uint32), ("max_report", ctypes.c_uint32), ("max_pkts", ctypes.c_uint64),
                ("max_host_pkts", ctypes.c_uint64), ("budget_bytes", ctypes.c_uint64)]


class srla_server_result(ctypes.Structure):
    _fields_ = [("key", ctypes.c_uint64), ("first", ctypes.c_uint32), ("count", ctypes.c_uint32),
                ("stats", srla_slice_stats)]


class Server:
    """Serving loop over one link group: links open and close, batches arrive, tick() closes
    a slice for every admitted link (admission in arrival order under a byte budget)."""

    def __init__(self, max_links, max_pkts, budget_bytes, arena_bytes=None, max_host_pkts=0, max_report=1 << 20,
                 device="cuda", stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libsrla needs a CUDA device")
        self.L = lib()
        self.cfg = srla_server_config(max_links, max_report, max_pkts, max_host_pkts, budget_bytes)
        arena = int(arena_bytes if arena_bytes is not None else budget_bytes + (64 << 20))
        nbytes = self.L.srla_server_workspace_bytes(ctypes.byref(self.cfg), arena)
        if nbytes == 0:
            raise SRLAError(E_INVAL, "srla_server_workspace_bytes")
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            h = ctypes.c_void_p()
            _ck(self.L.srla_server_create(ctypes.byref(self.cfg), ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                          ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
                "srla_server_create")
        self._h = h
        self.params = {}
        self._keep = []
        self._res = (srla_server_result * max_links)()
        self._ent = np.empty(max_report, dtype=ENTRY_DTYPE)

    def open(self, key: int, params: srla_params):
        _ck(self.L.srla_server_open(self._h, key, ctypes.byref(params)), "srla_server_open")
        self.params[key] = params

    def close(self, key: int):
        _ck(self.L.srla_server_close(self._h, key), "srla_server_close")

    def submit(self, key: int, pairs) -> bool:
        """Queue a batch; False if the link is not admitted yet (the batch is not taken)."""
        ptr, n, on_dev, keep = _pairs_arg(pairs)
        rc = self.L.srla_server_submit(self._h, key, ctypes.c_void_p(ptr), n, on_dev)
        if rc == E_ORDER:
            return False
        _ck(rc, "srla_server_submit")
        self._keep.append(keep)
        return True

    def submit_many(self, keys, batches) -> int:
        """Queue many device batches in one call (all CUDA tensors); returns how many were taken."""
        n = len(keys)
        if n == 0:
            return 0
        karr = (ctypes.c_uint64 * n)(*keys)
        parr = (ctypes.c_void_p * n)(*[b.data_ptr() for b in batches])
        narr = (ctypes.c_uint64 * n)(*[b.numel() // 2 for b in batches])
        if not all(b.is_cuda and b.is_contiguous() for b in batches):
            raise ValueError("submit_many takes contiguous CUDA tensors")
        taken = ctypes.c_uint32()
        _ck(self.L.srla_server_submit_many(self._h, n, karr, parr, narr, 1, ctypes.byref(taken)),
            "srla_server_submit_many")
        self._keep.extend(batches)
        return taken.value

    def autotune(self, reps=3):
        _ck(self.L.srla_server_autotune(self._h, reps), "srla_server_autotune")

    def tick(self):
        sl, adm, wt = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32()
        _ck(self.L.srla_server_tick(self._h, ctypes.byref(sl), ctypes.byref(adm), ctypes.byref(wt)), "srla_server_tick")
        self._keep = self._keep[-8192:]
        return sl.value, adm.value, wt.value

    def poll(self, slice_id: int):
        """{key: report dict} of the links admitted in that slice."""
        nr, ne = ctypes.c_size_t(), ctypes.c_size_t()
        rc = self.L.srla_server_poll(self._h, slice_id, self._res, len(self._res), ctypes.byref(nr),
                                     ctypes.c_void_p(self._ent.ctypes.data), len(self._ent), ctypes.byref(ne))
        if rc not in (OK, E_CAPACITY):
            raise SRLAError(rc, "srla_server_poll")
        out = {}
        for i in range(nr.value):
            r = self._res[i]
            e = self._ent[r.first:r.first + r.count]
            u = self.params[r.key].u if r.key in self.params else MAX_ROWS
            out[r.key] = {"aip": e["aip"].copy(), "w": e["w"].copy(), "est": e["est"].copy(),
                          "flags": e["flags"].copy(), "stats": _stats_dict(r.stats, u), "rc": rc}
        return out

    def used_bytes(self) -> int:
        return self.L.srla_server_used_bytes(self._h)

    def state_arrays(self, key: int):
        """An admitted link's exported state (srla_server_export_state), as Link.state_arrays."""
        n = self.L.srla_server_state_bytes(self._h, key)
        if n == 0:
            raise SRLAError(E_ORDER, "srla_server_state_bytes")
        buf = ctypes.create_string_buffer(n)
        _ck(self.L.srla_server_export_state(self._h, key, buf, n), "srla_server_export_state")
        return state_arrays_of(self.params[key], buf.raw)

    def destroy(self):
        if getattr(self, "_h", None):
            self.L.srla_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def batch_report_static(params: srla_params, pairs, stream=None, cap=None, allow_overflow=False):
    """Report of one device batch through the allocation-free entry point (no workspace).

    Same result as a fresh Link that pushes `pairs` and closes its first slice.  The library
    keeps one fixed scratch array per GPU, so calls must not overlap on the device."""
    import torch

    if not (isinstance(pairs, torch.Tensor) and pairs.is_cuda and pairs.is_contiguous()):
        raise ValueError("pairs must be a contiguous CUDA tensor of shape (n, 2)")
    if stream is None:
        stream = torch.cuda.current_stream(pairs.device)
    if cap is None:
        cap = params.max_candidates
    out = np.zeros(cap, dtype=ENTRY_DTYPE)
    n = ctypes.c_size_t()
    st = srla_slice_stats()
    rc = lib().srla_batch_report_static(ctypes.byref(params), ctypes.c_void_p(pairs.data_ptr()), pairs.numel() // 2,
                                        ctypes.c_void_p(stream.cuda_stream), ctypes.c_void_p(out.ctypes.data), cap,
                                        ctypes.byref(n), ctypes.byref(st))
    if rc != OK and not (allow_overflow and rc == E_CAPACITY):
        raise SRLAError(rc, "srla_batch_report_static")
    e = out[:min(n.value, cap)]
    stats = {f: getattr(st, f) for f, _ in srla_slice_stats._fields_ if f != "census"}
    stats["census"] = np.array(st.census[: params.u], dtype=np.uint64)
    return {"aip": e["aip"].copy(), "w": e["w"].copy(), "est": e["est"].copy(), "flags": e["flags"].copy(),
            "stats": stats, "rc": rc}
