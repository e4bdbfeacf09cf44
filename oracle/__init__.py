"""CPU oracle for SRLA (arXiv 1803.10369) -- TEST INFRASTRUCTURE ONLY.

A plain single-threaded C restatement of the method (``srla_oracle.c``) behind a ctypes
wrapper.  Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg may import this package; the product path never does.  It shares no code with the
CUDA library: the two meet only through the seeded inputs of the ``synth`` package.

``build()`` compiles the C file with gcc into ``oracle/_build/`` (on first use if needed).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "srla_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None

SUPER, SATURATED, CARRIED, NEW = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library; returns its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = f"{_LIB_PATH}.{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        u32, u64, i32, sz = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t
        dbl = ctypes.c_double
        sig = {
            "orc_lsb": (i32, [u32]),
            "orc_tau": (i32, [u32, u32]),
            "orc_rho": (dbl, []),
            "orc_rho_g": (u32, [u32]),
            "orc_hash_ab": (u32, [u64, u64, u32]),
            "orc_estimate": (dbl, [u32, dbl, dbl, P]),
            "orc_create": (P, [u32, u32, u32, u32, u32, u32, u32, P, P, u64]),
            "orc_destroy": (None, [P]),
            "orc_push": (i32, [P, P, sz]),
            "orc_end_slice": (ctypes.c_long, [P]),
            "orc_get_report": (None, [P, P, P, P, P]),
            "orc_get_census": (None, [P, P, P, P]),
            "orc_slice": (u64, [P]),
            "orc_tau_of": (i32, [P]),
            "orc_rho_g_of": (u32, [P]),
            "orc_n_carry": (sz, [P]),
            "orc_get_carry": (None, [P, P]),
            "orc_get_state": (None, [P, P, P]),
            "orc_n_sampled": (sz, [P]),
            "orc_get_sampled": (None, [P, P]),
            "orc_set_state": (i32, [P, P, P, u64, P, sz]),
            "orc_hash_many": (None, [P, i32, P, sz, P]),
            "orc_ure_count": (u32, [P, u32, u32]),
            "orc_ule_count": (u32, [P, u32, u32]),
            "orc_set_inline": (i32, [P, i32]),
            "orc_get_si": (None, [P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ definitions ----

def lsb(x: int) -> int:
    """Definition of LSB (Section 3.2); LSB(0) is taken as 32."""
    return _load().orc_lsb(int(x) & 0xFFFFFFFF)


def tau(theta: int, g: int) -> int:
    """Eq. 1."""
    return _load().orc_tau(theta, g)


def rho() -> float:
    """Section 3.2: rho = 0.99 (1 - e^{-1/3})."""
    return _load().orc_rho()


def rho_g(g: int) -> int:
    return _load().orc_rho_g(g)


def hash_ab(a: int, b: int, x: int) -> int:
    """One member of the hash family: low 32 bits of (a x + b) mod (2^61 - 1)."""
    return _load().orc_hash_ab(int(a), int(b), int(x) & 0xFFFFFFFF)


def estimate(gl: int, up: float, w: float) -> tuple[float, int]:
    """Eq. 9 with the oracle's edge rules; returns (estimate, SATURATED flag or 0)."""
    f = ctypes.c_uint32(0)
    v = _load().orc_estimate(gl, float(up), float(w), ctypes.byref(f))
    return v, f.value


# ------------------------------------------------------------------- estimator ----

class Oracle:
    """One monitored link: the sliding estimator array and its candidate lists."""

    def __init__(self, u, v, g, gl, z, k, theta, ha, hb, start_slice=0, inline=False):
        self._lib = _load()
        self.u, self.v, self.g, self.gl, self.z, self.k, self.theta = u, v, g, gl, z, k, theta
        ha = np.ascontiguousarray(ha, dtype=np.uint64)
        hb = np.ascontiguousarray(hb, dtype=np.uint64)
        if ha.size < u + 3 or hb.size < u + 3:
            raise ValueError("need u + 3 hash coefficient pairs")
        self._h = self._lib.orc_create(u, v, g, gl, z, k, theta, _ptr(ha), _ptr(hb), start_slice)
        if not self._h:
            raise ValueError("invalid oracle parameters")
        self.inline = bool(inline)
        if self.inline and self._lib.orc_set_inline(self._h, 1) != 0:
            raise MemoryError("oracle inline mode")

    @classmethod
    def for_workload(cls, w, ha, hb, inline=False):
        return cls(w.u, w.v, w.g, w.gl, w.z, w.k, w.theta, ha, hb, w.start_slice, inline=inline)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    @property
    def slice(self) -> int:
        return self._lib.orc_slice(self._h)

    @property
    def tau(self) -> int:
        return self._lib.orc_tau_of(self._h)

    @property
    def rho_g(self) -> int:
        return self._lib.orc_rho_g_of(self._h)

    def push(self, pairs: np.ndarray):
        pairs = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
        if self._lib.orc_push(self._h, _ptr(pairs), pairs.shape[0]) != 0:
            raise MemoryError("oracle push")

    def end_slice(self) -> dict:
        n = self._lib.orc_end_slice(self._h)
        if n < 0:
            raise MemoryError("oracle end_slice")
        aip = np.zeros(n, np.uint32)
        w = np.zeros(n, np.uint32)
        est = np.zeros(n, np.float64)
        flags = np.zeros(n, np.uint32)
        self._lib.orc_get_report(self._h, _ptr(aip), _ptr(w), _ptr(est), _ptr(flags))
        cnt = np.zeros(self.u, np.uint64)
        up = ctypes.c_double(0)
        sizes = np.zeros(4, np.uint64)
        self._lib.orc_get_census(self._h, _ptr(cnt), ctypes.byref(up), _ptr(sizes))
        return {"aip": aip, "w": w, "est": est, "flags": flags, "cnt": cnt, "up": up.value,
                "n_sampled_unique": int(sizes[0]), "n_new": int(sizes[1]),
                "n_candidates": int(sizes[2]), "n_carry": int(sizes[3])}

    def state(self):
        """Literal recorder distances: (re[u, v, g], le[u, v, gl]) as uint16."""
        re = np.zeros((self.u, self.v, self.g), np.uint16)
        le = np.zeros((self.u, self.v, self.gl), np.uint16)
        self._lib.orc_get_state(self._h, _ptr(re), _ptr(le))
        return re, le

    def carry(self) -> np.ndarray:
        n = self._lib.orc_n_carry(self._h)
        out = np.zeros(n, np.uint32)
        self._lib.orc_get_carry(self._h, _ptr(out))
        return out

    def sampled(self) -> np.ndarray:
        n = self._lib.orc_n_sampled(self._h)
        out = np.zeros(n, np.uint32)
        self._lib.orc_get_sampled(self._h, _ptr(out))
        return out

    def set_state(self, re, le, T, carry):
        re = np.ascontiguousarray(re, np.uint16)
        le = np.ascontiguousarray(le, np.uint16)
        carry = np.ascontiguousarray(carry, np.uint32)
        if self._lib.orc_set_state(self._h, _ptr(re), _ptr(le), T, _ptr(carry), carry.size) != 0:
            raise MemoryError("oracle set_state")

    def si(self) -> np.ndarray:
        """Super point indicator bits (inline mode): si[u, v] as uint16."""
        out = np.zeros((self.u, self.v), np.uint16)
        self._lib.orc_get_si(self._h, _ptr(out))
        return out

    def hash(self, role: int, x) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.uint32).ravel()
        out = np.zeros(x.size, np.uint32)
        self._lib.orc_hash_many(self._h, role, _ptr(x), x.size, _ptr(out))
        return out

    def ure_count(self, aip: int, limit: int | None = None) -> int:
        return self._lib.orc_ure_count(self._h, int(aip), self.k if limit is None else limit)

    def ule_count(self, aip: int, limit: int | None = None) -> int:
        return self._lib.orc_ule_count(self._h, int(aip), self.k if limit is None else limit)
