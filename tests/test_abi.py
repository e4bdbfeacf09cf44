"""The C ABI without a GPU: the library loads, exports every declared symbol, its structs
have the layout the header gives, and the host-side parameter logic (validation, sizes,
derived constants) is right.  No compute call is made here."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import synth
from paper_1803_10369_b300 import srla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "srla.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(srla_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = srla.lib()
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(srla.SIGNATURES)


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "srla.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(srla_params), '
                    'sizeof(srla_entry), sizeof(srla_slice_stats), offsetof(srla_params, hash_a), '
                    'offsetof(srla_slice_stats, census));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), "-o", str(exe), str(prog)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(srla.srla_params), ctypes.sizeof(srla.srla_entry), ctypes.sizeof(srla.srla_slice_stats),
            srla.srla_params.hash_a.offset, srla.srla_slice_stats.census.offset]
    assert got == want


def _params(**kw):
    a, b = synth.hash_coefficients(1, 19)
    base = dict(u=4, v=1024, g=64, gl=64, dr_bytes=1, z=8, k=4, theta=1024)
    base.update(kw)
    return srla.make_params(hash_a=a, hash_b=b, **base)


def test_param_validation():
    assert srla.check_params(_params()) == 0
    bad = [dict(u=0), dict(u=17), dict(v=1000), dict(g=48), dict(gl=0), dict(dr_bytes=3), dict(z=9),
           dict(pair_slots_log2=9), dict(pair_slots_log2=29), dict(pair_slots_log2=-2),
           dict(dr_bytes=2, z=17), dict(k=0), dict(k=256), dict(z=3, k=8), dict(theta=0),
           dict(g=2, dr_bytes=1), dict(v=1, g=4, gl=4)]
    for kw in bad:
        assert srla.check_params(_params(**kw)) == srla.E_INVAL, kw
        assert srla.workspace_bytes(_params(**kw)) == 0
    p = _params()
    p.hash_a[3] = 0
    assert srla.check_params(p) == srla.E_INVAL
    p = _params()
    p.hash_b[0] = synth.MERSENNE_61
    assert srla.check_params(p) == srla.E_INVAL
    # k = 2^z - 1 is the largest window a z-bit recorder can express (Section 3.2)
    assert srla.check_params(_params(z=3, k=7)) == 0
    assert srla.check_params(_params(z=1, k=1)) == 0


def test_one_bit_recorders():
    """dr_bytes = 0 packs one-bit recorders (z = 1, the discrete window): valid only with z = 1,
    rows of at least 128 recorders, and 1/8 of the recorder bytes of 1-byte cells."""
    one = _params(dr_bytes=0, z=1, k=1)
    assert srla.check_params(one) == 0
    for kw in (dict(z=2, k=1), dict(z=1, k=2), dict(g=2, gl=64), dict(v=16, g=4, gl=64)):
        assert srla.check_params(_params(dr_bytes=0, **{"z": 1, "k": 1, **kw})) == srla.E_INVAL, kw
    big = dict(u=4, v=1 << 16, g=8, gl=1024, z=1, k=1)
    bits = srla.workspace_bytes(_params(dr_bytes=0, **big))
    bytes1 = srla.workspace_bytes(_params(dr_bytes=1, **big))
    cells = 4 * (1 << 16) * (8 + 1024)
    assert bytes1 - bits == cells - cells // 8


def test_inline_mode_params():
    """The inline candidate mode adds the SI words (u*v 32-bit words per slice parity) and is a
    single-link mode: groups refuse it."""
    base = srla.workspace_bytes(_params())
    inl = srla.workspace_bytes(_params(mode=srla.MODE_INLINE))
    assert inl >= base + 2 * 4 * 1024 * 4
    assert srla.check_params(_params(mode=2)) == srla.E_INVAL
    assert srla.Group.link_bytes(_params()) > 0
    assert srla.Group.link_bytes(_params(mode=srla.MODE_INLINE)) == 0


def test_workspace_grows_with_sketch():
    small = srla.workspace_bytes(_params())
    big = srla.workspace_bytes(_params(v=1 << 14, gl=256, g=128, u=8, dr_bytes=2, z=16, k=300))
    assert small > 4 * 1024 * 64 * 2
    assert big > 8 * (1 << 14) * (256 + 128) * 2
    assert small % 256 == 0


def test_derived_constants_agree_with_the_oracle():
    for g in (8, 16, 64, 128, 256):
        for theta in (1, 7, 100, 1000, 1024, 1025, 5000, 1 << 20):
            tau, rg, P = srla.derived(_params(g=g, theta=theta, v=64))
            assert tau == oracle.tau(theta, g)
            assert rg == oracle.rho_g(g)
            assert P == 255


def test_strerror():
    L = srla.lib()
    for c in range(0, -7, -1):
        assert L.srla_strerror(c)


def test_measurement_and_selftest_entry_points_validate_arguments():
    """Argument checks happen before any GPU work (no device needed)."""
    import ctypes

    L = srla.lib()
    fake = ctypes.c_void_p(256)
    assert L.srla_scatter_probe(fake, 1024, 3, 10, 1, 0, None) == srla.E_INVAL
    assert L.srla_scatter_probe(fake, 1, 2, 10, 1, 0, None) == srla.E_INVAL
    assert L.srla_scatter_probe(None, 1024, 2, 10, 1, 0, None) == srla.E_INVAL
    assert L.srla_scatter_probe(fake, 1024, 2, 10, 1, 3, None) == srla.E_INVAL       # unknown policy
    assert L.srla_scatter_probe(ctypes.c_void_p(258), 1024, 2, 10, 1, 1, None) == srla.E_INVAL  # not word-aligned
    assert L.srla_scatter_probe(fake, 3, 1, 10, 1, 1, None) == srla.E_INVAL  # no whole word for the CAS loop
    assert L.srla_wait_selftest(fake, 256, None, 1, 0, 10) == srla.E_INVAL
    assert L.srla_wait_selftest(fake, 256, None, 4, 4, 10) == srla.E_INVAL
    assert L.srla_wait_selftest(fake, 128, None, 4, 1, 10) == srla.E_INVAL
