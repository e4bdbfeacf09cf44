"""Steady state at the benchmarked geometries, against the CPU oracle.

The benchmark runs the paper-scale link (u = 8, v = 2^14, g = 128, g' = 256, 16-bit
recorders, k = 300) after filling its window with k slices.  These tests check that state:

* a run of k + 8 slices at that geometry (packets per slice reduced so that the oracle keeps
  up), compared with the oracle every slice (reports) and every 50 slices (every recorder
  distance and the carried list): recorders age out of a full window (Algorithm 3's slide),
  and the traffic alternates between the flow model and runs of uniform destinations, so the
  per-slice pair table is switched off and on again and the scan runs both of its builds;
* states that hold distances from the whole range [1, 2^z - 1] (stamps about to saturate,
  stamps at the window's edge), built by the oracle and imported into the library at a slice
  index where the 16-bit stamps wrap, then continued slice by slice: this is where the sweep
  clears the stamps whose distance reaches 2^z - 1 (Section 3.2's saturation), at the paper-
  scale geometry and at the paper's own (u = 4, v = 65536, g = 8, g' = 1024).
"""
import dataclasses

import numpy as np
import pytest

import synth
from gpu_helpers import compare_reports, compare_state, make_pair
from paper_1803_10369_b300 import srla

pytestmark = pytest.mark.gpu

PAPER = synth.workload("paper")
PAPER_OWN = synth.workload("paperown")


def _slice(w, s, device, pkts_uniform=100_000):
    """Slice s of w's traffic (drawn on the GPU; the same bytes go to both sides); slices
    20..39 of every 80 send uniform destinations instead (almost no pair repeats: the pair
    table is switched off and the read-first scan runs)."""
    if (s // 20) % 4 == 1:
        spec = dataclasses.replace(w.traffic, dst_model="uniform", dst_space=1 << 20, pkts_per_slice=pkts_uniform)
        return synth.generate_slice(spec, s, device=device)
    return synth.generate_slice(w.traffic, s, device=device)


def test_paper_geometry_full_window(cuda_device):
    w = PAPER.replace(pkts_per_slice=250_000)
    o, link = make_pair(w)
    n = w.k + 8
    table = set()
    n_cand = 0
    for s in range(n):
        pk = _slice(w, s, cuda_device)
        o.push(synth.pairs_to_numpy(pk))
        link.push(pk)
        ro = o.end_slice()
        rg = link.report(link.end_slice())
        compare_reports(ro, rg, f"slice {s}")
        table.add(int(rg["stats"]["pair_table"]))
        n_cand = max(n_cand, ro["n_candidates"])
        if (s + 1) % 50 == 0 or s == n - 1:
            compare_state(o, link, f"slice {s}")
    plain, read_first, _ = link.scan_builds()
    assert table == {0, 1}, table            # the pair table was switched off and on again
    assert plain > 0 and read_first > 0, (plain, read_first)
    assert n_cand >= 100
    link.close()
    o.close()


def _designed_state(w, rng):
    """Recorder distances drawn over [1, 2^z - 1]: empty cells, cells inside or at the edge of
    the window, cells a few slices from saturation (their stamps alias the open slice's next
    codes), and cells anywhere in between."""
    P = (1 << w.z) - 1

    def draw(shape):
        n = int(np.prod(shape))
        kind = rng.random(n)
        d = np.full(n, P, dtype=np.int64)
        a = kind < 0.15
        d[a] = rng.integers(1, w.k + 6, size=a.sum())
        b = (kind >= 0.15) & (kind < 0.30)
        d[b] = rng.integers(P - 16, P, size=b.sum())
        c = (kind >= 0.30) & (kind < 0.60)
        d[c] = rng.integers(1, P, size=c.sum())
        return d.astype(np.uint16).reshape(shape)

    return draw((w.u, w.v, w.g)), draw((w.u, w.v, w.gl))


def _import_and_continue(w, n_slices, cuda_device, T0, seed):
    rng = np.random.default_rng(seed)
    o, link = make_pair(w)
    re, le = _designed_state(w, rng)
    first = synth.pairs_to_numpy(synth.generate_slice(w.traffic, 0, device=cuda_device))
    carry = np.unique(first[:, 0])[:500]  # carried into the first slice (Algorithm 3)
    o.set_state(re, le, T0, carry)
    blob = bytearray(link.export_state())
    hdr = np.frombuffer(bytes(blob[:56]), dtype=np.uint32).copy()
    hdr[10:12] = np.frombuffer(np.uint64(T0).tobytes(), dtype=np.uint32)
    hdr[12] = carry.size
    link.import_state(hdr.tobytes() + re.tobytes() + le.tobytes() + carry.astype(np.uint32).tobytes())
    compare_state(o, link, "after import")
    for s in range(n_slices):
        pk = synth.generate_slice(w.traffic, s, device=cuda_device)
        o.push(synth.pairs_to_numpy(pk))
        link.push(pk)
        compare_reports(o.end_slice(), link.report(link.end_slice()), f"{w.name} slice {T0 + s}")
        compare_state(o, link, f"{w.name} slice {T0 + s}")
    link.close()
    o.close()


def test_paper_geometry_saturating_stamps_after_import(cuda_device):
    """Stamps of distance 2^16 - 2 saturate at the first slice end; the open slice index
    crosses a multiple of 2^16 - 1 (the stamp code wraps) after five slices."""
    w = PAPER.replace(pkts_per_slice=250_000)
    P = (1 << w.z) - 1
    _import_and_continue(w, 12, cuda_device, T0=2 * P - 5, seed=5)


def test_paper_own_geometry_saturating_stamps_after_import(cuda_device):
    w = PAPER_OWN.replace(pkts_per_slice=250_000)
    P = (1 << w.z) - 1
    _import_and_continue(w, 8, cuda_device, T0=3 * P - 3, seed=6)
