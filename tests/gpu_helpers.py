"""Helpers shared by the GPU parity tests: run the oracle and the CUDA path side by side on
the same seeded packets and compare everything they expose."""
from __future__ import annotations

import math

import numpy as np

import oracle
import synth
from paper_1803_10369_b300 import srla

EST_RTOL = 1e-5  # FP32 estimates against the FP64 oracle (relative)


def compare_reports(ro: dict, rg: dict, where: str = ""):
    """Bit-exact integers; estimates within EST_RTOL relative (infinities must match)."""
    assert rg["aip"].tolist() == ro["aip"].tolist(), f"{where}: candidate lists differ"
    assert np.array_equal(rg["w"], ro["w"]), f"{where}: union SLE weights differ"
    assert np.array_equal(rg["flags"], ro["flags"]), f"{where}: flags differ"
    eo = ro["est"]
    eg = rg["est"].astype(np.float64)
    inf_o, inf_g = np.isinf(eo), np.isinf(eg)
    assert np.array_equal(inf_o, inf_g), f"{where}: saturation differs"
    fin = ~inf_o
    err = np.abs(eg[fin] - eo[fin])
    assert (err <= EST_RTOL * np.abs(eo[fin]) + 1e-30).all(), f"{where}: estimates off by {err.max() if err.size else 0}"
    st = rg["stats"]
    assert np.array_equal(st["census"], ro["cnt"]), f"{where}: row census differs"
    assert math.isclose(st["up"], ro["up"], rel_tol=1e-12, abs_tol=0.0), f"{where}: UP differs"
    assert st["n_sampled"] == ro["n_sampled_unique"], f"{where}: sampled host count differs"
    assert st["n_new"] == ro["n_new"], f"{where}: new candidate count differs"
    assert st["n_candidates"] == ro["n_candidates"], f"{where}: candidate count differs"
    assert st["n_carry_out"] == ro["n_carry"], f"{where}: carried count differs"


def compare_state(o: "oracle.Oracle", link, where: str = ""):
    """Exported recorder distances, open slice and carried list against the oracle's.  `link`
    is a srla.Link, or the (re, le, slice, carry) tuple of a group or served link's export."""
    re_g, le_g, T_g, carry_g = link if isinstance(link, tuple) else link.state_arrays()
    re_o, le_o = o.state()
    assert T_g == o.slice, f"{where}: open slice differs"
    assert np.array_equal(re_g, re_o), f"{where}: SRE recorders differ ({(re_g != re_o).sum()} cells)"
    assert np.array_equal(le_g, le_o), f"{where}: SLE recorders differ ({(le_g != le_o).sum()} cells)"
    assert carry_g.tolist() == o.carry().tolist(), f"{where}: carried lists differ"


def make_pair(w, device="cuda", **over):
    ha, hb = synth.hash_coefficients(w.hash_seed, w.u + 3)
    o = oracle.Oracle.for_workload(w, ha, hb)
    link = srla.Link(srla.params_for(w, ha, hb, **over), device=device)
    return o, link


def oracle_for(params, start_slice=None) -> "oracle.Oracle":
    """An oracle with the geometry, window, threshold and hash coefficients of libsrla
    parameters (one-bit recorders are z = 1 distances, as everywhere)."""
    u = params.u
    ha = np.array([params.hash_a[r] for r in range(u + 3)], dtype=np.uint64)
    hb = np.array([params.hash_b[r] for r in range(u + 3)], dtype=np.uint64)
    return oracle.Oracle(u, params.v, params.g, params.gl, params.z, params.k, params.theta, ha, hb,
                         params.start_slice if start_slice is None else start_slice)
