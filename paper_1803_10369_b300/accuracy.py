"""Detection accuracy of the CUDA library against the precise method (Section 5).

The precise method counts, for every host ``aip``, the distinct opposite hosts of its pairs in
the window exactly (here: a sort of the window's 64-bit pair keys on the GPU).  With N true
super points (cardinality >= theta), N+ reported hosts that are not super points and N-
super points that are not reported, the paper's rates are FPR = N+/N, FNR = N-/N and
TFR = FPR + FNR (Section 5, definition of FPR/FNR).

Two studies on seeded synthetic traffic (the paper's traces are not available):

* ``discrete``: the parameter sweep of Section 5 under the discrete window (z = 1, k = 1,
  one-bit recorders): g' in {1024 .. 8192}, v in {16384 .. 131072}, u in {2, 4, 8}, g = 8.
  A window is 300 one-second slices of the paper-own traffic pushed into one slice.
* ``sliding``: the sliding window of Section 5 (k = 300, z = 16): windows ending at several
  slices, for the paper's own sketch sizes and for the larger-SRE link of the benchmark, in
  both candidate modes (order-free and the inline test of Algorithm 2).

Run: ``python -m paper_1803_10369_b300.accuracy --study discrete --out results.jsonl``.
"""
from __future__ import annotations

import argparse
import json
import time

import torch

from . import srla

SUPER = srla.SUPER


def pair_keys(batch: torch.Tensor) -> torch.Tensor:
    """(n, 2) int32 pairs -> int64 keys ordered by (aip, bip): equal aips are contiguous."""
    a = batch[:, 0].to(torch.int64)
    b = batch[:, 1].to(torch.int64) & 0xFFFFFFFF
    return (a << 32) | b


def exact_super_points(batches, theta: int) -> set:
    """Hosts with at least theta distinct opposite hosts over all pairs of `batches`."""
    keys = torch.unique(torch.cat([pair_keys(b) for b in batches]))
    hosts, counts = torch.unique_consecutive(keys >> 32, return_counts=True)
    sup = hosts[counts >= theta] & 0xFFFFFFFF
    return set(sup.tolist())


def rates(reported: set, truth: set) -> dict:
    n = len(truth)
    fp = len(reported - truth)
    fn = len(truth - reported)
    fpr = fp / n if n else 0.0
    fnr = fn / n if n else 0.0
    return {"N": n, "reported": len(reported), "N_plus": fp, "N_minus": fn, "fpr": fpr, "fnr": fnr,
            "tfr": fpr + fnr}


def reported_super(rep: dict) -> set:
    return {int(a) for a, f in zip(rep["aip"].tolist(), rep["flags"].tolist()) if f & SUPER}


def _link(w, device, stream, **over):
    import synth

    ha, hb = synth.hash_coefficients(w.hash_seed, w.u + 3)
    p = srla.params_for(w, ha, hb, **over)
    return srla.Link(p, device=device, stream=stream)


def discrete_study(device, windows: int = 2, sub_slices: int = 300, out=print):
    """Section 5's sweep of g', v and u under the discrete window."""
    import synth

    base = synth.workload("paperown").replace(planted_spread=sub_slices)
    stream = torch.cuda.Stream(device)
    data = []
    with torch.cuda.stream(stream):
        for wi in range(windows):
            bs = [synth.generate_slice(base.traffic, wi * sub_slices + s, device=device) for s in range(sub_slices)]
            data.append((torch.cat(bs), exact_super_points(bs, base.theta)))
            del bs
    torch.cuda.synchronize(device)
    for u in (2, 4, 8):
        for v in (1 << 14, 1 << 15, 1 << 16, 1 << 17):
            for gl in (1024, 2048, 4096, 8192):
                w = base.replace(u=u, v=v, gl=gl, g=8, dr_bytes=0, z=1, k=1, max_sampled=1 << 20,
                                 max_candidates=1 << 18)
                link = _link(w, device, stream)
                tot = {"N": 0, "N_plus": 0, "N_minus": 0, "reported": 0}
                t0 = time.perf_counter()
                for pk, truth in data:
                    link.push(pk)
                    r = rates(reported_super(link.report(link.end_slice())), truth)
                    for key in tot:
                        tot[key] += r[key]
                link.close()
                n = max(tot["N"], 1)
                out({"study": "discrete", "u": u, "v": v, "g": 8, "gl": gl, "windows": windows,
                     "pkts_per_window": int(data[0][0].shape[0]), **tot, "fpr": tot["N_plus"] / n,
                     "fnr": tot["N_minus"] / n, "tfr": (tot["N_plus"] + tot["N_minus"]) / n,
                     "seconds": round(time.perf_counter() - t0, 3)})


def sliding_study(device, ends=(300, 350, 400), out=print):
    """Sliding windows of k = 300 one-second slices, both candidate modes."""
    import synth

    stream = torch.cuda.Stream(device)
    for name in ("paperown", "paper"):
        w = synth.workload(name)
        last = max(ends)
        with torch.cuda.stream(stream):
            slices = [synth.generate_slice(w.traffic, s, device=device) for s in range(last)]
        torch.cuda.synchronize(device)
        truth = {e: exact_super_points(slices[e - w.k:e], w.theta) for e in ends}
        for mode in (srla.MODE_ORDER_FREE, srla.MODE_INLINE):
            link = _link(w, device, stream, mode=mode, staging_pkts=w.pkts_per_slice)
            tot = {"N": 0, "N_plus": 0, "N_minus": 0, "reported": 0}
            for s in range(last):
                link.push(slices[s])
                rep = link.report(link.end_slice())
                if s + 1 in truth:
                    r = rates(reported_super(rep), truth[s + 1])
                    for key in tot:
                        tot[key] += r[key]
            link.close()
            n = max(tot["N"], 1)
            out({"study": "sliding", "workload": w.name, "mode": "inline" if mode else "order-free",
                 "u": w.u, "v": w.v, "g": w.g, "gl": w.gl, "k": w.k, "z": w.z, "windows": list(ends), **tot,
                 "fpr": tot["N_plus"] / n, "fnr": tot["N_minus"] / n, "tfr": (tot["N_plus"] + tot["N_minus"]) / n})
        del slices
        torch.cuda.empty_cache()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--study", choices=["discrete", "sliding", "all"], default="all")
    ap.add_argument("--out", default=None, help="JSON lines file (default: stdout)")
    ap.add_argument("--windows", type=int, default=2)
    args = ap.parse_args(argv)
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    fh = open(args.out, "w") if args.out else None

    def out(rec):
        line = json.dumps(rec)
        print(line, flush=True)
        if fh:
            fh.write(line + "\n")
            fh.flush()

    if args.study in ("discrete", "all"):
        discrete_study(device, windows=args.windows, out=out)
    if args.study in ("sliding", "all"):
        sliding_study(device, out=out)
    if fh:
        fh.close()


if __name__ == "__main__":
    main()
