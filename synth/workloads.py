"""Named workloads: sketch geometry plus the synthetic traffic that drives it.

Geometry symbols follow the paper: ``u`` rows and ``v`` columns of sliding estimators
(Section 4.1), ``g`` SRE cells and ``gl`` (the paper's g') SLE cells per estimator, ``z``-bit
distance recorders stored in ``dr_bytes`` bytes, window ``k`` slices (Section 3.1) and
threshold ``theta`` (Definition 2).  ``gl`` is the per-row SLE size divided by ``v``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .traces import TrafficSpec


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    u: int
    v: int
    g: int
    gl: int
    dr_bytes: int
    z: int
    k: int
    theta: int
    n_slices: int
    traffic: TrafficSpec
    hash_seed: int = 1
    start_slice: int = 0
    max_sampled: int = 1 << 16
    max_candidates: int = 1 << 14

    @property
    def pkts_per_slice(self) -> int:
        return self.traffic.pkts_per_slice

    def replace(self, **kw) -> "Workload":
        tkw = {k: kw.pop(k) for k in list(kw) if k in TrafficSpec.__dataclass_fields__}
        w = dataclasses.replace(self, **kw)
        if tkw:
            w = dataclasses.replace(w, traffic=dataclasses.replace(w.traffic, **tkw))
        return w


# 1 link, 16 slices of 2^16 packets, window 4 slices, 8-bit recorders.
TINY = Workload(
    name="tiny-1link-u4-v1024-g64-gl64-z8-k4",
    u=4, v=1 << 10, g=64, gl=64, dr_bytes=1, z=8, k=4, theta=1024, n_slices=16,
    traffic=TrafficSpec(
        seed=1, pkts_per_slice=1 << 16, n_src=1 << 12, zipf_s=1.1,
        dst_model="uniform", dst_space=1 << 20,
        n_planted=20, planted_card=(500, 3000), planted_card_dist="uniform",
        planted_spread=16),
    max_sampled=1 << 14, max_candidates=1 << 13,
)

# Paper-scale single link: 1 s slices, window 300 slices, ~5M packets per slice.
PAPER = Workload(
    name="paper-1link-u8-v16384-g128-gl256-z16-k300-5Mpps",
    u=8, v=1 << 14, g=128, gl=256, dr_bytes=2, z=16, k=300, theta=1024, n_slices=320,
    traffic=TrafficSpec(
        seed=2, pkts_per_slice=5_000_000, n_src=1 << 20, zipf_s=1.2,
        dst_model="pool", pool_alpha=1.5, pool_max=128,
        n_planted=500, planted_card=(1 << 10, 1 << 16), planted_card_dist="loguniform",
        planted_spread=300, churn_frac=0.3, churn_run=(75, 300)),
    max_sampled=1 << 20, max_candidates=1 << 18,
)

# Long-window stress: window 1024 slices, 2M packets per slice, stamp wraparound,
# one heavy source with 10% of the packets, a flood of 2^24 spoofed one-packet sources
# spread over 16 slices.
LONGWIN = Workload(
    name="longwin-1link-u8-v16384-g128-gl256-z16-k1024-2Mpps-flood",
    u=8, v=1 << 14, g=128, gl=256, dr_bytes=2, z=16, k=1024, theta=1024, n_slices=1040,
    traffic=TrafficSpec(
        seed=3, pkts_per_slice=2_000_000, n_src=1 << 20, zipf_s=1.2,
        dst_model="pool", pool_alpha=1.5, pool_max=128,
        n_planted=500, planted_card=(1 << 10, 1 << 16), planted_card_dist="loguniform",
        planted_spread=1024, churn_frac=0.3, churn_run=(256, 1024),
        heavy_frac=0.10, flood_sources=1 << 24, flood_slices=(4, 20)),
    start_slice=(1 << 16) - 1 - 8,
    max_sampled=1 << 21, max_candidates=1 << 20,
)

# The paper's own parameters (Section 5): u=4 rows, v=65536 columns, g=8 SRE cells and
# g'=1024 SLE cells per estimator, 16-bit recorders, window 300 slices, 4.5M packets per slice
# (the traces' average rate); same traffic recipe as PAPER.
PAPER_OWN = Workload(
    name="paperown-1link-u4-v65536-g8-gl1024-z16-k300-4.5Mpps",
    u=4, v=1 << 16, g=8, gl=1024, dr_bytes=2, z=16, k=300, theta=1024, n_slices=320,
    traffic=dataclasses.replace(PAPER.traffic, seed=6, pkts_per_slice=4_500_000),
    max_sampled=1 << 18, max_candidates=1 << 18,
)

# The paper's discrete-window regime (Section 5: z = 1, k = 1) at its own sketch sizes, with
# one-bit recorders packed 32 to a word (33 MiB of recorders instead of 516 MiB at 16 bits).
# Each slice is a whole window, so a planted host reaches its cardinality within one slice;
# 60 planted hosts keep their packets near a fifth of the slice.
DISCRETE = PAPER_OWN.replace(
    name="discrete-1link-u4-v65536-g8-gl1024-z1-k1-bits-4.5Mpps", dr_bytes=0, z=1, k=1, n_slices=16,
    n_planted=60, planted_spread=1, churn_run=(1, 4))

# Paper-scale traffic in flow bursts: every background pair sends a geometric number of
# packets (mean 8) back to back, so warps see runs of the same pair (duplicate elision).
BURST = PAPER.replace(name="burst-1link-u8-v16384-g128-gl256-z16-k300-5Mpps-mean8", seed=7, burst_mean=8.0)

# The literal reading of the paper-scale traffic: background destinations uniform over 2^20
# addresses.  About 10^9 distinct pairs per window saturate every SRE and SLE row, so nearly
# every sampled source becomes a candidate and is reported saturated (a stress case: candidate
# lists of about a million hosts to sort, estimate and carry every slice).
UNIFORM = PAPER.replace(name="uniform-1link-u8-v16384-g128-gl256-z16-k300-5Mpps-saturating", seed=8,
                        dst_model="uniform", dst_space=1 << 20, max_candidates=1 << 21)

WORKLOADS = {"tiny": TINY, "paper": PAPER, "longwin": LONGWIN, "paperown": PAPER_OWN, "discrete": DISCRETE,
             "burst": BURST, "uniform": UNIFORM}


def workload(name: str) -> Workload:
    return WORKLOADS[name]


def batched_links(n_links: int = 64, seed: int = 4):
    """Many independent links of uneven rates (one estimator array each).

    Rates are log-uniform in [10^4, 5*10^6] packets per slice, windows log-uniform in
    [16, 300] slices, 8- or 16-bit recorders (8-bit only where the window fits), and the SLE
    is scaled to the rate (2^16 .. 2^22 cells per row, g' = 256).  Returns a list of
    (Workload, pair_slots_log2) with the per-slice pair table sized to the rate.
    """
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 0xBA7C])))
    out = []
    for i in range(n_links):
        rate = int(math.exp(rng.uniform(math.log(1e4), math.log(5e6))))
        k = int(round(math.exp(rng.uniform(math.log(16), math.log(300)))))
        one_byte = k <= 255 and rng.random() < 0.5
        cells = 1 << int(np.clip(round(math.log2(rate)), 16, 22))
        gl = 256
        traffic = TrafficSpec(
            seed=1000 + i, pkts_per_slice=rate, n_src=int(np.clip(rate // 5, 1 << 10, 1 << 20)), zipf_s=1.2,
            dst_model="pool", pool_alpha=1.5, pool_max=128,
            n_planted=max(1, rate // 20000), planted_card=(1 << 10, 1 << 16), planted_card_dist="loguniform",
            planted_spread=k, churn_frac=0.3, churn_run=(max(4, k // 4), k))
        w = Workload(
            name=f"link{i}-r{rate}-k{k}", u=8, v=cells // gl, g=128, gl=gl, dr_bytes=1 if one_byte else 2,
            z=8 if one_byte else 16, k=k, theta=1024, n_slices=16, traffic=traffic, hash_seed=100 + i,
            max_sampled=1 << int(np.clip(math.ceil(math.log2(max(rate, 1) / 4)), 12, 20)),
            max_candidates=1 << 14)
        out.append((w, int(np.clip(round(math.log2(rate / 2)), 12, 21))))
    return out


def served_links(n_links: int = 256, seed: int = 5):
    """Link identities of the serving workload: like batched_links, with Zipf(1.1) sources and
    1 to 50 planted super points per link.  Returns a list of (Workload, pair_slots_log2)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 0x5E7F])))
    out = []
    for i, (w, plog) in enumerate(batched_links(n_links, seed)):
        t = dataclasses.replace(w.traffic, seed=5000 + i, zipf_s=1.1, n_planted=int(rng.integers(1, 51)))
        out.append((dataclasses.replace(w, name=f"served-{w.name}", traffic=t, hash_seed=700 + i), plog))
    return out
