"""Seeded synthetic IP-pair traces.

A packet is a pair ``(aip, bip)`` of IPv4 addresses held as uint32 values in host order
(Section 3.2, definition of an IP pair): ``aip`` is the host of the monitored network A
whose cardinality is estimated, ``bip`` its opposite host in network B.  A slice is an
``(n, 2)`` array of such pairs, interleaved ``aip, bip`` in memory (8 bytes per packet).

The traffic model stands in for the CERNET traces of Section 5, which are not available:

* background sources follow a Zipf law over ``n_src`` addresses;
* their destinations are either uniform over ``dst_space`` addresses ("uniform") or drawn
  from a fixed per-source pool whose size has a truncated Pareto tail ("pool", a flow model:
  most hosts talk to a handful of peers);
* ``n_planted`` super points contact fresh, never repeated destinations, evenly spread so
  that ``planted_spread`` consecutive slices hold ``card`` distinct destinations; a share of
  them switch on and off (churn);
* optional adversarial parts: one heavy source sending a share of all packets to random
  destinations, and a flood of spoofed one-packet sources;
* optional flow bursts: each background pair sends a geometric number of packets (mean
  ``burst_mean``) back to back, so that consecutive packets repeat the same pair.

Every slice is generated from ``(seed, slice index)`` alone, so any slice can be rebuilt on
its own, on the CPU or on a CUDA device (the two devices draw different streams; tests make
one copy and hand the same bytes to both the oracle and the CUDA path).
"""
from __future__ import annotations

import dataclasses
import functools
import math

import numpy as np
import torch

MERSENNE_61 = (1 << 61) - 1
_M32 = 0xFFFFFFFF

# Salts that keep the address populations apart.
_SALT_A = 0x2545F491      # A-side (source) address population
_SALT_POOL = 0x68E31DA4   # per-source pool size draw
_SALT_DST = 0x1B56C4E9    # per-source pool base
_SALT_UNI = 0x7F4A7C15    # uniform destination population
_SALT_PLANT = 0x3C6EF372  # planted-host destination base


def hash_coefficients(seed: int, n_roles: int) -> tuple[np.ndarray, np.ndarray]:
    """Draw ``n_roles`` members ``h(x) = (a*x + b) mod (2^61 - 1)`` of the polynomial family.

    Returns ``(a, b)`` as uint64 arrays with ``a`` in ``[1, p-1]`` and ``b`` in ``[0, p-1]``.
    The estimator draws its hash functions at random (Section 3.2 cites a min-wise independent
    family); the draw is made here and passed in, so that both sides use the same functions.
    """
    ss = np.random.SeedSequence([int(seed) & ((1 << 63) - 1), 0x5EED0001])
    rng = np.random.Generator(np.random.PCG64(ss))
    a = rng.integers(1, MERSENNE_61, size=n_roles, dtype=np.uint64)
    b = rng.integers(0, MERSENNE_61, size=n_roles, dtype=np.uint64)
    return a, b


def _fmix32(h: torch.Tensor) -> torch.Tensor:
    """A bijective 32-bit mixer (MurmurHash3 finaliser) on int64 tensors holding uint32 values."""
    h = h & _M32
    h = h ^ (h >> 16)
    h = (h * 0x85EBCA6B) & _M32
    h = h ^ (h >> 13)
    h = (h * 0xC2B2AE35) & _M32
    h = h ^ (h >> 16)
    return h


def _to_i32(x: torch.Tensor) -> torch.Tensor:
    """int64 holding uint32 values -> int32 with the same bit pattern."""
    x = x & _M32
    return torch.where(x >= (1 << 31), x - (1 << 32), x).to(torch.int32)


@dataclasses.dataclass(frozen=True)
class TrafficSpec:
    seed: int
    pkts_per_slice: int
    n_src: int
    zipf_s: float
    dst_model: str = "uniform"          # "uniform" | "pool"
    dst_space: int = 1 << 20
    pool_alpha: float = 1.5
    pool_max: int = 128
    n_planted: int = 0
    planted_card: tuple = (500, 3000)
    planted_card_dist: str = "uniform"  # "uniform" | "loguniform"
    planted_spread: int = 16
    churn_frac: float = 0.0
    churn_run: tuple = (75, 300)        # on/off run lengths (slices) of churning hosts
    heavy_frac: float = 0.0
    flood_sources: int = 0
    flood_slices: tuple = (0, 0)        # [first, last) slice of the spoofed flood
    burst_mean: float = 0.0             # > 0: background pairs in back-to-back bursts of this mean


@functools.lru_cache(maxsize=8)
def _zipf_cdf_cpu(n: int, s: float) -> torch.Tensor:
    w = torch.arange(1, n + 1, dtype=torch.float64).pow(-s)
    c = torch.cumsum(w, 0)
    return c / c[-1]


def _zipf_cdf(n: int, s: float, device) -> torch.Tensor:
    return _zipf_cdf_cpu(n, s).to(device)


@functools.lru_cache(maxsize=16)
def _planted_params(spec: TrafficSpec):
    """Per planted host: address index, cardinality, churn (on, off, phase). Slice independent."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([spec.seed, 0xB1A5])))
    n = spec.n_planted
    lo, hi = spec.planted_card
    if spec.planted_card_dist == "loguniform":
        card = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))
    else:
        card = rng.uniform(lo, hi, size=n)
    card = np.floor(card).astype(np.int64)
    churn = rng.random(n) < spec.churn_frac
    r0, r1 = spec.churn_run
    on = rng.integers(r0, r1 + 1, size=n)
    off = rng.integers(r0, r1 + 1, size=n)
    phase = rng.integers(0, 1 << 30, size=n)
    return card, churn, on, off, phase


def planted_hosts(spec: TrafficSpec):
    """Addresses (uint32 numpy) and total cardinalities of the planted hosts.

    A planted host contacts ``card`` fresh destinations over every ``planted_spread``
    consecutive slices in which it is active.
    """
    card, churn, on, off, phase = _planted_params(spec)
    h = torch.arange(spec.n_planted, dtype=torch.int64)
    addr = _fmix32(h + spec.n_src + _SALT_A).numpy().astype(np.uint32)
    return addr, card.copy(), churn.copy()


def _planted_packets(spec: TrafficSpec, s: int, device):
    if spec.n_planted == 0:
        z = torch.zeros(0, dtype=torch.int64, device=device)
        return z, z
    card, churn, on, off, phase = _planted_params(spec)
    S = spec.planted_spread
    first = (s * card) // S
    last = ((s + 1) * card) // S
    cnt = last - first
    active = ~churn | (((s + phase) % (on + off)) < on)
    cnt = np.where(active, cnt, 0)
    hosts = np.repeat(np.arange(spec.n_planted, dtype=np.int64), cnt)
    if hosts.size == 0:
        z = torch.zeros(0, dtype=torch.int64, device=device)
        return z, z
    starts = np.repeat(first, cnt)
    offs = np.arange(hosts.size, dtype=np.int64) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    j = torch.from_numpy(starts + offs).to(device)
    h = torch.from_numpy(hosts).to(device)
    aip = _fmix32(h + spec.n_src + _SALT_A)
    base = _fmix32(h + _SALT_PLANT)
    bip = _fmix32(base + j)
    return aip, bip


def generate_slice(spec: TrafficSpec, s: int, device="cpu") -> torch.Tensor:
    """Packets of slice ``s`` as an ``(n, 2)`` int32 tensor holding uint32 bit patterns."""
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed((spec.seed * 1000003 + s * 7919 + 12345) & ((1 << 62) - 1))
    n = spec.pkts_per_slice

    p_aip, p_bip = _planted_packets(spec, s, dev)

    n_heavy = int(round(spec.heavy_frac * n))
    h_aip = torch.full((n_heavy,), 0, dtype=torch.int64, device=dev)
    h_aip = _fmix32(h_aip + spec.n_src + spec.n_planted + _SALT_A)
    h_bip = torch.randint(0, 1 << 32, (n_heavy,), generator=gen, device=dev, dtype=torch.int64)

    f0, f1 = spec.flood_slices
    if spec.flood_sources and f0 <= s < f1:
        span = f1 - f0
        a = ((s - f0) * spec.flood_sources) // span
        b = ((s - f0 + 1) * spec.flood_sources) // span
        j = torch.arange(a, b, dtype=torch.int64, device=dev)
        f_aip = _fmix32(j + spec.n_src + spec.n_planted + 1 + _SALT_A)
        f_bip = torch.randint(0, 1 << 32, (b - a,), generator=gen, device=dev, dtype=torch.int64)
    else:
        f_aip = torch.zeros(0, dtype=torch.int64, device=dev)
        f_bip = f_aip

    n_bg = max(0, n - p_aip.numel() - n_heavy - f_aip.numel())
    burst = None
    if spec.burst_mean > 0 and n_bg > 0:
        # packets per background flow ~ Geometric(1/mean) >= 1, drawn until they cover n_bg
        m = int(math.ceil(n_bg / spec.burst_mean * 1.25)) + 64
        burst = torch.empty(m, device=dev, dtype=torch.float64).geometric_(1.0 / spec.burst_mean, generator=gen)
        burst = burst.to(torch.int64)
        ends = torch.cumsum(burst, 0)
        f = int(torch.searchsorted(ends, torch.tensor([n_bg], device=dev, dtype=torch.int64)).item()) + 1
        if f > m:
            raise ValueError("burst draw did not cover the slice")
        burst = burst[:f].clone()
        burst[-1] -= int(ends[f - 1].item()) - n_bg
        n_bg = f
    u = torch.rand(n_bg, generator=gen, device=dev, dtype=torch.float64)
    rank = torch.searchsorted(_zipf_cdf(spec.n_src, spec.zipf_s, dev), u, right=True)
    rank = rank.clamp_(max=spec.n_src - 1).to(torch.int64)
    bg_aip = _fmix32(rank + _SALT_A)
    if spec.dst_model == "pool":
        um = (_fmix32(rank ^ _SALT_POOL).to(torch.float64) + 0.5) / 4294967296.0
        m = torch.floor(um.pow(-1.0 / spec.pool_alpha)).clamp_(1, spec.pool_max)
        idx = torch.floor(torch.rand(n_bg, generator=gen, device=dev, dtype=torch.float64) * m)
        bg_bip = _fmix32(_fmix32(rank + _SALT_DST) + idx.to(torch.int64))
    elif spec.dst_model == "uniform":
        d = torch.randint(0, spec.dst_space, (n_bg,), generator=gen, device=dev, dtype=torch.int64)
        bg_bip = _fmix32(d + _SALT_UNI)
    else:
        raise ValueError(f"unknown dst_model {spec.dst_model!r}")

    aip = torch.cat([bg_aip, p_aip, h_aip, f_aip])
    bip = torch.cat([bg_bip, p_bip, h_bip, f_bip])
    perm = torch.randperm(aip.numel(), generator=gen, device=dev)
    if burst is not None:  # shuffle whole bursts, then expand each into its packets
        reps = torch.cat([burst, torch.ones(aip.numel() - n_bg, dtype=torch.int64, device=dev)])[perm]
        aip = torch.repeat_interleave(aip[perm], reps)
        bip = torch.repeat_interleave(bip[perm], reps)
        return torch.stack([_to_i32(aip), _to_i32(bip)], dim=1).contiguous()
    return torch.stack([_to_i32(aip[perm]), _to_i32(bip[perm])], dim=1).contiguous()


def generate_trace(spec: TrafficSpec, n_slices: int, device="cpu", first: int = 0):
    return [generate_slice(spec, s, device) for s in range(first, first + n_slices)]


def pairs_to_numpy(t: torch.Tensor) -> np.ndarray:
    """(n, 2) int32 tensor -> contiguous (n, 2) uint32 numpy array (same bytes)."""
    return np.ascontiguousarray(t.detach().cpu().numpy()).view(np.uint32)


def random_pairs(seed: int, n: int, n_src: int, n_dst: int) -> np.ndarray:
    """Small uniform trace over tiny address sets (dense duplicates and collisions)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 0xD1CE])))
    a = rng.integers(0, n_src, size=n, dtype=np.uint64)
    b = rng.integers(0, n_dst, size=n, dtype=np.uint64)
    # spread the small ids over the 32-bit space with a fixed odd multiplier (bijective)
    a = (a * np.uint64(0x9E3779B1) + np.uint64(17)) & np.uint64(_M32)
    b = (b * np.uint64(0x85EBCA77) + np.uint64(5)) & np.uint64(_M32)
    return np.stack([a, b], axis=1).astype(np.uint32)
