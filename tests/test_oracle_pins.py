"""Pins of the CPU oracle to facts fixed by the paper and by mathematics (no GPU).

Each check is independent of the oracle's own code: worked examples printed in the paper,
closed forms, special cases that reduce to a textbook formula, and the probability laws of
Lemma 1 / Theorem 1 / Eq. 2-5 checked by Monte Carlo.
"""
import math
import os
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ----------------------------------------------------------------------- LSB -------

def test_lsb_worked_examples():
    """Section 3.2 prints LSB(3) = 0 and LSB(40) = 3."""
    for val, want in _golden("lsb_examples.txt"):
        assert oracle.lsb(int(val)) == int(want)


def test_lsb_powers_and_odd_multiples():
    # LSB(m * 2^j) = j for every odd m; LSB(0) is taken as 32 (no 1 bit).
    rng = np.random.default_rng(5)
    for j in range(32):
        for m in rng.integers(0, 1 << 16, size=8) * 2 + 1:
            x = (int(m) << j) & 0xFFFFFFFF
            if x:
                assert oracle.lsb(x) == j
    assert oracle.lsb(0) == 32


# ------------------------------------------------------------------- tau, rho -------

def test_tau_closed_form():
    """Eq. 1: tau = ceil(log2(theta/g)) is the least n >= 0 with g * 2^n >= theta."""
    for g in (1, 2, 8, 64, 128, 1024):
        for theta in list(range(1, 5000, 7)) + [1 << 20, (1 << 20) + 1, (1 << 31) - 1]:
            n = 0
            while g * (1 << n) < theta:
                n += 1
            assert oracle.tau(theta, g) == n, (theta, g)


def test_tau_paper_values():
    p = {k: int(v) for k, v in _golden("paper_parameters.txt")}
    # theta = 1024 with the paper's g = 8 gives tau = 7 (sampling rate 1/128).
    assert oracle.tau(p["theta"], p["g"]) == 7
    assert oracle.tau(1024, 64) == 4 and oracle.tau(1024, 128) == 3


def test_rho_against_series():
    """rho = 0.99 (1 - e^{-1/3}) checked against an independent 50-digit series for e^{-1/3}."""
    getcontext().prec = 60
    x = Decimal(-1) / Decimal(3)
    term, total = Decimal(1), Decimal(1)
    for n in range(1, 80):
        term = term * x / n
        total += term
    rho = Decimal("0.99") * (1 - total)
    assert abs(Decimal(repr(oracle.rho())) - rho) < Decimal("1e-15")
    for g in (8, 64, 128, 256, 1000):
        want = math.ceil(Fraction(str(rho)) * g)  # rho*g is never an integer for these g
        assert oracle.rho_g(g) == want
    assert (oracle.rho_g(8), oracle.rho_g(64), oracle.rho_g(128)) == (3, 18, 36)


# ------------------------------------------------------------------ hash family -----

def test_hash_special_cases():
    p = synth.MERSENNE_61
    M = 0xFFFFFFFF
    assert oracle.hash_ab(1, 0, 12345) == 12345                 # identity member
    assert oracle.hash_ab(7, 99, 0) == 99                       # h(0) = b
    assert oracle.hash_ab(p - 1, 0, 1) == (p - 1) & M           # -1 mod p
    assert oracle.hash_ab(p - 1, 1, 1) == 0                     # (p - 1 + 1) mod p = 0
    assert oracle.hash_ab(1 << 60, 0, 4) == 2                   # 2^62 = 2 (mod 2^61 - 1)
    assert oracle.hash_ab(1 << 60, p - 2, 4) == 0               # 2 + p - 2 = p = 0
    assert oracle.hash_ab((1 << 32) + 3, 0, 1 << 31) == ((1 << 63) + 3 * (1 << 31)) % p & M


def test_hash_low_bits_uniform():
    """Low bits of random members are close to uniform (chi-square over 64 cells)."""
    from scipy.stats import chi2

    a, b = synth.hash_coefficients(77, 8)
    x = np.arange(20000, dtype=np.uint32) * np.uint32(2654435761)
    o = oracle.Oracle(4, 64, 8, 8, 1, 1, 1, a, b)
    for role in range(7):
        h = o.hash(role, x) & 63
        cnt = np.bincount(h, minlength=64)
        e = x.size / 64
        stat = ((cnt - e) ** 2 / e).sum()
        assert stat < chi2.ppf(0.9999, 63)
    o.close()


# ------------------------------------------------------------------ Eq. 6 / Eq. 9 ----

def test_eq9_reduces_to_linear_counting_when_no_noise():
    """With UP = 0, Eq. 9 is Whang's linear counting, Eq. 6: -g' ln((g' - w)/g')."""
    for gl in (64, 256, 1024):
        for w in range(1, gl):
            est, f = oracle.estimate(gl, 0.0, w)
            assert f == 0
            assert est == pytest.approx(-gl * math.log((gl - w) / gl), rel=1e-12)


def test_eq9_removes_the_modelled_noise():
    """Section 4.2 models |ULE| = d1 + (g' - d1) UP with d1 = g' - g' e^{-n/g'}; Eq. 9 of that
    expected count must return n exactly (up to rounding)."""
    for gl in (64, 256, 1024, 8192):
        for up in (1e-6, 0.01, 0.137, 0.5, 0.9):
            for n in (1, 10, 100, 1000, 5000):
                if n > 8 * gl:
                    continue  # e^{-n/g'} vanishes next to 1: the count is saturated
                d1 = gl - gl * math.exp(-n / gl)
                w = d1 + (gl - d1) * up
                est, f = oracle.estimate(gl, up, w)
                assert f == 0
                assert est == pytest.approx(n, rel=1e-7)


def test_eq9_edges():
    est, f = oracle.estimate(256, 0.1, 256)
    assert math.isinf(est) and f == oracle.SATURATED
    est, f = oracle.estimate(256, 1.0, 17)
    assert math.isinf(est) and f == oracle.SATURATED
    est, f = oracle.estimate(256, 0.25, 64)       # w = g' UP exactly: no signal left
    assert est == 0.0 and f == 0
    est, f = oracle.estimate(256, 0.25, 10)       # below the noise floor
    assert est == 0.0 and f == 0
    # monotone in w above the noise floor
    prev = 0.0
    for w in range(65, 256):
        est, _ = oracle.estimate(256, 0.25, w)
        assert est > prev
        prev = est


# --------------------------------------------------------- Lemma 1 / Theorem 1 -------

def _fn(alpha, g, memo):
    """Lemma 1: FN(alpha, g) = g^alpha - sum_{i<g} C(g, i) FN(alpha, i), FN(alpha, 1) = 1."""
    if (alpha, g) in memo:
        return memo[(alpha, g)]
    if g == 1:
        r = 1
    else:
        r = g ** alpha - sum(math.comb(g, i) * _fn(alpha, i, memo) for i in range(1, g))
    memo[(alpha, g)] = r
    return r


def _pr_fill(n, g, tau, g1, memo):
    """Eq. 4: probability that g1 of the g SRE recorders are set by n distinct hosts."""
    q = Fraction(1, 2 ** tau)
    tot = Fraction(0)
    for alpha in range(g1, n + 1):
        pa = math.comb(n, alpha) * q ** alpha * (1 - q) ** (n - alpha)            # Eq. 3
        pg = Fraction(math.comb(g, g1) * _fn(alpha, g1, memo), g ** alpha)        # Eq. 2, Thm 1
        tot += pa * pg
    return tot


def test_lemma1_matches_surjection_count():
    # FN(alpha, g) counts surjections: it must also equal the inclusion-exclusion sum.
    memo = {}
    for g in range(1, 9):
        for alpha in range(0, 12):
            ie = sum((-1) ** j * math.comb(g, j) * (g - j) ** alpha for j in range(g + 1))
            if alpha == 0:
                continue
            assert _fn(alpha, g, memo) == ie


@pytest.mark.parametrize("n,tau", [(12, 0), (60, 2)])
def test_sre_fill_distribution_monte_carlo(n, tau):
    """One host, one estimator (u = v = 1), g = 16: the oracle's SRE weight after n distinct
    opposite hosts follows Eq. 4 (chi-square test over many random hash draws)."""
    from scipy.stats import chi2

    g = 16
    theta = g << tau
    memo = {}
    probs = np.array([float(_pr_fill(n, g, tau, g1, memo)) for g1 in range(g + 1)])
    assert abs(probs.sum() - 1) < 1e-9
    trials = 3000
    rng = np.random.default_rng(1234 + n)
    hist = np.zeros(g + 1, np.int64)
    for t in range(trials):
        a, b = synth.hash_coefficients(10_000 + t, 4)
        o = oracle.Oracle(1, 1, g, 16, 1, 1, theta, a, b)
        bips = rng.choice(1 << 32, size=n, replace=False).astype(np.uint32)
        pairs = np.stack([np.full(n, 0x0A000001, np.uint32), bips], axis=1)
        o.push(pairs)
        hist[o.ure_count(0x0A000001)] += 1
        o.close()
    exp = probs * trials
    keep = exp >= 5
    obs = np.append(hist[keep], hist[~keep].sum())
    ex = np.append(exp[keep], exp[~keep].sum())
    if ex[-1] < 1e-9:
        obs, ex = obs[:-1], ex[:-1]
    stat = ((obs - ex) ** 2 / ex).sum()
    assert stat < chi2.ppf(0.9999, len(ex) - 1), (stat, obs, ex)


def test_linear_counting_unbiased_monte_carlo():
    """u = v = 1, one host with n distinct opposite hosts: mean of Eq. 6 estimates is n within
    the standard error of Whang's variance g'(e^t - t - 1), t = n / g'."""
    gl, n, trials = 256, 300, 600
    rng = np.random.default_rng(99)
    ests = []
    for t in range(trials):
        a, b = synth.hash_coefficients(50_000 + t, 4)
        o = oracle.Oracle(1, 1, 8, gl, 1, 1, 1, a, b)
        bips = rng.choice(1 << 32, size=n, replace=False).astype(np.uint32)
        o.push(np.stack([np.full(n, 7, np.uint32), bips], axis=1))
        w = o.ule_count(7)
        ests.append(oracle.estimate(gl, 0.0, w)[0])
        o.close()
    tt = n / gl
    sd = math.sqrt(gl * (math.exp(tt) - tt - 1))
    bias = (math.exp(tt) - tt - 1) / 2
    assert abs(np.mean(ests) - n - bias) < 5 * sd / math.sqrt(trials)
