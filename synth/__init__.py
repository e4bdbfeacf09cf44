"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the CPU oracle.

This package only draws random numbers and lays them out as IP-pair packets or as hash
coefficients.  It holds none of the estimator's arithmetic (no hashing into sketches, no
distance recorders, no estimates), so that the oracle and the CUDA path stay independent.
"""
from .traces import (  # noqa: F401
    MERSENNE_61,
    TrafficSpec,
    generate_slice,
    generate_trace,
    hash_coefficients,
    pairs_to_numpy,
    planted_hosts,
    random_pairs,
)
from .workloads import WORKLOADS, Workload, batched_links, served_links, workload  # noqa: F401
