"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and the
benchmark: counter-based random numbers, quenched U(1) gauge fields, Gaussian
right-hand sides and the workload table.

This package holds none of the solver's arithmetic.  The gauge generator is a
plain Metropolis sampler of the compact plaquette action of Sec. 2 (Eq. 2.3);
it only produces inputs.
"""
from .rng import rng_u64, uniform01, cgauss
from .gauge import metropolis_u1, unit_gauge, random_gauge_transform
from .workloads import WORKLOADS, workload, rhs_batch

__all__ = [
    "rng_u64", "uniform01", "cgauss", "metropolis_u1", "unit_gauge",
    "random_gauge_transform", "WORKLOADS", "workload", "rhs_batch",
]
