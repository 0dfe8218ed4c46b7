"""Seeded synthetic workloads for the SIMP/OC hot path.

This package only builds problem *inputs* (grid sizes, clamped-dof masks, load
vectors, passive-element masks, random vectors).  It contains none of the
method's arithmetic, so both the CPU oracle's tests and the CUDA path's tests
and benchmark can draw the same inputs from it.
"""
from .problems import (  # noqa: F401
    Problem, cantilever, config_small, config_void_cylinder, config_large,
    config_paper_benchmark, config_batched, random_density, random_vector,
    node_count, element_count,
)
