"""Seeded synthetic rock-like images and partitions.

This package holds the input generators shared by the tests, the benchmark and
the examples. It contains none of the homogenization arithmetic: it only draws
seeded random numbers and turns them into uint8 phase maps, phase-moduli tables
and subimage box lists. Both the CUDA path and the CPU oracle receive what it
produces as plain arrays.
"""

from .images import (  # noqa: F401
    splitmix64,
    uniform01,
    normal01,
    gaussian_random_field,
    threshold_bands,
    grf_two_phase,
    grf_three_phase,
    boolean_spheres,
    multiscale_carbonate,
    uneven_partition,
    uniform_partition,
    laminate,
    image_sha256,
    PHASES_QUARTZ_PORE_PAPER,
    PHASES_APPENDIX_B,
    PHASES_SOLID_PORE,
    PHASES_SOLID_CLAY_PORE,
    PHASES_CARBONATE,
    workload,
)
