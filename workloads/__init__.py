"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This package holds input generation and the request format only: no part of the
absorption method's arithmetic lives here.
"""
from .synth import (  # noqa: F401
    LINE_DTYPE,
    SPECIES_DTYPE,
    Workload,
    config0_tiny,
    config1_venus,
    config2_batch,
    config3_earth,
    make_lines,
    tiny_workload,
    venus_profile,
)
