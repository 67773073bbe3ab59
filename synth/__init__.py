"""Seeded synthetic fields shaped like the paper's workloads (Table II).

This module holds no dual-quantization arithmetic: it only draws inputs.  The
oracle tests, the CUDA parity tests and the benchmark all take their inputs
from here, so that both sides of every comparison see the same arrays.
"""
from .fields import (  # noqa: F401
    fourier2d, grf3d, lognormal3d, random_walk1d, tuner_field, cfg1_field,
    cfg2_field, cfg3_fields, cfg5_fields, adversarial_values,
)
