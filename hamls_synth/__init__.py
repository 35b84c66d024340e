"""Seeded synthetic inputs for HAMLS on the sphere.

This package produces node sets, field coefficients and sampled values. It is
shared by the tests, the benchmark and the oracle's callers, and it holds none
of the HAMLS arithmetic itself (no support radius, no local least squares, no
quadrature): only random numbers, sampling geometry and the evaluation of the
synthetic ground-truth field.
"""
from .gen import (  # noqa: F401
    SplitMix64,
    uniform_sphere,
    remove_caps,
    track_hole_nodes,
    uniform_minus_cap_nodes,
    bump_field,
    random_field_coeffs,
    synth_field,
    workload,
    WORKLOADS,
    FitSpec,
    batch_specs,
    serving_trace,
    fit_workload,
)
