"""Seeded synthetic inputs for the radiation transport solve.

This package only synthesises inputs (opacity chi, source function S, boundary
arrays, loss targets). It holds none of the solver's arithmetic, so both the
CPU oracle and the CUDA path can be fed from it without sharing method code.
"""
from .atmosphere import (  # noqa: F401
    stratified_atmosphere,
    band_stack,
    WORKLOADS,
    workload,
    batched_subdomain_shapes,
    batched_bands,
)
