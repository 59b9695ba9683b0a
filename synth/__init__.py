"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This package holds input generation only: brain-shaped material maps, the tumor seed, the
parameter sets of the benchmark workloads and seeded random draws.  It contains none of the
time-step arithmetic (no operators, solvers, interpolation or reaction terms), so both the
oracle and the GPU path can consume its output without sharing any of the method.
"""
from .brain import synthetic_brain, initial_state, initial_state_single, grf_terms, evaluate_grf
from .params import table_setup_params, workload_params, batch_workload, WORKLOADS

__all__ = [
    "synthetic_brain",
    "initial_state",
    "initial_state_single",
    "grf_terms",
    "evaluate_grf",
    "table_setup_params",
    "workload_params",
    "WORKLOADS",
    "batch_workload",
]
