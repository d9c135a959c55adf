"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This package holds the system models of the paper's illustrations (state
dimension, grid bounds, prior, F, Q, R, measurement functions), seeded
trajectory simulation (Sec. 1, Eqs. asx/asz) and seeded random test inputs.
It contains none of the filter's arithmetic: no grid, transition, update,
rounding or moment computation.
"""
from .workloads import (Model, config1, config1_linear, config2, config3, config4, radar, range3,
                        random_index_bumps_tt, simulate)

__all__ = ["Model", "config1", "config1_linear", "config2", "config3", "config4", "radar", "range3",
           "random_index_bumps_tt", "simulate"]
