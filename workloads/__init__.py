"""Seeded synthetic inputs for the TreeRay/OnTheSpot hot path.

This package only draws random numbers and lays them out as arrays: density
fields, point-source lists and the named workload configurations.  It holds
none of the method's arithmetic (no netting, no tree, no rays), so both the
CPU oracle and the CUDA path can take their inputs from here without sharing
any of the computation they are compared on.
"""
from .fields import (PC_CM, ALPHA_B, HNU_EUV, Workload, uniform_density,
                     lognormal_density, uniform_sources, powerlaw_sources,
                     workload, WORKLOADS)

__all__ = ["PC_CM", "ALPHA_B", "HNU_EUV", "Workload", "uniform_density",
           "lognormal_density", "uniform_sources", "powerlaw_sources",
           "workload", "WORKLOADS"]
