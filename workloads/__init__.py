"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds problem data only (mesh maps, media, initial states,
source and receiver placements, the five workload descriptions) and none of
the method's arithmetic: no derivative operators, metrics, fluxes, penalties,
time stepping or energy.  Every generator is a closed-form function of node
coordinates and a seed, written against an array module ``xp`` (numpy or
torch), so that either side can evaluate it at any subset of nodes.
"""
from .configs import CONFIGS, WorkloadConfig, config_by_name  # noqa: F401
