"""Seeded synthetic inputs for the multicontinuum workloads.

This package only draws coefficient fields, sources and initial states from
seeded random generators. It holds none of the method's arithmetic (no
transmissibilities, no exchange scaling, no time stepping): the FP64 oracle and
the CUDA path each apply the finite-volume discretisation of Section 3.1 to
these raw fields on their own.

The paper's own workload (25 fracture lines, Fig. 1, Section 5) exists only as
a figure, so the workloads here are synthetic stand-ins with the shapes,
contrasts and source structure of the paper's 2C/3C problems (`paper_wells`
also takes the paper's initial state, time span and well parameters).
"""

from .fields import correlated_lognormal, segment_lengths, random_segments
from .configs import (Workload, dual_64, triple_1024, precision_4096,
                      fracture_instance, batched_instances, nlmc_1024, paper_wells, scaled,
                      by_name, Fracture1D, fracture1d, fracture1d_sources)

__all__ = [
    "correlated_lognormal", "segment_lengths", "random_segments", "Workload",
    "dual_64", "triple_1024", "precision_4096", "fracture_instance", "batched_instances",
    "nlmc_1024", "paper_wells", "scaled", "by_name", "Fracture1D", "fracture1d",
    "fracture1d_sources",
]
