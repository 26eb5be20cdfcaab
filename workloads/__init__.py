"""Seeded synthetic inputs for the spectrum-reweighting likelihood.

This package builds the inputs that both the CUDA library and the FP64 oracle
consume: recoil and reconstructed binnings, solar-neutrino energy nodes with
their weights and survival probabilities, the detector response matrix R,
background templates, parameter points theta, and the stored pseudo-data
counts.  It contains none of the method's arithmetic (no cross sections, no
folding, no likelihood): every array here is an *input* to the method.

Shapes follow the solar workloads the method is applied to (Sec. II-III of the
paper: pp / 7Be / pep / CNO / 8B components, a few-thousand-bin recoil grid, a
Gaussian-resolution response with quenching, beta-like background templates).
"""

from .solar import (  # noqa: F401
    THETA_NAMES,
    WORKLOADS,
    be7_line_workload,
    solar_set_workload,
    batched_scan_workload,
    uneven_groups_workload,
    uneven_group_inputs,
    group_counts_path,
    load_group_counts,
    theta_box,
    fit_region_points,
    box_sample,
    poisson_counts,
    load_counts,
    counts_path,
)
from .joint import (  # noqa: F401
    solar_components,
    solar_joint_workload,
    joint_workload,
    live_time,
    mc_histogram,
    scale_factor,
)
