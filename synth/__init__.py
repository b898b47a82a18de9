"""Seeded synthetic lidar scans for the G-VOM map update.

This module generates INPUTS only: terrain scenes, vehicle trajectories, and
the lidar returns a spinning sensor would report. It holds none of the
mapping method's arithmetic (no voxel binning, traversal, origin choice or 2D
products), and both the CUDA path and the CPU oracle consume what it makes.

The paper's recordings (Ouster OS1-64/128 on the RELLIS campus) are not
available, so scenes stand in for them with the same structure: organised
beam-major scans (row = beam, column = azimuth), zero points where a beam
returned nothing, ground with slopes and undulations, box obstacles,
ditches, and vegetation that some rays pass through.
"""
from .scenes import (  # noqa: F401
    LidarSpec,
    MapSpec,
    Scan,
    Scene,
    single_scan,
    sequence_config,
    sequence_scans,
    batched_scans,
    served_stream,
    WORKLOADS,
    SEED_BASE,
    SEEDS,
)
