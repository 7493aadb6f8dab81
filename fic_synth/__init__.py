"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds image and arrival-stream generators only; it contains none of
the encoder's arithmetic, so the CPU oracle and the CUDA path stay independent.
"""
from .images import (  # noqa: F401
    one_over_f,
    with_step_edges,
    workload_image,
    batch_images,
    poisson_requests,
    WORKLOADS,
)
