"""Seeded synthetic inputs of the tests: re-exported from the package's
workload module, which holds none of the generators' arithmetic."""
from paper_1003_1898_gb300.workloads import *  # noqa: F401,F403
from paper_1003_1898_gb300.workloads import (GENS, JUMP, JUMP_X0, LUX_SWEEP, LUXURY_LEVELS, PLANAR_LEVELS,  # noqa: F401
                                             ROOFLINE, ROOFLINE_MT, SEED_BASE, SMALL,
                                             batched_requests, jump_offsets, request_split,
                                             sample_rows)
