"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

Nothing here computes any part of the ReaxFF method: only types, positions,
velocities, boxes and parameter tables.
"""
from synth.crystal import (ACC_CONV, CELL, KB, MASS, TYPE_NAMES, crystal, random_cluster,  # noqa: F401
                           unit_cell, velocities)
from synth.params import make_params  # noqa: F401
from synth.workloads import OPTIONS_DEFAULT, fixed_charges, workload  # noqa: F401
