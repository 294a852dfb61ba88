"""FP64 CPU oracle of the ReaxFF timestep -- test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference legs use it.
"""
from oracle.reaxff_oracle import (TERMS, Model, blocks_of, build_lists, far_list_bruteforce,  # noqa: F401
                                  far_list_cells, free_flight, gmres, half_mask, kinetic, pcg, pcg_block, sort_key, taper, verlet)
