"""FP64 CPU oracle of the fully-coupled DG/CZM + lubrication Newton step.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline legs of bench.py, never by the product path.  Shares no code with
the CUDA library.
"""
from .fem import Oracle, Params, simplex_rule, p2_values, p2_dlam, face_local_nodes, lame
