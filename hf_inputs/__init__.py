"""Seeded synthetic inputs (meshes, parameters, seed states) shared by the
oracle, the tests and the bench.  Holds none of the method's arithmetic."""
from .mesh import (Mesh, square_p2, cube_p2, pressure_nodes, seed_faces, seed_state,
                   batch_instances, round_even, far_field_load, split_triangles, TRI_EDGES, TET_EDGES)
from .workloads import (Workload, kgd_2d, penny_3d, c1_kgd_toughness, c2_kgd_viscosity, c3_penny,
                        sample_parameters, sweep_instances, serving_requests, toughness_consistent,
                        balanced_fluid_length)
