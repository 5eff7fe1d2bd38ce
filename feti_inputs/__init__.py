"""Seeded synthetic inputs for the FETI solvers: meshes, partitions, boundary data.

This package describes problems; it computes nothing of the method itself
(no element integrals, no loads, no operators).  Both the CPU oracle and the
GPU library read the same problem description produced here.

Workloads follow the shapes of the paper's test problems: a structured unit
cube cut into sub-cubes (Sec. 5.1) and a thick-walled tube under internal
pressure standing in for the artery segments of Sec. 5.2 (Table 1 material).
"""
from .mesh import (Problem, cube_problem, cylinder_problem, config_problem,
                   jittered_cylinder_problem, kelvin_cube_problem, kelvin_displacement)

__all__ = ["Problem", "cube_problem", "cylinder_problem", "config_problem",
           "jittered_cylinder_problem", "kelvin_cube_problem", "kelvin_displacement"]
