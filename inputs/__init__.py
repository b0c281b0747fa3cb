"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds only input generation (permeability fields, boundary
data, sources).  It contains none of the method's arithmetic, so the oracle
and the CUDA path can both draw their inputs from it without sharing any
part of the computation.
"""
from .fields import (gaussian_random_field, lognormal_permeability, gaussian_random_field_3d,
                     lognormal_permeability_3d)
from .problems import (Problem, darcy_problem, config_64, config_1024,
                       config_4096, ensemble_member, NEUMANN, DIRICHLET, Problem3D,
                       darcy_problem_3d, config_3d)

__all__ = ["gaussian_random_field", "lognormal_permeability", "Problem",
           "darcy_problem", "config_64", "config_1024", "config_4096", "ensemble_member",
           "NEUMANN", "DIRICHLET", "gaussian_random_field_3d", "lognormal_permeability_3d",
           "Problem3D", "darcy_problem_3d", "config_3d"]
