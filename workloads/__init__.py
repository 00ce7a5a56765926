"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds geometry and random input generation only: blob shells,
body placements, orientations, active-slip draws and the grid descriptions of
the five benchmark workloads.  It contains none of the method's arithmetic
(no Stokes operator, kernel, spreading, solver or time stepping), so both the
CUDA path and the independent FP64 oracle may import it.

Randomness here uses numpy's Philox bit generator with a fixed seed per
workload; the method's own random draws (fluid noise, RFD forces) are not
made here.
"""
from .shells import icosahedral_shell, shell_12, shell_42
from .configs import (Workload, Body, two_sphere_cavity, single_sphere_box,
                      driven_monolayer, batched_ensemble, adjoint_suspension,
                      small_case, matvec_box, two_sphere_msd, boomerang_slit, WORKLOAD_SEED_BASE)

__all__ = ["icosahedral_shell", "shell_12", "shell_42", "Workload", "Body",
           "two_sphere_cavity", "single_sphere_box", "driven_monolayer",
           "batched_ensemble", "adjoint_suspension", "small_case", "matvec_box",
           "two_sphere_msd", "boomerang_slit", "WORKLOAD_SEED_BASE"]
