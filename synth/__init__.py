"""Seeded synthetic inputs for the CGKS-5 sweep.

This module only evaluates analytic initial fields (primitive variables
rho, U, V[, W], p at given physical points) and builds node coordinates of
structured meshes.  It contains none of the scheme's arithmetic (no cell
averaging, no derivatives, no fluxes), so it can feed both the CPU oracle and
the CUDA path.  Every function works on numpy arrays and on torch tensors
(the array namespace is taken from the arguments).
"""
from .fields import (  # noqa: F401
    shock_vortex_params, shock_vortex_upstream, shock_vortex_2d, shock_vortex_inflow,
    isentropic_vortex_2d, taylor_green_3d, density_sine_3d, uniform_state,
    sod_x, riemann4_2d, riemann4_params, turbulence_velocity_grid, random_smooth_3d, turbulence_field,
)
from .meshes import uniform_nodes, perturbed_nodes_3d, perturbed_nodes_xy  # noqa: F401
from .ensemble import ensemble_stream, ensemble_specs, spec_mesh, spec_field  # noqa: F401
