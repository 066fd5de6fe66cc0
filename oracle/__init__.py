"""CPU FP64 oracle for the D3Q19 flux-boundary LBM.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg; never by the library.  Shares no code with the
CUDA path.
"""
from .lbm_oracle import (  # noqa: F401
    XI, W, OPP, NQ, CS2, RHO0, D3Q19Oracle, equilibrium, moment_matrix, relaxation_rates,
    collide_mrt, collide_bgk, stream_pull, stream_pull_loops, inlet_known_sum,
    outlet_known_sum, flux_density, hh_closure_inlet, hh_closure_outlet, moments, steady_residual,
)
from .poiseuille import duct_velocity, duct_flow_rate_per_gradient  # noqa: F401
