"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This package holds geometry and random numbers only: voxel masks (ducts, sphere
packs, random tiny masks) and arrays of uniform random numbers. It contains none
of the lattice Boltzmann arithmetic, so both sides can draw identical inputs
from it without sharing any of the method's code.
"""
from .geometry import (  # noqa: F401
    duct_mask,
    random_mask,
    sphere_pack,
    keep_inlet_connected,
    uniform_field,
)
