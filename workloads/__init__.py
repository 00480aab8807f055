"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This package draws random numbers and lays out input arrays (basin masks, bathymetry,
wind stress, Coriolis parameter, right-hand sides, request streams). It holds none of the
finite element method's arithmetic: no element integrals, no assembly, no solver.
"""
from .basins import (  # noqa: F401
    Basin,
    WALL_WEST, WALL_EAST, WALL_SOUTH, WALL_NORTH, WALL_ALL,
    box_basin,
    ocean_basin,
    batch_basins,
    request_stream,
    Session,
    Request,
    mms_modes,
    manufactured_field,
    random_vector,
)
