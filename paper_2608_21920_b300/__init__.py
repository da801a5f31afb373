"""B300-native library for the time step of the 1D radiative particle-in-cell
model of pulsar polar-cap pair discharges, and for the batched concurrency
model with its adjoint (paper: "Pair Discharges and Radio Emission from Pulsar
Magnetospheres").

The compute path is libgap.so (hand-written CUDA for sm_103a, C ABI in
include/gap.h).  This package only marshals arguments: torch provides device
memory and streams.  Importing it does not require a GPU; creating a Gap or
calling the ODE functions does, and fails loudly if the library is missing.
"""
from ._abi import (GAP_BC_PERIODIC, GAP_BC_SURFACE, GAP_ELECTRON, GAP_FP32_STATE,  # noqa: F401
                   GAP_FP64_PLAIN, GAP_INIT_COLD, GAP_INIT_EMPTY, GAP_INIT_PAIR_THERMAL,
                   GAP_PHOTON, GAP_POSITRON, GapError, lib)
from .gap import Gap, make_params  # noqa: F401

__all__ = ["Gap", "make_params", "lib", "GapError"]
