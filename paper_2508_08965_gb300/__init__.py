"""GB300-native CGKS-5: the per-stage sweep of the fifth-order compact
gas-kinetic scheme (arXiv 2508.08965) as hand-written sm_103a CUDA behind a
C-ABI (include/cgks.h).  This package holds the ctypes binding (argument
marshalling only) and the in-tree build; there is no CPU fallback."""
from .binding import (  # noqa: F401
    CgksError, Mesh, Batch, lib, STATUS_NAMES, BC_PERIODIC, BC_OUTFLOW, BC_SLIP_WALL, BC_NOSLIP_WALL, BC_INFLOW,
)
