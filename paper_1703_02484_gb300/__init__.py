"""GB300-native Brownian hard-disk time stepper (arXiv:1703.02484 hot path).

The compute path is libbd_gb300.so (CUDA kernels for sm_103a behind the C ABI
of include/bd.h); this package only marshals arguments to it."""
from . import workloads  # noqa: F401
from .binding import (BOUNDARY_PERIODIC, BOUNDARY_WALLS, LAW_LONG, LAW_NONE, LAW_SHORT, LOSS_HIST, LOSS_MSD,  # noqa: F401
                      OVERLAP_DELAUNAY, OVERLAP_VERLET, PLACE_LATTICE, PLACE_RSA, BDError, System, load,
                      make_params, params_from_config, place_disks, rollout_loss)
