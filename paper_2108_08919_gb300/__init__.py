"""GB300 (sm_103a) SPH active-nematic solver (arXiv 2108.08919).

The physics runs in hand-written CUDA kernels behind the C-ABI of ``include/ann.h``; ``binding``
marshals Python arguments to it.  Importing the package does not load the library: the first call
of a ``binding`` function does, and raises if it has not been built (see ``build``).
"""
from . import binding  # noqa: F401
from .binding import (AnnError, FIELDS, ann_create, ann_default_params, ann_destroy,  # noqa: F401
                      ann_get_diagnostics, ann_get_field, ann_get_neighbors, ann_grid_info,
                      ann_kernel_count, ann_kernel_name, ann_last_error, ann_load_state,
                      ann_save_state, ann_set_particles, ann_set_record, ann_set_stream, ann_step,
                      ann_step_profile, ann_validate_params, ann_velocity_moments_noalloc,
                      ann_version)

__all__ = [n for n in dir() if n.startswith("ann_")] + ["AnnError", "FIELDS", "binding"]
