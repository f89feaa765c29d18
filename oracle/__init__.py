"""CPU FP64 oracle of the cube synthesis (test infrastructure only; see ``cube``)."""
from .cube import (valid_mask, valid_indices, path_terms, phase_cycles, cube_literal,
                   cube_separable, cube_entries, rel_l2)

from .estimation import range_doppler_power, max_power_velocity, e_velo
from . import raycast
from . import nufft

__all__ = ["valid_mask", "valid_indices", "path_terms", "phase_cycles", "cube_literal",
           "cube_separable", "cube_entries", "rel_l2", "range_doppler_power",
           "max_power_velocity", "e_velo", "raycast", "nufft"]
