"""CPU FP64 oracle of the cube synthesis (test infrastructure only; see ``cube``)."""
from .cube import (valid_mask, valid_indices, path_terms, phase_cycles, cube_literal,
                   cube_separable, cube_entries, rel_l2)

__all__ = ["valid_mask", "valid_indices", "path_terms", "phase_cycles", "cube_literal",
           "cube_separable", "cube_entries", "rel_l2"]
