"""Seeded synthetic water-like systems (positions, block-CSR overlap S and Hamiltonian H).

This package produces *inputs* only. It holds none of the NOLSM arithmetic (no submatrix
construction, inverse, sign iteration or write-back). Both the FP64 oracle (``oracle/``) and the GPU
path's tests and benchmark draw their inputs from here, so that the two sides share nothing else.
"""
from .systems import (SystemSpec, BlockCSR, System, make_system, spec_small_fp64, spec_batched_uneven, spec_batched_uneven_4096,
                      spec_streamed_bf16, spec_streamed_4096, spec_split_valence, spec_mixed, spec_tiny,
                      minimum_image_pairs)
from .sites import SiteSpec, SitePattern, make_site_pattern, site_system, spec_ions_in_water, spec_ions_in_water_small

__all__ = ["SystemSpec", "BlockCSR", "System", "make_system", "spec_small_fp64", "spec_batched_uneven", "spec_batched_uneven_4096",
           "spec_streamed_bf16", "spec_streamed_4096", "spec_split_valence", "spec_mixed", "spec_tiny", "minimum_image_pairs",
           "SiteSpec", "SitePattern", "make_site_pattern", "site_system", "spec_ions_in_water", "spec_ions_in_water_small"]
