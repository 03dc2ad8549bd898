"""FP64 CPU oracle of the layered UTR reconstruction (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs import this
package.  The reconstruction library neither imports nor links it; the two share
no code.  See ``recon_fp64`` for what it computes and the passage each step follows.
"""
from .recon_fp64 import (  # noqa: F401
    FILTER_DEPTH_COS, FILTER_DEPTH_SIN, FILTER_OFF, FILTER_PAIR, FILTER_TIKHONOV, depth_phase_filter, ctf_pair_filter, INPUT_CONTRAST, INPUT_INTENSITY, INTENSITY_FLOOR, LAYER_FRAC_BITS, LAYER_LINEAR,
    LAYER_NEAREST, layer_blend,
    backproject_direction, bilinear, contrast, ctf_filter, density_geometry, density_grid, density_weights, depth_extent, layer_centres, layer_constants,
    layer_index, layer_stack, padded_size, pixel_coefficients, ramp_weights, recon, signed_freq,
)
from . import learned_fp64 as learned  # noqa: F401,E402
from . import fourier_fp64 as fourier  # noqa: F401,E402
