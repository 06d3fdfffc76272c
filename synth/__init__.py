"""Seeded synthetic inputs for 2-D multi-reference alignment in a steerable basis.

This module only draws data from the observation model of Eq. (MRA_Model_FB):
v_i = a o exp(-i k theta_i) + eps_i with complex Gaussian noise.  It holds none
of the estimation arithmetic (synchronization, EM, prior learning); both the
CUDA path and the CPU oracle consume what it produces.
"""
from .instances import (  # noqa: F401
    CONFIGS,
    Instance,
    config,
    make_instance,
    make_signal,
    random_init,
    sigma2_for_snr,
    image_energy,
    NPIX,
    to_c64,
    c64_round,
    bf16_split,
    bf16_merge,
    config4_instances,
)
from .mra1d import Instance1D, coeffs_1d, make_instance_1d, sigma2_coeff, signal_1d  # noqa: F401,E402
from .fb_images import noisy_images, real_params, render, render_matrix  # noqa: F401,E402
