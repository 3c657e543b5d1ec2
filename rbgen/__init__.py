"""Seeded synthetic inputs for ring-array sound-speed tomography.

This module draws inputs only: acquisition geometry parameters, sound-speed
and absorption phantoms, the initial guess, and the raw normal draws used for
measurement noise.  It holds none of the inversion's arithmetic (no rays, no
Green's functions, no Born operators), so that both the CUDA path and the
FP64 oracle can take their inputs from here without sharing method code.

The acquisition shapes follow the ring-array experiments of the paper
(Sec. 4: 256-element ring of radius 11 cm, water at 1480 m/s, sets of
consecutive frequencies swept from low to high); the phantoms are stand-ins
for the in-vitro and in-vivo datasets, which are not available here.
"""
from .configs import (Config, config_by_name, tiny, breast256, breast512, CONFIGS, ring, batch_mix,  # noqa: F401
                      poisson_requests)
from .phantom import Inputs, make_inputs, ellipse_phantom, breast_phantom, initial_guess, noise_draws  # noqa: F401
