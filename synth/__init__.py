"""Seeded synthetic inputs for the FWI + SVGD hot path.

This package is shared by the CUDA product path, the benchmark and the FP64
oracle. It produces only inputs: grid geometry, velocity models shaped like the
paper's FWI example (Sec. 4.2), prior bounds, initial particles and unit-normal
noise arrays. It contains none of the method's arithmetic (no wave propagation,
no adjoint, no kernel or update rule); the one data-dependent rule here, the
noise level taken from clean traces, is part of the experiment description
(Sec. 4.2), not of the inversion method.
"""
from .configs import Config, CONFIGS, config, geometry
from .models import (true_model, prior_bounds, particles_from_prior,
                     unit_noise, sigma_from_traces)

__all__ = ["Config", "CONFIGS", "config", "geometry", "true_model",
           "prior_bounds", "particles_from_prior", "unit_noise",
           "sigma_from_traces"]
