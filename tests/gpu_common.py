"""Shared fixtures of the GPU parity tests: seeded problems and the oracle's
expected values (computed here, never from the CUDA path)."""
import functools

import numpy as np

import synth
from oracle import fwi as ofwi


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def problem(cfg, P, seed_particles=2):
    """(cfg, geometry dict, oracle Geom, v_true, particles [P, d], d_obs, sigma)
    with d_obs = oracle traces of v_true plus seeded noise (Sec. 4.2 recipe)."""
    geo = synth.geometry(cfg)
    g = ofwi.Geom.from_config(cfg, geo)
    v_true = synth.true_model(cfg)
    lo, hi = synth.prior_bounds(cfg, v_true)
    V = synth.particles_from_prior(lo, hi, P, seed=seed_particles)
    clean = np.stack([ofwi.forward(v_true, g, s) for s in range(g.nsrc)])
    sigma = synth.sigma_from_traces(clean, cfg.sigma_rule)
    d_obs = clean + sigma * synth.unit_noise(clean.shape, seed=1)
    return cfg, geo, g, v_true, V, d_obs, sigma, lo, hi


@functools.lru_cache(maxsize=None)
def cfg1_case(P=2):
    return problem(synth.config("cfg1"), P)


@functools.lru_cache(maxsize=None)
def cfg1_oracle_gradients(P=2):
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(P)
    return ofwi.gradients(V, g, d_obs, sigma)


def odd_config():
    """A ragged grid (37 x 53): not a multiple of any tile, band or vector
    width, with sources and receivers off the tile boundaries."""
    return synth.config("cfg1").with_(nz=37, nx=53, nt=150, nsrc=3, nrec=7)
