"""Shared fixtures of the GPU parity tests: seeded problems and the oracle's
expected values (computed here, never from the CUDA path)."""
import functools

import numpy as np

import synth
from oracle import fwi as ofwi


# Relative error bound of the misfit reduction (Eq. 26) on the GPU's own
# traces. Each residual r = d - d_obs is rounded to FP32 once, so r^2 is within
# 2 u of its exact value (u = 2^-24); each receiver's squares are summed in FP32
# over blocks of at most 16 steps, one FMA per step, whose 16 roundings of a
# sum of positive terms stay within 16 u of the block sum; the blocks, receivers
# and sources are then added in FP64. Together 18 u = 1.07e-6, held at 1.1e-6.
MISFIT_REDUCTION_TOL = 1.1e-6


def misfit_tolerance(traces, d_obs):
    """Relative tolerance of the misfit J (Eq. 26) against the oracle, derived
    from the FP32 trace bound rel(d) <= 1e-5: J = |r|^2 / (2 sigma^2) with
    r = d - d_obs, so dJ / J = 2 <r, dd> / |r|^2 <= 2 (|d| / |r|) rel(d), plus
    the reduction's own rounding (MISFIT_REDUCTION_TOL).
    traces [P, ...] are the oracle's traces of the particles, d_obs the
    observed data they are compared with (broadcast over P)."""
    t = np.asarray(traces, dtype=np.float64).reshape(len(traces), -1)
    r = t - np.asarray(d_obs, dtype=np.float64).reshape(1, -1)
    ratio = np.linalg.norm(t, axis=1) / np.linalg.norm(r, axis=1)
    return 2.0 * ratio.max() * 1e-5 + MISFIT_REDUCTION_TOL


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


# ---------------------------------------------------------------------------
# The FP64 oracle's independent pieces of work (one (particle, source) pair,
# one block of distance rows) run in a pool of spawned single-threaded
# processes: spawned, not forked, so no child inherits a CUDA context.
_POOL = None


def oracle_map(fn, jobs):
    """[fn(j) for j in jobs] in the spawned pool (in order)."""
    global _POOL
    jobs = list(jobs)
    if len(jobs) <= 1:
        return [fn(j) for j in jobs]
    if _POOL is None:
        import multiprocessing as mp
        import os
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        _POOL = mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1)))
    return _POOL.map(fn, jobs, chunksize=1)


def pair_job(job):
    """Oracle traces, gradient and imaging-term magnitude of one (model,
    source) pair: job = (geom, v [nz, nx], source, d_obs[source] or None,
    sigma). Without observed data only the traces are computed."""
    g, v, s, dobs_s, sigma = job
    if dobs_s is None:
        return ofwi.forward(v, g, s)
    tr, grad, mag = ofwi.pair_gradient(v, g, s, lambda t: (t - dobs_s) / sigma ** 2,
                                       magnitude=True)
    return tr, grad, mag


def sqdist_job(job):
    from oracle import svgd as osvgd
    path, rows = job
    return osvgd.sqdist_rows(np.load(path), rows)


def oracle_sqdist(X, blocks=32):
    """The oracle's full squared-distance matrix, its rows in parallel (the
    particles reach the workers through a temporary .npy file)."""
    import os
    import tempfile
    n = X.shape[0]
    parts = np.array_split(np.arange(n), min(blocks, n))
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "X.npy")
        np.save(path, np.asarray(X, dtype=np.float64))
        return np.vstack(oracle_map(sqdist_job, [(path, [int(i) for i in p]) for p in parts]))


def oracle_gradients(g, V, sources, d_obs, sigma):
    """Per particle: misfit J (Eq. 26), dJ/dv and the magnitude sum, over the
    listed sources (d_obs indexed like the geometry's sources)."""
    jobs = [(g, V[p].reshape(g.nz, g.nx), s, d_obs[s], sigma)
            for p in range(V.shape[0]) for s in sources]
    out = oracle_map(pair_job, jobs)
    J = np.zeros(V.shape[0])
    G = np.zeros((V.shape[0], g.nz * g.nx))
    M = np.zeros_like(G)
    traces = {}
    k = 0
    for p in range(V.shape[0]):
        for s in sources:
            tr, grad, mag = out[k]
            k += 1
            J[p] += ofwi.misfit(tr, d_obs[s], sigma)
            G[p] += grad.reshape(-1)
            M[p] += mag.reshape(-1)
            traces[(p, s)] = tr
    return J, G, M, traces
