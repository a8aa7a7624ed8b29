"""Seeded inputs for the travel-time tomography workload (inputs only).

The paper's tomography example (Sec. 4.1) inverts Love-wave group travel
times at 10 s period between 61 stations on a 37 x 40 grid of 0.33 degree
cells with a U(1.56, 4.8) km/s prior. Its ambient-noise dataset is not
available, so these generators stand in for it with the same shapes: a
regular grid, randomly placed stations, a smooth random group-velocity map
inside the prior, per-pair noise levels from the station distance, and
unit-normal noise. Nothing here evaluates travel times or gradients.

Seeds follow the FWI convention: model 0, data noise 1, particles 2,
stations 3. Arrays are float64 [ny][nx] with x (longitude) fastest.
"""
from dataclasses import dataclass, replace

import numpy as np
from scipy.ndimage import gaussian_filter

KM_PER_DEGREE = 111.195


@dataclass(frozen=True)
class TomoConfig:
    name: str
    ny: int               # latitude nodes (rows)
    nx: int               # longitude nodes (columns)
    h: float              # node spacing, km
    n_stations: int
    n_particles: int
    vmin: float = 1.56    # prior bounds, km/s
    vmax: float = 4.8

    @property
    def d(self):
        return self.ny * self.nx

    @property
    def n_pairs(self):
        return self.n_stations * (self.n_stations - 1) // 2

    def with_(self, **kw):
        return replace(self, **kw)


TOMO_CONFIGS = {
    # a few tiles and ragged rows, for element-by-element parity
    "tomo_small": TomoConfig("tomo_small", ny=18, nx=23, h=0.33 * KM_PER_DEGREE,
                             n_stations=9, n_particles=4),
    # the paper's British Isles grid and station count, 500 SVGD particles
    "tomo_uk": TomoConfig("tomo_uk", ny=40, nx=37, h=0.33 * KM_PER_DEGREE,
                          n_stations=61, n_particles=500),
}


def tomo_config(name):
    return TOMO_CONFIGS[name]


def stations(cfg, seed=3):
    """n_stations distinct node indices (row * nx + col), drawn uniformly
    from the nodes at least one node away from the grid edge."""
    rng = np.random.default_rng(seed)
    inner = [(i, j) for i in range(1, cfg.ny - 1) for j in range(1, cfg.nx - 1)]
    pick = rng.choice(len(inner), size=cfg.n_stations, replace=False)
    return np.array([inner[k][0] * cfg.nx + inner[k][1] for k in pick],
                    dtype=np.int32)


def true_group_velocity(cfg, seed=0):
    """Smooth random map: white noise Gaussian-filtered (sigma 3 nodes),
    scaled to a standard deviation of 0.45 km/s about 3.1 km/s and clipped to
    [1.8, 4.5] km/s, inside the U(1.56, 4.8) prior."""
    rng = np.random.default_rng(seed)
    w = gaussian_filter(rng.standard_normal((cfg.ny, cfg.nx)), sigma=3.0,
                        mode="reflect")
    w = (w - w.mean()) / w.std()
    return np.clip(3.1 + 0.45 * w, 1.8, 4.5)


def prior_bounds(cfg):
    lo = np.full((cfg.ny, cfg.nx), cfg.vmin)
    hi = np.full((cfg.ny, cfg.nx), cfg.vmax)
    return lo, hi


def pair_sigma(cfg, sta):
    """Per-pair noise standard deviation (s), ordered like the data (source
    station s < receiver station r, s major): 1% of the straight-line travel
    time at 3 km/s, at least 0.5 s."""
    iy, ix = np.divmod(np.asarray(sta, dtype=np.int64), cfg.nx)
    out = []
    for s in range(cfg.n_stations):
        for r in range(s + 1, cfg.n_stations):
            dist = cfg.h * np.hypot(iy[r] - iy[s], ix[r] - ix[s])
            out.append(max(0.5, 0.01 * dist / 3.0))
    return np.array(out)


def particles_from_prior(cfg, n, seed=2):
    """n particles uniform in the prior box, shape [n][ny*nx]."""
    rng = np.random.default_rng(seed)
    return cfg.vmin + (cfg.vmax - cfg.vmin) * rng.uniform(0.0, 1.0, size=(n, cfg.d))


def smooth_particles(cfg, n, seed=2):
    """n smooth random maps (sigma 2 nodes, std 0.4 km/s about U(2.6, 3.6)),
    clipped to [1.7, 4.6]: heterogeneous but ray-friendly test models."""
    rng = np.random.default_rng(seed)
    out = np.empty((n, cfg.d))
    for k in range(n):
        w = gaussian_filter(rng.standard_normal((cfg.ny, cfg.nx)), sigma=2.0,
                            mode="reflect")
        w = (w - w.mean()) / w.std()
        out[k] = np.clip(rng.uniform(2.6, 3.6) + 0.4 * w, 1.7, 4.6).reshape(-1)
    return out


def unit_noise(n, seed=1):
    return np.random.default_rng(seed).standard_normal(n)
