"""Workload configurations (grid, acquisition, time stepping, particle counts).

The paper's FWI example (Sec. 4.2) uses a 120 x 200 grid at 20 m, 10 sources
at 20 m depth, 200 receivers and a 10 Hz Ricker wavelet; the five workloads
below keep that shape at the sizes the benchmark and tests use:

  cfg1  64 x 64,   dx 10 m,  4 src,  32 rec,  400 steps, dt 1 ms,   8 particles
  cfg2  128 x 128, dx 10 m,  8 src,  64 rec,  800 steps, dt 1 ms   (gradient check)
  cfg3  120 x 300, dx 10 m, 20 src, 200 rec, 2000 steps, dt 1 ms, 600 particles
  cfg4  as cfg3 with reduced-precision wavefield storage and BF16 Gram
  cfg5  240 x 600, dx 10 m, 40 src, 400 rec, 3000 steps, dt 0.8 ms, 2000 particles

Sources and receivers sit on grid row iz = 2 (20 m below the top), equally
spaced between 20 m from either side: ix = round(linspace(2, nx - 3, count)).
Every padded grid adds a 20-cell absorbing sponge on each side.
"""
from dataclasses import dataclass, field
import numpy as np


@dataclass(frozen=True)
class Config:
    name: str
    nz: int
    nx: int
    dx: float
    dt: float
    nt: int
    nsrc: int
    nrec: int
    n_particles: int
    model: str                 # "linear_anomaly" or "layered"
    sigma_rule: str            # "rms1" (1% of RMS) or "medmax2" (2% of median trace max)
    prior_rule: str            # "trend500" or "band2000"
    f0: float = 10.0
    nsponge: int = 20
    sponge_alpha: float = 0.015
    src_iz: int = 2
    rec_iz: int = 2
    iters: int = 1
    ckpt_every: int = 1

    @property
    def NZ(self):
        return self.nz + 2 * self.nsponge

    @property
    def NX(self):
        return self.nx + 2 * self.nsponge

    @property
    def d(self):
        return self.nz * self.nx

    @property
    def t0(self):
        return 1.0 / self.f0

    def with_(self, **kw):
        f = dict(self.__dict__)
        f.update(kw)
        return Config(**f)


CONFIGS = {
    "cfg1": Config("cfg1", 64, 64, 10.0, 1e-3, 400, 4, 32, 8,
                   "linear_anomaly", "rms1", "trend500", iters=1),
    "cfg2": Config("cfg2", 128, 128, 10.0, 1e-3, 800, 8, 64, 4,
                   "linear_anomaly", "rms1", "trend500", ckpt_every=50),
    "cfg3": Config("cfg3", 120, 300, 10.0, 1e-3, 2000, 20, 200, 600,
                   "layered", "medmax2", "band2000", iters=50),
    "cfg4": Config("cfg4", 120, 300, 10.0, 1e-3, 2000, 20, 200, 600,
                   "layered", "medmax2", "band2000", iters=50),
    "cfg5": Config("cfg5", 240, 600, 10.0, 8e-4, 3000, 40, 400, 2000,
                   "layered", "medmax2", "band2000", iters=200),
}


def config(name):
    return CONFIGS[name]


def _line(count, n):
    if count == 1:
        return np.array([n // 2], dtype=np.int32)
    return np.rint(np.linspace(2, n - 3, count)).astype(np.int32)


def geometry(cfg):
    """Source and receiver grid indices (physical grid, row iz, column ix)."""
    src_ix = _line(cfg.nsrc, cfg.nx)
    rec_ix = _line(cfg.nrec, cfg.nx)
    src_iz = np.full(cfg.nsrc, cfg.src_iz, dtype=np.int32)
    rec_iz = np.full(cfg.nrec, cfg.rec_iz, dtype=np.int32)
    return dict(src_iz=src_iz, src_ix=src_ix, rec_iz=rec_iz, rec_ix=rec_ix)
