"""Seeded velocity models, prior bounds, particles and noise (inputs only).

Seeds follow one fixed convention: model 0, data noise 1, particles 2.
All arrays are float64 numpy, row-major [nz][nx] with x fastest.
"""
import numpy as np
from scipy.ndimage import gaussian_filter


def _linear_anomaly(cfg):
    """Linear 1500 -> 3000 m/s with depth times two +/-10% Gaussian anomalies
    (sigma 60 m) centred at (x, z) = (0.35, 0.45) L and (0.65, 0.65) L."""
    z = np.arange(cfg.nz) * cfg.dx
    x = np.arange(cfg.nx) * cfg.dx
    Lz, Lx = z[-1], x[-1]
    Z, X = np.meshgrid(z, x, indexing="ij")
    v = 1500.0 + 1500.0 * Z / Lz
    s = 60.0
    for fx, fz, amp in ((0.35, 0.45, +0.10), (0.65, 0.65, -0.10)):
        r2 = (X - fx * Lx) ** 2 + (Z - fz * Lz) ** 2
        v = v * (1.0 + amp * np.exp(-r2 / (2 * s * s)))
    return v


def _layered(cfg, rng):
    """Eight layers with sorted random interfaces and sorted U(1500, 4500)
    velocities, Gaussian-smoothed (sigma 3 cells), plus five Gaussian anomalies
    (sigma U(40, 100) m, amplitude +/-U(5, 15)%), clipped to [1500, 4500]."""
    nz, nx = cfg.nz, cfg.nx
    iface = np.sort(rng.uniform(0, nz, size=7))
    vel = np.sort(rng.uniform(1500.0, 4500.0, size=8))
    zi = np.arange(nz) + 0.5
    layer = np.searchsorted(iface, zi)
    v = np.repeat(vel[layer][:, None], nx, axis=1)
    v = gaussian_filter(v, sigma=3.0, mode="nearest")
    Z, X = np.meshgrid(np.arange(nz) * cfg.dx, np.arange(nx) * cfg.dx,
                       indexing="ij")
    for _ in range(5):
        cz = rng.uniform(0.15, 0.85) * (nz - 1) * cfg.dx
        cx = rng.uniform(0.15, 0.85) * (nx - 1) * cfg.dx
        s = rng.uniform(40.0, 100.0)
        amp = rng.uniform(0.05, 0.15) * rng.choice([-1.0, 1.0])
        v = v * (1.0 + amp * np.exp(-((Z - cz) ** 2 + (X - cx) ** 2)
                                    / (2 * s * s)))
    return np.clip(v, 1500.0, 4500.0)


def true_model(cfg, seed=0):
    rng = np.random.default_rng(seed)
    if cfg.model == "linear_anomaly":
        return _linear_anomaly(cfg)
    if cfg.model == "layered":
        return _layered(cfg, rng)
    raise ValueError(cfg.model)


def prior_bounds(cfg, v_true):
    """Per-cell uniform prior bounds (lo, hi), each [nz][nx].

    trend500: [max(trend - 500, 1500), trend + 500] about the linear trend
    1500 -> 3000 m/s. band2000: a 2 km/s band centred on a least-squares line
    through the true model's row means, floor 1500 m/s (the paper's extra
    lower bound, Sec. 4.2), cap 5000 m/s."""
    nz, nx = cfg.nz, cfg.nx
    z = np.arange(nz, dtype=np.float64)
    if cfg.prior_rule == "trend500":
        trend = 1500.0 + 1500.0 * z / z[-1]
        lo = np.maximum(trend - 500.0, 1500.0)
        hi = trend + 500.0
    elif cfg.prior_rule == "band2000":
        rm = v_true.mean(axis=1)
        c1, c0 = np.polyfit(z, rm, 1)
        centre = c0 + c1 * z
        lo = np.maximum(centre - 1000.0, 1500.0)
        hi = np.minimum(centre + 1000.0, 5000.0)
        hi = np.maximum(hi, lo + 1.0)
    else:
        raise ValueError(cfg.prior_rule)
    return (np.repeat(lo[:, None], nx, axis=1),
            np.repeat(hi[:, None], nx, axis=1))


def particles_from_prior(lo, hi, n, seed=2):
    """n particles drawn uniformly inside the prior box, shape [n][nz*nx]."""
    rng = np.random.default_rng(seed)
    lo = lo.reshape(-1)
    hi = hi.reshape(-1)
    u = rng.uniform(0.0, 1.0, size=(n, lo.size))
    return lo[None, :] + u * (hi - lo)[None, :]


def unit_noise(shape, seed=1):
    """Standard-normal array for the data noise (scaled by sigma later)."""
    return np.random.default_rng(seed).standard_normal(shape)


def sigma_from_traces(d_clean, rule):
    """Scalar data-noise standard deviation from clean traces [..., R, nt].

    rms1:    1% of the RMS amplitude over all samples.
    medmax2: 2% of the median over traces of each trace's maximum absolute
             amplitude (the paper's FWI noise level, Sec. 4.2)."""
    d = np.asarray(d_clean, dtype=np.float64)
    if rule == "rms1":
        return 0.01 * float(np.sqrt(np.mean(d * d)))
    if rule == "medmax2":
        tr = np.abs(d.reshape(-1, d.shape[-1])).max(axis=1)
        return 0.02 * float(np.median(tr))
    raise ValueError(rule)
