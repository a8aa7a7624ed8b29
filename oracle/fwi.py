"""FP64 oracle: 2-D constant-density acoustic FWI forward, misfit, adjoint, gradient.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper (Sec. 4.2) simulates waveforms "using a time-domain finite
difference method with a Ricker wavelet of 10 Hz", uses the Gaussian
likelihood of Eq. (26) and computes velocity gradients "using the adjoint
method" (Sec. 3). It leaves the scheme unstated; this oracle fixes it as:

  * PDE    (1/v^2) u_tt - lap(u) = f(t) delta(x - x_s)
  * space  8th-order central Laplacian, coefficients
           c = (-205/72, 8/5, -1/5, 8/315, -1/560), zero values outside the
           padded grid (a 4-cell Dirichlet ring)
  * model  v padded by edge replication into a 20-cell sponge on all sides
  * sponge Cerjan taper g = exp(-(alpha*dz)^2) exp(-(alpha*dx)^2), alpha 0.015,
           dz/dx the number of cells into the sponge (0 inside, 20 at the edge)
  * time   a^{n+1} = g [2 a^n + w (L a^n + s^n)] - g^2 a^{n-1},  w = vpad^2 dt^2,
           a^0 = a^{-1} = 0, s^n = f(n dt)/dx^2 at the source node
  * wavelet Ricker f(t) = (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2),
           tau = t - 1/f0
  * record d[r, n] = a^{n+1}[rec_r], n = 0 .. nt-1
  * misfit J = 1/2 sum ((d - d_obs)/sigma)^2   (negative log of Eq. 26)

The adjoint is the exact discrete adjoint of that recurrence:
  lambda^k = (2I + L W) G lambda^{k+1} - G^2 lambda^{k+2} + rho^k,
  rho^k = R^T (d[:, k-1] - d_obs[:, k-1]) / sigma^2,  lambda^{N+1} = lambda^{N+2} = 0,
and the gradient with respect to the padded velocity is
  dJ/dvpad = 2 vpad dt^2 sum_n g lambda^{n+1} (L a^n + s^n)
           = (2/vpad) sum_n lambda^{n+1} (a^{n+1} - 2 g a^n + g^2 a^{n-1}),
the second form being the discrete -2/v^3 * (second time derivative of the
forward field) x (adjoint field) imaging condition. Sponge cells are folded
onto the edge cells they replicate (chain rule of the padding).
"""
import numpy as np

C8 = (-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0)
HALO = 4


class Geom:
    """Grid, time axis and acquisition of one FWI problem (physical indices)."""

    def __init__(self, nz, nx, dx, dt, nt, src_iz, src_ix, rec_iz, rec_ix,
                 f0=10.0, t0=None, nsponge=20, alpha=0.015):
        self.nz, self.nx = int(nz), int(nx)
        self.dx, self.dt, self.nt = float(dx), float(dt), int(nt)
        self.src_iz = np.asarray(src_iz, dtype=np.int64)
        self.src_ix = np.asarray(src_ix, dtype=np.int64)
        self.rec_iz = np.asarray(rec_iz, dtype=np.int64)
        self.rec_ix = np.asarray(rec_ix, dtype=np.int64)
        self.f0 = float(f0)
        self.t0 = 1.0 / self.f0 if t0 is None else float(t0)
        self.nb = int(nsponge)
        self.alpha = float(alpha)

    @property
    def NZ(self):
        return self.nz + 2 * self.nb

    @property
    def NX(self):
        return self.nx + 2 * self.nb

    @property
    def nsrc(self):
        return self.src_ix.size

    @property
    def nrec(self):
        return self.rec_ix.size

    @classmethod
    def from_config(cls, cfg, geo):
        return cls(cfg.nz, cfg.nx, cfg.dx, cfg.dt, cfg.nt, geo["src_iz"],
                   geo["src_ix"], geo["rec_iz"], geo["rec_ix"], f0=cfg.f0,
                   nsponge=cfg.nsponge, alpha=cfg.sponge_alpha)


def pad_model(v, nb):
    """Edge-replicate the physical model into the sponge."""
    return np.pad(np.asarray(v, dtype=np.float64), nb, mode="edge")


def taper(NZ, NX, nb, alpha):
    """Cerjan sponge factor g(i, j) on the padded grid."""
    def profile(N):
        i = np.arange(N)
        into = np.maximum(np.maximum(nb - i, i - (N - 1 - nb)), 0)
        return np.exp(-(alpha * into) ** 2)
    return np.outer(profile(NZ), profile(NX))


def laplacian(u, dx):
    """8th-order 5-arm Laplacian with zero values outside the array."""
    NZ, NX = u.shape
    h = HALO
    up = np.zeros((NZ + 2 * h, NX + 2 * h))
    up[h:h + NZ, h:h + NX] = u
    out = 2.0 * C8[0] * u
    for k in range(1, 5):
        out = out + C8[k] * (up[h - k:h - k + NZ, h:h + NX]
                             + up[h + k:h + k + NZ, h:h + NX]
                             + up[h:h + NZ, h - k:h - k + NX]
                             + up[h:h + NZ, h + k:h + k + NX])
    return out / (dx * dx)


def ricker(t, f0, t0):
    tau = np.asarray(t, dtype=np.float64) - t0
    a = (np.pi * f0 * tau) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def _pad_index(geom, iz, ix):
    return np.asarray(iz) + geom.nb, np.asarray(ix) + geom.nb


def source_function(geom):
    """s^n at the source node: f(n dt)/dx^2, n = 0 .. nt-1."""
    return ricker(np.arange(geom.nt) * geom.dt, geom.f0, geom.t0) / geom.dx ** 2


def propagate(v, geom, src, q, keep=False):
    """Run the forward recurrence for one source.

    src  (iz, ix) physical index of the source node
    q    source time function added at that node, q[n] plays s^n
    keep also return the history a^{-1}, a^0, ..., a^N as an (N+2, NZ, NX) array

    Returns traces [R, nt] (and the history when keep is set)."""
    vpad = pad_model(v, geom.nb)
    w = (vpad * geom.dt) ** 2
    g = taper(geom.NZ, geom.NX, geom.nb, geom.alpha)
    sz, sx = _pad_index(geom, src[0], src[1])
    rz, rx = _pad_index(geom, geom.rec_iz, geom.rec_ix)
    a_prev = np.zeros((geom.NZ, geom.NX))
    a = np.zeros_like(a_prev)
    traces = np.zeros((geom.nrec, geom.nt))
    hist = [a_prev.copy(), a.copy()] if keep else None
    for n in range(geom.nt):
        lap = laplacian(a, geom.dx)
        lap[sz, sx] += q[n]
        a_next = g * (2.0 * a + w * lap) - g * g * a_prev
        traces[:, n] = a_next[rz, rx]
        a_prev, a = a, a_next
        if keep:
            hist.append(a.copy())
    if keep:
        return traces, np.stack(hist)
    return traces


def forward(v, geom, isrc):
    """Seismograms [R, nt] for source number isrc with the Ricker wavelet."""
    src = (geom.src_iz[isrc], geom.src_ix[isrc])
    return propagate(v, geom, src, source_function(geom))


def seismograms(V, geom):
    """Seismograms for a batch of particles V [P, nz*nx] -> [P, S, R, nt]."""
    V = np.asarray(V, dtype=np.float64).reshape(-1, geom.nz, geom.nx)
    out = np.zeros((V.shape[0], geom.nsrc, geom.nrec, geom.nt))
    for p in range(V.shape[0]):
        for s in range(geom.nsrc):
            out[p, s] = forward(V[p], geom, s)
    return out


def misfit(d, d_obs, sigma):
    """J = 1/2 sum ((d - d_obs)/sigma)^2, the negative log-likelihood of Eq. (26)
    up to its constant."""
    r = (np.asarray(d, dtype=np.float64) - d_obs) / sigma
    return 0.5 * float(np.sum(r * r))


def adjoint_fields(v, geom, resid):
    """Exact discrete adjoint for traces-space sensitivities resid [R, nt].

    resid[:, n] is dJ/dd[:, n]; rho^k = R^T resid[:, k-1]. Returns the list
    lambda^1 .. lambda^N as an (N+1, NZ, NX) array with index 0 unused (zeros)."""
    vpad = pad_model(v, geom.nb)
    w = (vpad * geom.dt) ** 2
    g = taper(geom.NZ, geom.NX, geom.nb, geom.alpha)
    rz, rx = _pad_index(geom, geom.rec_iz, geom.rec_ix)
    N = geom.nt
    lam = np.zeros((N + 1, geom.NZ, geom.NX))
    lam1 = np.zeros((geom.NZ, geom.NX))      # lambda^{k+1}
    lam2 = np.zeros_like(lam1)               # lambda^{k+2}
    for k in range(N, 0, -1):
        rho = np.zeros_like(lam1)
        np.add.at(rho, (rz, rx), resid[:, k - 1])
        lk = 2.0 * g * lam1 + laplacian(w * g * lam1, geom.dx) \
            - g * g * lam2 + rho
        lam[k] = lk
        lam2, lam1 = lam1, lk
    return lam


def fold(grad_pad, geom):
    """Chain rule of the edge-replication padding: each padded cell adds its
    value to the physical cell it copies."""
    nb = geom.nb
    iz = np.clip(np.arange(geom.NZ) - nb, 0, geom.nz - 1)
    ix = np.clip(np.arange(geom.NX) - nb, 0, geom.nx - 1)
    out = np.zeros((geom.nz, geom.nx))
    np.add.at(out, (iz[:, None], ix[None, :]), grad_pad)
    return out


def pair_gradient(v, geom, isrc, resid_fn, both_forms=False, magnitude=False):
    """Velocity gradient (physical grid) for one source.

    resid_fn(traces) -> dJ/dtraces [R, nt]. Returns (traces, grad[nz, nx]) and,
    if both_forms, also the two padded-grid gradients for comparison. With
    magnitude, returns (traces, grad, mag) where mag[nz, nx] is the same sum
    with every time term replaced by its absolute value,
    2 vpad dt^2 sum_n |g lambda^{n+1} (L a^n + s^n)|, folded: the scale
    against which the rounding of one factor of each term is measured."""
    src = (geom.src_iz[isrc], geom.src_ix[isrc])
    q = source_function(geom)
    traces, hist = propagate(v, geom, src, q, keep=True)
    resid = resid_fn(traces)
    lam = adjoint_fields(v, geom, resid)
    vpad = pad_model(v, geom.nb)
    g = taper(geom.NZ, geom.NX, geom.nb, geom.alpha)
    sz, sx = _pad_index(geom, src[0], src[1])
    # hist[j] = a^{j-1}
    acc1 = np.zeros_like(vpad)
    acc2 = np.zeros_like(vpad)
    accm = np.zeros_like(vpad)
    for n in range(geom.nt):
        a_nm1, a_n, a_np1 = hist[n], hist[n + 1], hist[n + 2]
        src_term = laplacian(a_n, geom.dx)
        src_term[sz, sx] += q[n]
        term = g * lam[n + 1] * src_term
        acc1 += term
        if magnitude:
            accm += np.abs(term)
        if both_forms:
            acc2 += lam[n + 1] * (a_np1 - 2.0 * g * a_n + g * g * a_nm1)
    gpad1 = 2.0 * vpad * geom.dt ** 2 * acc1
    grad = fold(gpad1, geom)
    if magnitude:
        return traces, grad, fold(2.0 * vpad * geom.dt ** 2 * accm, geom)
    if both_forms:
        gpad2 = 2.0 / vpad * acc2
        return traces, grad, gpad1, gpad2
    return traces, grad


def gradient(v, geom, d_obs, sigma, sources=None):
    """Misfit J and dJ/dv [nz, nx] for one model, summed over all sources, or
    over the listed sources only (a minibatch of the data, Sec. 3 after
    Eq. 22: (S / len(sources)) times the sum is an unbiased estimate of the
    full values when the minibatch is drawn uniformly).

    d_obs [S, R, nt] observed traces, sigma scalar noise standard deviation."""
    v = np.asarray(v, dtype=np.float64).reshape(geom.nz, geom.nx)
    J = 0.0
    grad = np.zeros((geom.nz, geom.nx))
    for s in (range(geom.nsrc) if sources is None else sources):
        def resid_fn(tr, s=s):
            return (tr - d_obs[s]) / sigma ** 2
        tr, gs = pair_gradient(v, geom, s, resid_fn)
        J += misfit(tr, d_obs[s], sigma)
        grad += gs
    return J, grad


def gradient_magnitude(v, geom, d_obs, sigma, sources=None):
    """Per physical cell, the sum over sources and time steps of the absolute
    values of the imaging-condition terms whose signed sum is dJ/dv (see
    pair_gradient): rounding one factor of every term to a relative
    precision u changes dJ/dv by at most u times this. Returns [nz, nx]."""
    v = np.asarray(v, dtype=np.float64).reshape(geom.nz, geom.nx)
    mag = np.zeros((geom.nz, geom.nx))
    for s in (range(geom.nsrc) if sources is None else sources):
        def resid_fn(tr, s=s):
            return (tr - d_obs[s]) / sigma ** 2
        _, _, m = pair_gradient(v, geom, s, resid_fn, magnitude=True)
        mag += m
    return mag


def gradients(V, geom, d_obs, sigma, sources=None):
    """Batch version: J [P] and dJ/dv [P, nz*nx]."""
    V = np.asarray(V, dtype=np.float64).reshape(-1, geom.nz, geom.nx)
    J = np.zeros(V.shape[0])
    G = np.zeros((V.shape[0], geom.nz * geom.nx))
    for p in range(V.shape[0]):
        J[p], g = gradient(V[p], geom, d_obs, sigma, sources)
        G[p] = g.reshape(-1)
    return J, G


def adjoint_of_upstream(v, geom, dseis):
    """dL/dv for an upstream sensitivity dseis = dL/dtraces [S, R, nt]
    (the backward of the seismogram map, used by autograd)."""
    v = np.asarray(v, dtype=np.float64).reshape(geom.nz, geom.nx)
    grad = np.zeros((geom.nz, geom.nx))
    for s in range(geom.nsrc):
        _, gs = pair_gradient(v, geom, s, lambda tr, s=s: dseis[s])
        grad += gs
    return grad


def source_adjoint(v, geom, src, resid):
    """Adjoint of the map q -> traces at fixed v: returns dJ/dq[n] =
    g w lambda^{n+1} at the source node, for the dot-product test."""
    vpad = pad_model(v, geom.nb)
    w = (vpad * geom.dt) ** 2
    g = taper(geom.NZ, geom.NX, geom.nb, geom.alpha)
    lam = adjoint_fields(v, geom, resid)
    sz, sx = _pad_index(geom, src[0], src[1])
    return np.array([g[sz, sx] * w[sz, sx] * lam[n + 1][sz, sx]
                     for n in range(geom.nt)])
