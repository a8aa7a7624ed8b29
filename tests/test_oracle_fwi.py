"""Pins of the FP64 FWI oracle against results fixed by mathematics.

* forward: the 2-D Green's function of (1/v^2) u_tt - lap u = f delta
  (Hankel-function solution) and second-order convergence in dt;
* adjoint recurrence: <F q, r> = <q, F^T r> to round-off;
* gradient: Taylor remainder of second order, central differences per cell
  (sponge-edge and corner cells included), and agreement of the two
  imaging-condition forms;
* misfit: exactly zero at the true model with noise-free data;
* padding fold: it is the transpose of edge replication.
"""
import numpy as np
import pytest
from scipy.special import hankel2

from oracle import fwi


def _small_geom(nz=16, nx=20, nt=150, nsrc=2, nrec=6, dt=1e-3):
    src_ix = np.rint(np.linspace(2, nx - 3, nsrc)).astype(int)
    rec_ix = np.rint(np.linspace(1, nx - 2, nrec)).astype(int)
    return fwi.Geom(nz, nx, 10.0, dt, nt, [2] * nsrc, src_ix,
                    [3] * nrec, rec_ix, nsponge=20, alpha=0.015)


def _small_model(nz, nx, seed=5):
    rng = np.random.default_rng(seed)
    z = np.arange(nz)[:, None] / (nz - 1)
    x = np.arange(nx)[None, :] / (nx - 1)
    v = 1800.0 + 900.0 * z + 150.0 * np.sin(3 * x + 2 * z)
    return v + rng.uniform(-40, 40, size=(nz, nx))


def _green_trace(dt, nt, r, v0, f0, t0):
    """Analytic u(r, t) = f * G, G = H(t - r/v) / (2 pi sqrt(t^2 - r^2/v^2)),
    evaluated in the frequency domain as U = F (-i/4) H0^(2)(w r / v) with
    numpy's e^{-i w t} transform (the conjugate of the outgoing
    (i/4) H0^(1) form), sampled at t = (n+1) dt."""
    M = 8 * nt
    t = np.arange(M) * dt
    F = np.fft.rfft(fwi.ricker(t, f0, t0))
    w = 2 * np.pi * np.fft.rfftfreq(M, dt)
    H = np.zeros_like(F)
    H[1:] = -0.25j * hankel2(0, w[1:] * r / v0)
    return np.fft.irfft(F * H, M)[1:nt + 1]


def test_forward_matches_green_function_second_order_in_time():
    n, dx, v0, T = 201, 10.0, 2000.0, 0.55
    c = n // 2
    rec_ix = np.array([c + 20, c + 40, c + 60])   # r = 200, 400, 600 m
    errs = {}
    for dt in (1e-3, 5e-4):
        nt = int(round(T / dt))
        g = fwi.Geom(n, n, dx, dt, nt, [c], [c], [c] * 3, rec_ix)
        tr = fwi.forward(np.full((n, n), v0), g, 0)
        e = []
        for k, ix in enumerate(rec_ix):
            ua = _green_trace(dt, nt, (ix - c) * dx, v0, g.f0, g.t0)
            e.append(np.linalg.norm(tr[k] - ua) / np.linalg.norm(ua))
        errs[dt] = np.array(e)
    # the time-discretisation phase error grows with the travel distance
    assert np.all(errs[1e-3] < 1e-2), errs
    assert np.all(errs[5e-4] < 2.5e-3), errs
    ratio = errs[1e-3] / errs[5e-4]
    assert np.all((ratio > 3.0) & (ratio < 5.0)), ratio


def test_adjoint_dot_product():
    g = _small_geom(nz=20, nx=26, nt=120, nrec=7)
    v = _small_model(g.nz, g.nx)
    rng = np.random.default_rng(11)
    q = rng.standard_normal(g.nt)
    r = rng.standard_normal((g.nrec, g.nt))
    src = (g.src_iz[0], g.src_ix[0])
    Fq = fwi.propagate(v, g, src, q)
    Ftr = fwi.source_adjoint(v, g, src, r)
    lhs = float(np.sum(Fq * r))
    rhs = float(np.sum(q * Ftr))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def _problem(seed=3):
    g = _small_geom()
    v_true = _small_model(g.nz, g.nx, seed=seed)
    d_obs = np.stack([fwi.forward(v_true, g, s) for s in range(g.nsrc)])
    sigma = 0.05 * float(np.sqrt(np.mean(d_obs ** 2)))
    v0 = v_true + np.random.default_rng(seed + 1).uniform(-60, 60, v_true.shape)
    return g, v_true, d_obs, sigma, v0


def _J(v, g, d_obs, sigma):
    return sum(fwi.misfit(fwi.forward(v, g, s), d_obs[s], sigma)
               for s in range(g.nsrc))


def test_misfit_is_zero_at_true_model():
    g, v_true, d_obs, sigma, _ = _problem()
    assert _J(v_true, g, d_obs, sigma) == 0.0
    J, grad = fwi.gradient(v_true, g, d_obs, sigma)
    assert J == 0.0 and np.all(grad == 0.0)


def test_gradient_taylor_remainder_is_second_order():
    g, _, d_obs, sigma, v0 = _problem()
    J0, grad = fwi.gradient(v0, g, d_obs, sigma)
    assert abs(J0 - _J(v0, g, d_obs, sigma)) <= 1e-12 * J0
    dv = np.random.default_rng(9).standard_normal(v0.shape) * 20.0
    hs = np.array([1.0, 0.5, 0.25, 0.125])
    rem = np.array([abs(_J(v0 + h * dv, g, d_obs, sigma) - J0
                        - h * np.sum(grad * dv)) for h in hs])
    slopes = np.log(rem[:-1] / rem[1:]) / np.log(2.0)
    assert np.all(np.abs(slopes - 2.0) < 0.1), slopes


def test_gradient_central_differences_per_cell():
    g, _, d_obs, sigma, v0 = _problem()
    _, grad = fwi.gradient(v0, g, d_obs, sigma)
    rng = np.random.default_rng(21)
    cells = {(0, 0), (0, g.nx - 1), (g.nz - 1, 0), (g.nz - 1, g.nx - 1),
             (0, g.nx // 2), (g.nz - 1, g.nx // 3), (g.nz // 2, 0),
             (g.nz // 3, g.nx - 1)}
    while len(cells) < 32:
        cells.add((int(rng.integers(g.nz)), int(rng.integers(g.nx))))
    # h = 1e-2 m/s balances the O(h^2) truncation against FP64 round-off of J
    h = 1e-2
    scale = np.abs(grad).max()
    for (i, j) in sorted(cells):
        vp = v0.copy()
        vm = v0.copy()
        vp[i, j] += h
        vm[i, j] -= h
        fd = (_J(vp, g, d_obs, sigma) - _J(vm, g, d_obs, sigma)) / (2 * h)
        assert abs(fd - grad[i, j]) <= 1e-6 * max(abs(grad[i, j]),
                                                  1e-3 * scale), (i, j, fd,
                                                                  grad[i, j])


def test_two_imaging_condition_forms_agree():
    g, _, d_obs, sigma, v0 = _problem()
    _, _, gp1, gp2 = fwi.pair_gradient(
        v0, g, 0, lambda tr: (tr - d_obs[0]) / sigma ** 2, both_forms=True)
    assert np.linalg.norm(gp1 - gp2) <= 1e-12 * np.linalg.norm(gp1)


def test_fold_is_transpose_of_padding():
    g = _small_geom(nz=7, nx=9)
    rng = np.random.default_rng(4)
    v = rng.standard_normal((g.nz, g.nx))
    u = rng.standard_normal((g.NZ, g.NX))
    lhs = np.sum(fwi.pad_model(v, g.nb) * u)
    rhs = np.sum(v * fwi.fold(u, g))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_upstream_adjoint_is_derivative_of_traces():
    g = _small_geom(nt=100)
    v = _small_model(g.nz, g.nx)
    rng = np.random.default_rng(8)
    dseis = rng.standard_normal((g.nsrc, g.nrec, g.nt))
    dv = rng.standard_normal(v.shape) * 10.0
    grad = fwi.adjoint_of_upstream(v, g, dseis)
    h = 1e-3

    def L(vv):
        return sum(np.sum(fwi.forward(vv, g, s) * dseis[s])
                   for s in range(g.nsrc))
    fd = (L(v + h * dv) - L(v - h * dv)) / (2 * h)
    an = np.sum(grad * dv)
    assert abs(fd - an) <= 1e-7 * abs(an)


def test_taper_and_stencil_constants():
    # Cerjan factor: 1 inside, exp(-(0.015*20)^2) at the outer edge.
    g = fwi.taper(50, 60, 20, 0.015)
    assert g[25, 30] == 1.0
    assert np.isclose(g[0, 30], np.exp(-0.09))
    assert np.isclose(g[0, 0], np.exp(-0.18))
    # The 8th-order stencil is exact on polynomials up to degree 9:
    # lap(x^2 + z^2) = 4 away from the zero ring.
    n = 30
    z, x = np.meshgrid(np.arange(n) * 10.0, np.arange(n) * 10.0, indexing="ij")
    lap = fwi.laplacian(x ** 2 + z ** 2, 10.0)
    assert np.allclose(lap[4:-4, 4:-4], 4.0, rtol=0, atol=1e-9)
    lap8 = fwi.laplacian(x ** 8, 10.0)
    assert np.allclose(lap8[4:-4, 4:-4], 56.0 * x[4:-4, 4:-4] ** 6,
                       rtol=1e-10, atol=1e-3)


def test_source_minibatch_sums_and_unbiased_scaling():
    """The minibatch gradient is the sum over its sources: a partition of the
    sources adds up to the full misfit and gradient, and (S / nb) times the
    minibatch value averaged over every subset of nb sources is the full
    value (the unbiased stochastic gradient of Sec. 3)."""
    import itertools
    g = _small_geom(nsrc=4, nt=120)
    v_true = _small_model(g.nz, g.nx)
    d_obs = fwi.seismograms(v_true[None], g)[0]
    v = v_true + 30.0
    J, G = fwi.gradient(v, g, d_obs, 1.0)
    Ja, Ga = fwi.gradient(v, g, d_obs, 1.0, sources=[0, 3])
    Jb, Gb = fwi.gradient(v, g, d_obs, 1.0, sources=[2, 1])
    assert np.isclose(Ja + Jb, J, rtol=1e-12)
    assert np.allclose(Ga + Gb, G, rtol=1e-10, atol=1e-12 * np.abs(G).max())
    nb = 2
    subsets = list(itertools.combinations(range(4), nb))
    per = {s: fwi.gradient(v, g, d_obs, 1.0, sources=[s]) for s in range(4)}
    Jm = np.mean([(4 / nb) * sum(per[s][0] for s in B) for B in subsets])
    Gm = np.mean([(4 / nb) * sum(per[s][1] for s in B) for B in subsets], axis=0)
    assert np.isclose(Jm, J, rtol=1e-12)
    assert np.allclose(Gm, G, rtol=1e-10, atol=1e-12 * np.abs(G).max())


def test_gradient_magnitude_bounds_and_symmetries():
    """The per-cell sum of the imaging terms' magnitudes: it bounds |dJ/dv|
    (triangle inequality) and the sum of the per-source magnitudes is the
    magnitude over all sources; flipping the sign of the adjoint source flips
    the gradient but leaves the magnitude unchanged (each term is linear in
    the adjoint field), and scaling sigma by 2 scales both by 1/4."""
    g, _, d_obs, sigma, v0 = _problem()
    J, G = fwi.gradient(v0, g, d_obs, sigma)
    M = fwi.gradient_magnitude(v0, g, d_obs, sigma)
    assert np.all(M >= np.abs(G) * (1 - 1e-12))
    assert M.sum() > 1.01 * np.abs(G).sum()          # the time sum cancels
    parts = sum(fwi.gradient_magnitude(v0, g, d_obs, sigma, sources=[s])
                for s in range(g.nsrc))
    assert np.allclose(parts, M, rtol=1e-12, atol=0)
    f = lambda tr: (tr - d_obs[0]) / sigma ** 2
    _, g1, m1 = fwi.pair_gradient(v0, g, 0, f, magnitude=True)
    _, g2, m2 = fwi.pair_gradient(v0, g, 0, lambda tr: -f(tr), magnitude=True)
    assert np.allclose(g2, -g1, rtol=1e-12, atol=0)
    assert np.allclose(m2, m1, rtol=1e-12, atol=0)
    M2 = fwi.gradient_magnitude(v0, g, d_obs, 2 * sigma)
    assert np.allclose(M2, M / 4, rtol=1e-12, atol=0)
