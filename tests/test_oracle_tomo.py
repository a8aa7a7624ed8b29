"""Pins of the tomography oracle (Sec. 4.1) to facts outside itself: closed
forms of the first-order upwind eikonal scheme, the discrete equations
written from their definition, convergence to analytic travel times,
scaling and symmetry laws, and finite differences of the misfit."""
import numpy as np
import pytest

import synth.tomo as st
from oracle import tomo


def _residual_of_definition(T, v, h, src):
    """|((t-a)^+)^2 + ((t-b)^+)^2 - f^2| / f^2 at every node but the source,
    a and b the smaller neighbour times along x and y (all neighbours)."""
    ny, nx = T.shape
    worst = 0.0
    for i in range(ny):
        for j in range(nx):
            if (i, j) == src:
                continue
            a = min(T[i, m] for m in (j - 1, j + 1) if 0 <= m < nx)
            b = min(T[m, j] for m in (i - 1, i + 1) if 0 <= m < ny)
            f = h / v[i, j]
            t = T[i, j]
            lhs = max(t - a, 0.0) ** 2 + max(t - b, 0.0) ** 2
            worst = max(worst, abs(lhs - f * f) / (f * f))
    return worst


def test_pair_index_is_a_bijection():
    ns = 7
    idx = [tomo.pair_index(s, r, ns) for s in range(ns) for r in range(s + 1, ns)]
    assert idx == list(range(ns * (ns - 1) // 2))


def test_uniform_medium_is_exact_along_the_axes():
    # the first-order scheme propagates exactly along grid lines
    v = np.full((15, 17), 3.0)
    h = 2.5
    T = tomo.fast_marching(v, h, (7, 8))
    for j in range(17):
        assert T[7, j] == pytest.approx(abs(j - 8) * h / 3.0, rel=1e-14, abs=1e-14)
    for i in range(15):
        assert T[i, 8] == pytest.approx(abs(i - 7) * h / 3.0, rel=1e-14, abs=1e-14)


def test_first_diagonal_node_closed_form():
    # both neighbours at f: t = f (1 + 1/sqrt 2)
    v = np.full((9, 9), 2.0)
    T = tomo.fast_marching(v, 1.0, (4, 4))
    f = 0.5
    for di, dj in ((1, 1), (-1, 1), (1, -1), (-1, -1)):
        assert T[4 + di, 4 + dj] == pytest.approx(f * (1 + 1 / np.sqrt(2)), rel=1e-14)


@pytest.mark.parametrize("kind", ["smooth", "rough"])
def test_fast_marching_solves_the_discrete_equations(kind):
    rng = np.random.default_rng(11)
    cfg = st.tomo_config("tomo_small")
    if kind == "smooth":
        v = st.smooth_particles(cfg, 1, seed=4)[0].reshape(cfg.ny, cfg.nx)
    else:
        v = np.exp(rng.uniform(np.log(1.5), np.log(5.0), size=(cfg.ny, cfg.nx)))
    src = (5, 13)
    T = tomo.fast_marching(v, cfg.h, src)
    assert T[src] == 0.0 and np.all(np.isfinite(T))
    assert _residual_of_definition(T, v, cfg.h, src) < 1e-12


def test_scaling_law():
    # T is homogeneous of degree -1 in v and degree 1 in h
    cfg = st.tomo_config("tomo_small")
    v = st.smooth_particles(cfg, 1, seed=5)[0].reshape(cfg.ny, cfg.nx)
    T = tomo.fast_marching(v, cfg.h, (3, 4))
    T2 = tomo.fast_marching(2.0 * v, 3.0 * cfg.h, (3, 4))
    np.testing.assert_allclose(T2, 1.5 * T, rtol=1e-13)


def test_converges_to_euclidean_distance():
    # uniform medium: error at fixed points shrinks with refinement
    errs = []
    for N in (21, 41, 81):
        L = 100.0
        h = L / (N - 1)
        T = tomo.fast_marching(np.full((N, N), 3.0), h, (0, 0))
        errs.append(abs(T[-1, -1] * 3.0 / np.hypot(L, L) - 1.0))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.015 and errs[1] / errs[2] > 1.4


def test_converges_in_a_constant_gradient_medium():
    # v = v0 + g y has T = arccosh(1 + g^2 r^2 / (2 v(src) v(x))) / g
    means = []
    for N in (21, 41, 81):
        L = 100.0
        h = L / (N - 1)
        y = np.arange(N) * h
        v0, g = 2.0, 0.02
        v = np.repeat((v0 + g * y)[:, None], N, axis=1)
        src = (0, N // 2)
        T = tomo.fast_marching(v, h, src)
        Y, X = np.meshgrid(y, np.arange(N) * h, indexing="ij")
        r2 = (X - X[src]) ** 2 + Y ** 2
        exact = np.arccosh(1 + g * g * r2 / (2 * v0 * (v0 + g * Y))) / g
        far = r2 > (L / 4) ** 2
        means.append(np.mean(np.abs(T[far] - exact[far]) / exact[far]))
    assert means[0] > means[1] > means[2]
    assert means[2] < 0.02


def test_ray_in_uniform_medium_runs_along_the_row():
    ny, nx, h, v0 = 11, 30, 4.0, 2.5
    v = np.full((ny, nx), v0)
    src, rcv = (5, 3), (5, 26)
    T = tomo.fast_marching(v, h, src)
    segs = tomo.trace_ray(T, src, rcv)
    assert all(p[0] == 5.0 and q[0] == 5.0 for p, q in segs)
    K = tomo.ray_sensitivity(segs, ny, nx)
    assert K.sum() == pytest.approx(23.0, rel=1e-13)
    assert np.all(K[np.arange(ny) != 5] == 0.0)
    # Euler's relation for T(v) homogeneous of degree -1: sum v dT/dv = -T
    dTdv = -h * K / (v * v)
    assert np.sum(v * dTdv) == pytest.approx(-T[rcv], rel=1e-13)


def test_ray_slowness_integral_matches_the_travel_time():
    # the ray's slowness integral approximates the eikonal time
    cfg = st.tomo_config("tomo_small")
    sta = st.stations(cfg)
    v = st.smooth_particles(cfg, 1, seed=6)[0].reshape(cfg.ny, cfg.nx)
    errs = []
    for s in range(3):
        src = divmod(int(sta[s]), cfg.nx)
        T = tomo.fast_marching(v, cfg.h, src)
        for r in range(s + 1, cfg.n_stations):
            rcv = divmod(int(sta[r]), cfg.nx)
            K = tomo.ray_sensitivity(tomo.trace_ray(T, src, rcv), cfg.ny, cfg.nx)
            errs.append(np.sum(cfg.h * K / v) / T[rcv] - 1.0)
    errs = np.abs(errs)
    assert errs.max() < 0.15 and errs.mean() < 0.06


def test_perfect_data_have_zero_misfit_and_gradient():
    cfg = st.tomo_config("tomo_small").with_(n_stations=5)
    sta = st.stations(cfg)
    v = st.smooth_particles(cfg, 1, seed=7)[0].reshape(cfg.ny, cfg.nx)
    d = tomo.traveltimes(v, cfg.h, sta)
    J, g = tomo.misfit_gradient(v, cfg.h, sta, d, st.pair_sigma(cfg, sta))
    assert J == 0.0 and np.all(g == 0.0)


def test_ray_gradient_follows_finite_differences():
    # the ray gradient approximates the derivative of the discrete misfit:
    # same direction, a sign or transposition error would break it
    cfg = st.tomo_config("tomo_small").with_(ny=9, nx=11, n_stations=5)
    sta = st.stations(cfg)
    sig = st.pair_sigma(cfg, sta)
    d = tomo.traveltimes(st.true_group_velocity(cfg), cfg.h, sta)
    v = st.smooth_particles(cfg, 1, seed=8)[0].reshape(cfg.ny, cfg.nx)
    J, g = tomo.misfit_gradient(v, cfg.h, sta, d, sig)

    def misfit(vv):
        t = tomo.traveltimes(vv, cfg.h, sta)
        return 0.5 * np.sum(((t - d) / sig) ** 2)

    assert J == pytest.approx(misfit(v), rel=1e-13)
    fd = np.zeros_like(v)
    eps = 1e-5
    for i in range(cfg.ny):
        for j in range(cfg.nx):
            e = np.zeros_like(v)
            e[i, j] = eps
            fd[i, j] = (misfit(v + e) - misfit(v - e)) / (2 * eps)
    cos = np.sum(fd * g) / (np.linalg.norm(fd) * np.linalg.norm(g))
    assert cos > 0.85
    assert np.linalg.norm(g) / np.linalg.norm(fd) == pytest.approx(1.0, abs=0.35)


def test_source_minibatches_partition_the_misfit_and_gradient():
    # a partition of the source stations adds up to the full sums, and the
    # (ns - 1) / nb scaled minibatch averaged over all subsets is the full value
    import itertools
    cfg = st.tomo_config("tomo_small").with_(ny=10, nx=12, n_stations=5)
    sta = st.stations(cfg)
    sig = st.pair_sigma(cfg, sta)
    d = tomo.traveltimes(st.true_group_velocity(cfg), cfg.h, sta)
    v = st.smooth_particles(cfg, 1, seed=9)[0].reshape(cfg.ny, cfg.nx)
    J, g = tomo.misfit_gradient(v, cfg.h, sta, d, sig)
    J1, g1 = tomo.misfit_gradient(v, cfg.h, sta, d, sig, sources=[0, 2])
    J2, g2 = tomo.misfit_gradient(v, cfg.h, sta, d, sig, sources=[1, 3])
    assert J1 + J2 == pytest.approx(J, rel=1e-13)
    np.testing.assert_allclose(g1 + g2, g, rtol=1e-12, atol=1e-12 * np.abs(g).max())
    S, nb = cfg.n_stations - 1, 2
    subsets = list(itertools.combinations(range(S), nb))
    Jm = np.mean([tomo.misfit_gradient(v, cfg.h, sta, d, sig, sources=list(c))[0]
                  for c in subsets]) * S / nb
    assert Jm == pytest.approx(J, rel=1e-12)


def test_rays_converge_to_the_circular_ray_of_a_constant_gradient_medium():
    # in v = v0 + g y every ray is a circular arc centred at depth -v0/g;
    # two surface stations 40 km apart: radius sqrt(20^2 + (v0/g)^2)
    v0, g = 2.0, 0.05
    cx, cy = 40.0, -v0 / g
    R = np.hypot(20.0, cy)
    rms = []
    for N, h in ((41, 2.0), (81, 1.0), (161, 0.5)):
        v = np.repeat((v0 + g * np.arange(N) * h)[:, None], N, axis=1)
        src, rcv = (0, int(20 / h)), (0, int(60 / h))
        segs = tomo.trace_ray(tomo.fast_marching(v, h, src), src, rcv)
        pts = np.array([p for p, q in segs] + [segs[-1][1]]) * h
        d = np.hypot(pts[:, 1] - cx, pts[:, 0] - cy) - R
        rms.append(np.sqrt(np.mean(d * d)))
        assert pts[:, 0].max() < R + cy + 0.5        # never below the true turning depth
    assert rms[0] > rms[1] > rms[2] and rms[2] < 0.5
