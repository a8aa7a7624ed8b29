"""GPU parity of the travel-time tomography path (Sec. 4.1) against the FP64
oracle, through the C ABI.

Tolerances. The device relaxes the same upwind equations in FP32; each
travel time is a chain of at most a few hundred node updates, each rounded
once, so times agree to TOL_T = 4e-6 relative (an FP32 emulation of the
relaxation with exact square roots stays within 2.1e-7; the device's
q * rsqrt(q) adds a few 1e-7 per update, relative to that update's
increment only). The misfit then differs by at most
sum_i |res_i| TOL_T T_i / sigma_i^2 plus FP32 rounding of the residuals.
Ray gradients move continuously with the travel times (the traced field is
interpolated from nodal gradients, so a perturbation shifts a ray without
switching cells abruptly): an FP32 emulation of the tracer stays within
1.5e-6 of max |dJ/dv| on the small grid and 7.6e-6 on the full one, and
the oracle itself moves by 3.4e-6 under a 1e-6 relative change of the
velocities; the bound is TOL_G = 2e-4 max |dJ/dv|.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth.tomo as st
from oracle import tomo as otomo
import paper_2310_13325_gb300 as vg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL_T = 4e-6
TOL_G = 2e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_13325_gb300 import build
    build.build()


def _t(a, dtype=torch.float32):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


def _case(cfg, P, kind, seed=2, sta=None):
    """FP32-rounded inputs (the oracle sees exactly what the device sees)."""
    sta = st.stations(cfg) if sta is None else np.asarray(sta, dtype=np.int32)
    cfg = cfg.with_(n_stations=len(sta))
    sig = st.pair_sigma(cfg, sta).astype(np.float32).astype(np.float64)
    d = otomo.traveltimes(st.true_group_velocity(cfg), cfg.h, sta)
    d = (d + sig * st.unit_noise(d.size)).astype(np.float32).astype(np.float64)
    gen = st.smooth_particles if kind == "smooth" else st.particles_from_prior
    V = gen(cfg, P, seed=seed).astype(np.float32).astype(np.float64)
    return cfg, sta, sig, d, V


def _check_times(Tg, To):
    err = np.abs(Tg - To)
    assert np.all(err <= TOL_T * To + 1e-9), float(np.max(err / To))


def _check_gradient(cfg, sta, sig, d, V, Jg, Gg, Tg, rows):
    h = np.float32(cfg.h).astype(np.float64)      # the device's spacing
    for row, p in enumerate(rows):
        v = V[p].reshape(cfg.ny, cfg.nx)
        To = otomo.traveltimes(v, h, sta)
        Jo, go = otomo.misfit_gradient(v, h, sta, d, sig)
        _check_times(Tg[row], To)
        res = np.abs(To - d)
        bound = np.sum(res * TOL_T * To / sig ** 2) + 1e-6 * Jo
        assert abs(Jg[row] - Jo) <= bound, (Jg[row], Jo, bound)
        gmax = np.max(np.abs(go))
        assert np.max(np.abs(Gg[row].reshape(-1) - go.reshape(-1))) <= TOL_G * gmax


@pytest.mark.parametrize("kind", ["smooth", "prior"])
def test_traveltimes_match_fast_marching(kind):
    cfg, sta, sig, d, V = _case(st.tomo_config("tomo_small"), 4, kind)
    tm = vg.Tomo.from_config(cfg, sta)
    T = tm.traveltimes(_t(V)).cpu().numpy()
    assert tm.last_status() == 0
    h = np.float32(cfg.h).astype(np.float64)
    for p in range(len(V)):
        _check_times(T[p], otomo.traveltimes(V[p].reshape(cfg.ny, cfg.nx), h, sta))


@pytest.mark.parametrize("kind", ["smooth", "prior"])
def test_gradient_matches_the_ray_oracle(kind):
    cfg, sta, sig, d, V = _case(st.tomo_config("tomo_small"), 4, kind, seed=3)
    tm = vg.Tomo.from_config(cfg, sta)
    T = torch.empty((len(V), tm.n_pairs), device=DEV)
    J, G = tm.gradient(_t(V), _t(d), _t(sig), T=T)
    assert tm.last_status() == 0
    _check_gradient(cfg, sta, sig, d, V, J.cpu().numpy(), G.cpu().numpy(),
                    T.cpu().numpy(), range(len(V)))
    # the times the gradient call reports are the forward call's
    T2 = tm.traveltimes(_t(V)).cpu().numpy()
    np.testing.assert_allclose(T.cpu().numpy(), T2, rtol=1e-6)


def test_full_size_batch_on_sampled_particles():
    # the benchmark's launch: 500 prior particles, 40 x 37 nodes, 61 stations
    cfg, sta, sig, d, V = _case(st.tomo_config("tomo_uk"), 500, "prior")
    tm = vg.Tomo.from_config(cfg, sta)
    T = torch.empty((len(V), tm.n_pairs), device=DEV)
    J, G = tm.gradient(_t(V), _t(d), _t(sig), T=T)
    assert tm.last_status() == 0
    rows = [0, 499]
    Jh, Gh, Th = J.cpu().numpy(), G.cpu().numpy(), T.cpu().numpy()
    _check_gradient(cfg, sta, sig, d, V, Jh[rows], Gh[rows], Th[rows], rows)
    assert np.all(np.isfinite(Jh)) and np.all(np.isfinite(Gh))


def test_grid_beyond_the_register_slots():
    # more than 2 x 3 x 256 nodes: the relaxation's general loop
    cfg, sta, sig, d, V = _case(st.tomo_config("tomo_small").with_(ny=48, nx=50,
                                                                   n_stations=5), 2, "smooth")
    tm = vg.Tomo.from_config(cfg, sta)
    T = torch.empty((len(V), tm.n_pairs), device=DEV)
    J, G = tm.gradient(_t(V), _t(d), _t(sig), T=T)
    assert tm.last_status() == 0
    _check_gradient(cfg, sta, sig, d, V, J.cpu().numpy(), G.cpu().numpy(),
                    T.cpu().numpy(), range(len(V)))


def test_source_minibatch_matches_the_oracle_and_partitions():
    cfg, sta, sig, d, V = _case(st.tomo_config("tomo_small"), 3, "smooth", seed=4)
    tm = vg.Tomo.from_config(cfg, sta)
    h = np.float32(cfg.h).astype(np.float64)
    Vt, dt, st_ = _t(V), _t(d), _t(sig)
    parts = ([0, 3, 6], [1, 2, 4, 5, 7])
    Jf, Gf = tm.gradient(Vt, dt, st_)
    Jf, Gf = Jf.cpu().numpy(), Gf.cpu().numpy().reshape(len(V), -1)
    Js, Gs = 0.0, 0.0
    ns = cfg.n_stations
    To = [otomo.traveltimes(v.reshape(cfg.ny, cfg.nx), h, sta) for v in V]
    for part in parts:
        J, G = tm.gradient(Vt, dt, st_, sources=part)
        assert tm.last_status() == 0
        J, G = J.cpu().numpy(), G.cpu().numpy().reshape(len(V), -1)
        mine = [otomo.pair_index(s, r, ns) for s in part for r in range(s + 1, ns)]
        for p in range(len(V)):
            Jo, go = otomo.misfit_gradient(V[p].reshape(cfg.ny, cfg.nx), h, sta, d, sig,
                                           sources=part)
            t = To[p][mine]
            bound = np.sum(np.abs(t - d[mine]) * TOL_T * t / sig[mine] ** 2) + 1e-6 * Jo
            assert abs(J[p] - Jo) <= bound
            assert np.max(np.abs(G[p] - go.reshape(-1))) <= TOL_G * np.max(np.abs(go))
        Js, Gs = Js + J, Gs + G
    # the same per-source work, summed in another grouping: FP32 atomics only
    np.testing.assert_allclose(Js, Jf, rtol=1e-12)
    assert np.max(np.abs(Gs - Gf)) <= 1e-5 * np.max(np.abs(Gf))
    with pytest.raises(vg.VipError):
        tm.gradient(Vt, dt, st_, sources=[0, 0])
    with pytest.raises(vg.VipError):
        tm.gradient(Vt, dt, st_, sources=[cfg.n_stations - 1])


def test_edge_stations_minimal_grid_and_empty_batch():
    # stations on corners and edges, adjacent stations, the smallest grid
    base = st.tomo_config("tomo_small")
    for ny, nx, sta in ((2, 3, [0, 5, 1]), (7, 2, [0, 13, 6, 7]),
                        (9, 10, [0, 9, 80, 89, 44, 45, 54])):
        cfg, sta, sig, d, V = _case(base.with_(ny=ny, nx=nx), 3, "prior", sta=sta)
        tm = vg.Tomo.from_config(cfg, sta)
        T = torch.empty((len(V), tm.n_pairs), device=DEV)
        J, G = tm.gradient(_t(V), _t(d), _t(sig), T=T)
        assert tm.last_status() == 0
        _check_gradient(cfg, sta, sig, d, V, J.cpu().numpy(), G.cpu().numpy(),
                        T.cpu().numpy(), range(len(V)))
    out = tm.traveltimes(torch.empty((0, cfg.ny * cfg.nx), device=DEV))
    assert out.shape == (0, tm.n_pairs)


def test_invalid_arguments_and_velocity_flag():
    with pytest.raises(vg.VipError):
        vg.Tomo(5, 5, 1.0, [3, 3])                 # repeated station
    with pytest.raises(vg.VipError):
        vg.Tomo(5, 5, 1.0, [0, 25])                # outside the grid
    with pytest.raises(vg.VipError):
        vg.Tomo(1, 5, 1.0, [0, 1])                 # grid too small
    tm = vg.Tomo(6, 7, 10.0, [8, 33])
    v = torch.full((1, 42), 3.0, device=DEV)
    v[0, 20] = 0.0                                 # flagged, stays in bounds
    tm.traveltimes(v)
    assert tm.last_status() == -1
    tm.traveltimes(torch.full((1, 42), 3.0, device=DEV))
    assert tm.last_status() == 0
