"""GPU parity of the FWI path (fwi_forward, fwi_gradient, fwi_adjoint) against
the FP64 oracle, through the C ABI.

Tolerances: relative L2 <= 1e-5 for FP32 traces and gradients driven by data
residuals. The misfit (Eq. 26) rounds each residual to FP32 once (2^-24), sums
the squares of each receiver's residuals in FP32 over blocks of 16 steps
(relative error <= 16 * 2^-24 ~ 1e-6) and accumulates those block sums per
receiver in FP64, then over receivers in a fixed order: the reduction is held
to its rounding bound, 18 * 2^-24 ~ 1.07e-6 (MISFIT_REDUCTION_TOL = 1.1e-6),
against an FP64 sum of the same GPU traces, and its value against the oracle to
a tolerance derived per case from the trace tolerance: dJ/J ~ 2 <r, dd> / |r|^2
<= 2 (|d| / |r|) rel(d) + 1.1e-6, |d| / |r| measured on the oracle's traces
(misfit_tolerance).
Reduced-precision snapshots are measured and held to the bounds stated with
each test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle import fwi as ofwi
import paper_2310_13325_gb300 as vg
from gpu_common import (MISFIT_REDUCTION_TOL, cfg1_case, cfg1_oracle_gradients,
                        misfit_tolerance, odd_config, oracle_gradients, problem, rel)

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a, dtype=torch.float32):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


def _cfg1_jtol(P=2):
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(P)
    return misfit_tolerance(ofwi.seismograms(V, g), d_obs)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_13325_gb300 import build
    build.build()


def test_forward_traces_match_oracle_cfg1():
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(2)
    ref = ofwi.seismograms(V, g)
    fwi = vg.Fwi.from_config(cfg, geo)
    out = fwi.forward(_t(V)).cpu().numpy()
    assert out.shape == ref.shape
    for p in range(2):
        for s in range(g.nsrc):
            assert rel(out[p, s], ref[p, s]) <= 1e-5, (p, s, rel(out[p, s], ref[p, s]))
    assert fwi.last_status() == 0


def test_gradient_and_misfit_match_oracle_cfg1():
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(2)
    J_ref, G_ref = cfg1_oracle_gradients(2)
    fwi = vg.Fwi.from_config(cfg, geo)
    J, G = fwi.gradient(_t(V), _t(d_obs), sigma)
    J = J.cpu().numpy()
    G = G.reshape(2, -1).cpu().numpy()
    for p in range(2):
        assert rel(G[p], G_ref[p]) <= 1e-5, rel(G[p], G_ref[p])
    jtol = _cfg1_jtol()
    print("misfit rel. error %s, tolerance %.2e" % (np.abs(J - J_ref) / J_ref, jtol))
    assert np.all(np.abs(J - J_ref) <= jtol * np.abs(J_ref)), (J, J_ref)
    # the reduction itself, on the GPU's own traces, against an FP64 sum
    tr = fwi.forward(_t(V)).double().cpu().numpy()
    J_host = 0.5 * ((tr - d_obs.astype(np.float32)[None]) ** 2).sum(axis=(1, 2, 3)) / sigma ** 2
    print("misfit reduction rel. error:", np.abs(J - J_host) / J_host)
    assert np.all(np.abs(J - J_host) <= MISFIT_REDUCTION_TOL * J_host), (J, J_host)


def test_plain_loop_equals_batched_bit_for_bit():
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(2)
    fwi = vg.Fwi.from_config(cfg, geo)
    Vt, Dt = _t(V), _t(d_obs)
    # one cluster per particle (all sources in one work item) accumulates the
    # sources in the same order as the plain loop
    fwi.set_plan(0, 0, 0, g.nsrc)
    Jb, Gb = fwi.gradient(Vt, Dt, sigma)
    Sb = fwi.forward(Vt)
    fwi.set_mode(vg.FWI_MODE_PLAIN, 1)
    Jp, Gp = fwi.gradient(Vt, Dt, sigma)
    Sp = fwi.forward(Vt)
    assert torch.equal(Sb, Sp)
    assert torch.equal(Gb, Gp)
    # same FP32 residuals, whose squares the plain loop adds in FP64; the
    # batched kernel sums them in FP32 over 16 steps per receiver before the
    # FP64 accumulation (bound 16 * 2^-24, within MISFIT_REDUCTION_TOL)
    print("batched / plain misfit rel. difference:", ((Jb - Jp).abs() / Jp).tolist())
    assert torch.allclose(Jb, Jp, rtol=MISFIT_REDUCTION_TOL, atol=0)


@pytest.mark.parametrize("K", [7, 50])
def test_checkpoint_recompute_equals_store_all(K):
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(2)
    fwi = vg.Fwi.from_config(cfg, geo)
    Vt, Dt = _t(V), _t(d_obs)
    # all sources of a particle in one work item: the association the plain
    # loop uses (splitting the sources over clusters only reorders the sum)
    fwi.set_plan(0, 0, 0, g.nsrc)
    J1, G1 = fwi.gradient(Vt, Dt, sigma)
    G1 = G1.clone()
    fwi.set_mode(vg.FWI_MODE_BATCHED, K)
    JK, GK = fwi.gradient(Vt, Dt, sigma)
    assert torch.equal(G1, GK)
    assert torch.equal(J1, JK)
    fwi.set_mode(vg.FWI_MODE_PLAIN, K)
    Jp, Gp = fwi.gradient(Vt, Dt, sigma)
    assert torch.equal(G1, Gp)


def test_ragged_grid_every_launch_shape_agrees_with_oracle():
    cfg = odd_config()
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = problem(cfg, 3)
    J_ref, G_ref = ofwi.gradients(V, g, d_obs, sigma)
    jtol = misfit_tolerance(ofwi.seismograms(V, g), d_obs)
    fwi = vg.Fwi.from_config(cfg, geo)
    Vt, Dt = _t(V), _t(d_obs)
    base = None
    # (Q, V, T, coefficients: 1 shared memory, 2 global memory)
    shapes = [(1, 4, 0, 1), (2, 4, 0, 1), (3, 8, 0, 1), (5, 4, 64, 1), (7, 4, 0, 1),
              (2, 8, 96, 1), (1, 10, 0, 1), (2, 10, 96, 1), (4, 10, 0, 1),
              (1, 5, 0, 2), (3, 8, 0, 2), (4, 4, 64, 2), (2, 8, 96, 2)]
    for Q, Vr, T, co in shapes:
        fwi.set_plan(Q, Vr, T, coeff=co)
        plan = fwi.query_plan(3)
        assert plan["coefficients"] == ("global" if co == 2 else "shared")
        assert (plan["cluster_ctas"], plan["rows_per_thread"]) == (Q, Vr), plan
        J, G = fwi.gradient(Vt, Dt, sigma)
        G = G.reshape(3, -1).cpu().numpy()
        for p in range(3):
            assert rel(G[p], G_ref[p]) <= 1e-5, (Q, Vr, T, co, p, rel(G[p], G_ref[p]))
        assert np.all(np.abs(J.cpu().numpy() - J_ref) <= jtol * J_ref)
        # gradients and misfits do not depend on the launch shape
        if base is None:
            base, baseJ = G, J.cpu().numpy()
        else:
            assert np.array_equal(G, base), (Q, Vr, T, co)
            assert np.array_equal(J.cpu().numpy(), baseJ), (Q, Vr, T, co)


def test_autograd_backward_is_the_oracle_adjoint():
    """FwiSeis backward (fwi_adjoint) for the misfit's own upstream
    sensitivity equals fwi_gradient and the oracle to 1e-5. For a white-noise
    upstream sensitivity the imaging time sum cancels far more: with every
    term mu^k D^k held to a relative 1e-5 (the FP32 field bound), the gradient
    moves by at most 1e-5 of the sum of the terms' magnitudes M, i.e. a
    relative error of 1e-5 kappa with kappa = |M| / |G| from the oracle."""
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(2)
    J_ref, G_ref = cfg1_oracle_gradients(2)
    fwi = vg.Fwi.from_config(cfg, geo)
    v = _t(V).reshape(2, cfg.nz, cfg.nx).requires_grad_(True)
    seis = vg.FwiSeis.apply(v, fwi)
    loss = 0.5 * (((seis - _t(d_obs)[None]) / sigma) ** 2).sum()
    loss.backward()
    got = v.grad.reshape(2, -1).cpu().numpy()
    _, G = fwi.gradient(_t(V), _t(d_obs), sigma)
    G = G.reshape(2, -1).cpu().numpy()
    for p in range(2):
        assert rel(got[p], G_ref[p]) <= 1e-5, rel(got[p], G_ref[p])
        assert rel(got[p], G[p]) <= 1e-6, rel(got[p], G[p])
    rng = np.random.default_rng(12)
    dseis = rng.standard_normal((2, g.nsrc, g.nrec, g.nt))
    ref, mag = [], []
    for p in range(2):
        gp_ = np.zeros((cfg.nz, cfg.nx))
        mp_ = np.zeros((cfg.nz, cfg.nx))
        for s in range(g.nsrc):
            _, gs, ms = ofwi.pair_gradient(V[p].reshape(cfg.nz, cfg.nx), g, s,
                                           lambda tr, s=s, p=p: dseis[p, s], magnitude=True)
            gp_ += gs
            mp_ += ms
        ref.append(gp_.reshape(-1))
        mag.append(mp_.reshape(-1))
    v.grad = None
    seis = vg.FwiSeis.apply(v, fwi)
    (seis * _t(dseis)).sum().backward()
    got = v.grad.reshape(2, -1).cpu().numpy()
    for p in range(2):
        kappa = np.linalg.norm(mag[p]) / np.linalg.norm(ref[p])
        e = rel(got[p], ref[p])
        print("white-noise upstream, particle %d: rel-L2 %.2e, kappa %.1f, tolerance %.2e"
              % (p, e, kappa, 1e-5 * kappa))
        assert e <= 1e-5 * kappa, (p, e, kappa)


# The imaging condition sums products mu^k D^k in which only the stored
# snapshot D^k is rounded, by at most the format's unit roundoff u (2^-8 for
# BF16, 2^-11 for FP16), while mu and the FP32 forward sweep are unchanged. Per
# cell, dJ/dv therefore moves by at most u times the sum of the magnitudes of
# its imaging terms (M, from the oracle) plus the FP32 rounding of the two
# accumulations over N steps (2 N 2^-24 M) and of the result (2 2^-24 M); FP16
# values below the normal range after the per-block scaling carry an absolute
# error under 2^-39 of the block's largest value (slack 1e-7 max M). Against
# the oracle the gradient is stated, not gated: the time sum cancels, so the
# relative L2 error is not bounded by u.
@pytest.mark.parametrize("prec,u", [(vg.FWI_CKPT_BF16, 2.0 ** -8),
                                    (vg.FWI_CKPT_FP16, 2.0 ** -11)])
def test_reduced_precision_snapshots_error_is_bounded(prec, u):
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(2)
    J_ref, G_ref, M_ref, _ = oracle_gradients(g, V, range(g.nsrc), d_obs, sigma)
    fwi = vg.Fwi.from_config(cfg, geo)
    J32, G32 = fwi.gradient(_t(V), _t(d_obs), sigma)
    G32 = G32.reshape(2, -1).double().cpu().numpy()
    J, G = fwi.gradient(_t(V), _t(d_obs), sigma, precision=prec)
    G = G.reshape(2, -1).double().cpu().numpy()
    for p in range(2):
        bound = (u + (2 * cfg.nt + 2) * 2.0 ** -24) * M_ref[p] * 1.001 + 1e-7 * M_ref[p].max()
        print("snapshot precision %d, particle %d: gradient rel-L2 vs oracle %.2e; largest "
              "|G - G_fp32| / bound %.3f" % (prec, p, rel(G[p], G_ref[p]),
                                              (np.abs(G[p] - G32[p]) / bound).max()))
        assert np.all(np.abs(G[p] - G32[p]) <= bound)
    # the misfit comes from the FP32 forward sweep and is unaffected
    assert np.all(np.abs(J.cpu().numpy() - J_ref) <= _cfg1_jtol() * J_ref)
    # the same snapshots with the coefficients in global memory: identical
    # (a fresh context per layout, so no cached launch is shared between them)
    out = {}
    for co in (1, 2):
        f = vg.Fwi.from_config(cfg, geo)
        f.set_plan(2, 4, 0, g.nsrc, coeff=co)
        assert f.query_plan(2, prec)["coefficients"] == ("global" if co == 2 else "shared")
        Jc, Gc = f.gradient(_t(V), _t(d_obs), sigma, precision=prec)
        out[co] = (Jc.clone(), Gc.clone())
        f.close()
    assert torch.equal(out[1][1], out[2][1]) and torch.equal(out[1][0], out[2][0])


@pytest.mark.parametrize("K", [1, 9])
def test_global_coefficients_equal_shared_bit_for_bit(K):
    """w' and the gradient accumulator in global memory (the layout for
    large grids) give the same traces, misfits and gradients as the
    shared-memory layout, with and without restart checkpoints, and the
    adjoint-only mode agrees too."""
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(2)
    Vt, Dt = _t(V), _t(d_obs)
    out = {}
    for co in (1, 2):
        # a fresh context per layout: no cached launch is shared between them
        fwi = vg.Fwi.from_config(cfg, geo)
        fwi.set_mode(vg.FWI_MODE_BATCHED, K)
        fwi.set_plan(3, 8, 0, g.nsrc, coeff=co)
        assert fwi.query_plan(2)["coefficients"] == ("global" if co == 2 else "shared")
        S = fwi.forward(Vt).clone()
        J, G = fwi.gradient(Vt, Dt, sigma)
        J, G = J.clone(), G.clone()
        A = fwi.adjoint(Vt, S - Dt[None]).clone()
        out[co] = (S, J, G, A)
    for a, b in zip(out[1], out[2]):
        assert torch.equal(a, b)


def test_noise_free_data_give_zero_misfit_and_gradient():
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(2)
    fwi = vg.Fwi.from_config(cfg, geo)
    vt = _t(v_true)[None]
    clean = fwi.forward(vt)[0].contiguous()
    J, G = fwi.gradient(vt, clean, sigma)
    assert J.item() == 0.0
    assert torch.count_nonzero(G).item() == 0


def test_unstable_velocity_is_reported():
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(2)
    fwi = vg.Fwi.from_config(cfg, geo)
    v = torch.full((1, cfg.nz, cfg.nx), 6000.0, device=DEV)   # 6000 * 1e-3 / 10 = 0.6
    fwi.forward(v)
    assert fwi.last_status() == -2
    fwi.forward(_t(V))
    assert fwi.last_status() == 0


def test_single_particle_and_source_split_work_items():
    # P = 1 spreads the sources of one particle over several clusters
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(2)
    J_ref, G_ref = cfg1_oracle_gradients(2)
    fwi = vg.Fwi.from_config(cfg, geo)
    plan = fwi.query_plan(1)
    J, G = fwi.gradient(_t(V[:1]), _t(d_obs), sigma)
    assert rel(G.reshape(-1).cpu().numpy(), G_ref[0]) <= 1e-5
    assert abs(J.item() - J_ref[0]) <= _cfg1_jtol() * J_ref[0]
    assert plan["sources_per_item"] >= 1


def test_empty_batch_is_a_no_op():
    """P = 0 (a rank or a minibatch that holds no particles) returns VIP_OK with
    empty results from every FWI entry point, the P-sized pointers may be NULL,
    the other arguments are still checked, and the context computes normally
    afterwards."""
    import ctypes
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(2)
    J_ref, G_ref = cfg1_oracle_gradients(2)
    fwi = vg.Fwi.from_config(cfg, geo)
    v0 = torch.empty((0, cfg.nz, cfg.nx), device=DEV)
    dobs = _t(d_obs)
    assert tuple(fwi.forward(v0).shape) == (0, g.nsrc, g.nrec, g.nt)
    J, G = fwi.gradient(v0, dobs, sigma)
    assert tuple(J.shape) == (0,) and tuple(G.shape) == (0, cfg.nz, cfg.nx)
    J, G = fwi.gradient(v0, dobs, sigma, sources=[0, 2])
    assert tuple(J.shape) == (0,) and tuple(G.shape) == (0, cfg.nz, cfg.nx)
    dseis = torch.empty((0, g.nsrc, g.nrec, g.nt), device=DEV)
    assert tuple(fwi.adjoint(v0, dseis).shape) == (0, cfg.nz, cfg.nx)
    L, h = fwi._L, fwi._h
    src = (ctypes.c_int * 1)(1)
    assert L.fwi_forward(h, None, 0, None, None) == 0
    assert L.fwi_gradient(h, None, 0, None, sigma, None, None, 0, None) == 0
    assert L.fwi_gradient_sources(h, None, 0, None, sigma, ctypes.cast(src, ctypes.c_void_p), 1,
                                  None, None, 0, None) == 0
    assert L.fwi_adjoint(h, None, 0, None, None, 0, None) == 0
    assert L.fwi_forward(h, None, -1, None, None) == -1
    assert L.fwi_gradient(h, None, 0, None, -1.0, None, None, 0, None) == -1
    assert L.fwi_gradient(h, None, 0, None, sigma, None, None, 7, None) == -1
    assert L.fwi_gradient_sources(h, None, 0, None, sigma, None, 1, None, None, 0, None) == -1
    torch.cuda.synchronize()
    J, G = fwi.gradient(_t(V), dobs, sigma)
    assert rel(G.reshape(2, -1).cpu().numpy(), G_ref) <= 1e-5
    assert np.all(np.abs(J.cpu().numpy() - J_ref) <= _cfg1_jtol() * J_ref)
    assert fwi.last_status() == 0


def test_full_size_cfg3_sampled_traces_and_gradient_direction():
    """cfg3 grid (120 x 300, 2000 steps, 200 receivers) in the launch shape the
    benchmark uses: traces of sampled (particle, source) pairs against the
    oracle one by one, and the directional derivative of the misfit."""
    cfg = synth.config("cfg3")
    geo = synth.geometry(cfg)
    g = ofwi.Geom.from_config(cfg, geo)
    v_true = synth.true_model(cfg)
    lo, hi = synth.prior_bounds(cfg, v_true)
    V = synth.particles_from_prior(lo, hi, 2, seed=2)
    fwi = vg.Fwi.from_config(cfg, geo)
    seis = fwi.forward(_t(V))
    for p, s in ((0, 0), (1, 13)):
        ref = ofwi.forward(V[p].reshape(cfg.nz, cfg.nx), g, s)
        e = rel(seis[p, s].cpu().numpy(), ref)
        assert e <= 1e-5, (p, s, e)
    # directional derivative at full size (property check, any size)
    obs = fwi.forward(_t(v_true)[None])[0].contiguous()
    sigma = 1e-3
    v0 = _t(V[:1])
    J0, G0 = fwi.gradient(v0, obs, sigma)
    dv = torch.randn(v0.shape, generator=torch.Generator(device=DEV).manual_seed(3),
                     device=DEV) * 2.0
    h = 0.5
    Jp, _ = fwi.gradient(v0 + h * dv, obs, sigma)
    Jm, _ = fwi.gradient(v0 - h * dv, obs, sigma)
    fd = (Jp.item() - Jm.item()) / (2 * h)
    an = float((G0.reshape(-1).double() * dv.reshape(-1).double()).sum())
    assert abs(fd - an) <= 2e-3 * abs(an), (fd, an)


def test_largest_grid_sampled_traces_and_gradient_direction():
    """240 x 600 grid (280 x 640 padded), 3000 steps at 0.8 ms: the largest
    workload's geometry needs clusters beyond the portable size of 8 CTAs.
    Two sources, one particle: traces against the oracle, the linearisation
    dot product, and the plan for 2000 particles fits memory."""
    cfg = synth.config("cfg5").with_(nsrc=2)
    geo = synth.geometry(cfg)
    g = ofwi.Geom.from_config(cfg, geo)
    v_true = synth.true_model(cfg)
    lo, hi = synth.prior_bounds(cfg, v_true)
    V = synth.particles_from_prior(lo, hi, 1, seed=2)
    fwi = vg.Fwi.from_config(cfg, geo)
    seis = fwi.forward(_t(V))
    ref = ofwi.forward(V[0].reshape(cfg.nz, cfg.nx), g, 1)
    assert rel(seis[0, 1].cpu().numpy(), ref) <= 1e-5
    # linearisation dot product <J dv, r> = <dv, J^T r>: central difference of
    # the traces along a smooth perturbation dv (0.5 to 1.5 m/s) with h = 0.5.
    # A smooth dv moves every arrival coherently (phase shift near 2e-2 rad
    # over 2.4 s), so the FP32 noise of the two forward runs stays below 1e-3
    # of their difference and the O(h^2) term near 1e-4. (A white-noise dv
    # scatters incoherently: the trace change is then comparable to the FP32
    # noise and the check measures round-off, not the adjoint.)
    gen = torch.Generator(device=DEV).manual_seed(5)
    v0 = _t(V).reshape(1, cfg.nz, cfg.nx)
    zz = torch.arange(cfg.nz, device=DEV, dtype=torch.float32)[:, None] / cfg.nz
    xx = torch.arange(cfg.nx, device=DEV, dtype=torch.float32)[None, :] / cfg.nx
    dv = (1.0 + 0.5 * torch.sin(2 * np.pi * zz) * torch.cos(2 * np.pi * xx))[None]
    r = torch.randn((1, g.nsrc, g.nrec, g.nt), generator=gen, device=DEV)
    h = 0.5
    Jdv = (fwi.forward(v0 + h * dv) - fwi.forward(v0 - h * dv)).double() / (2 * h)
    lhs = float((Jdv * r.double()).sum())
    rhs = float((fwi.adjoint(v0, r).double() * dv.double()).sum())
    assert abs(lhs - rhs) <= 2e-3 * abs(rhs), (lhs, rhs)
    full = vg.Fwi.from_config(synth.config("cfg5"), synth.geometry(synth.config("cfg5")))
    plan = full.query_plan(2000)
    print("largest workload plan:", plan)
    assert plan["cluster_ctas"] >= 1 and plan["concurrent_pairs"] >= 1


def test_source_minibatch_gradient_matches_oracle():
    """fwi_gradient_sources: misfit and gradient summed over a minibatch of
    the sources (for sSVGD with stochastic gradients) against the oracle;
    two minibatches partitioning the sources add up to the full gradient;
    a full call after minibatch calls is unchanged (separate graphs)."""
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(2)
    fwi = vg.Fwi.from_config(cfg, geo)
    Vt, Dt = _t(V), _t(d_obs)
    J0, G0 = fwi.gradient(Vt, Dt, sigma)
    J0, G0 = J0.clone(), G0.clone()
    Ja, Ga = fwi.gradient(Vt, Dt, sigma, sources=[3, 1])
    Ja, Ga = Ja.clone(), Ga.clone()
    J_ref, G_ref = ofwi.gradients(V, g, d_obs, sigma, sources=[3, 1])
    Gh = Ga.reshape(2, -1).cpu().numpy()
    for p in range(2):
        assert rel(Gh[p], G_ref[p]) <= 1e-5, rel(Gh[p], G_ref[p])
    sub = np.stack([ofwi.seismograms(V, g)[:, s] for s in (3, 1)], axis=1)
    assert np.all(np.abs(Ja.cpu().numpy() - J_ref) <= misfit_tolerance(sub, d_obs[[3, 1]]) * J_ref)
    Jb, Gb = fwi.gradient(Vt, Dt, sigma, sources=[0, 2])
    Gs = (Ga + Gb).reshape(2, -1).cpu().numpy()
    Gf = G0.reshape(2, -1).cpu().numpy()
    for p in range(2):
        assert rel(Gs[p], Gf[p]) <= 1e-6
    assert np.allclose((Ja + Jb).cpu().numpy(), J0.cpu().numpy(), rtol=1e-6)
    J1, G1 = fwi.gradient(Vt, Dt, sigma)
    assert torch.equal(G1, G0) and torch.equal(J1, J0)
    with pytest.raises(vg.VipError):
        fwi.gradient(Vt, Dt, sigma, sources=[0, 7])
