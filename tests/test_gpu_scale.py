"""GPU parity at the benchmark's own sizes and launch shapes, against the FP64
oracle (element by element on sampled outputs the oracle can afford).

* FWI, 120 x 300 grid (160 x 340 padded), 200 receivers, 2000 steps: the
  launch shape the benchmark runs (4-CTA clusters, 10 rows x 4 cells per
  thread, 352 threads, coefficients in shared memory), one prior particle and
  two of the sources (0 and 13): traces and gradient rel-L2 <= 1e-5, the misfit
  within the tolerance derived from the trace bound (2 (|d|/|r|) 1e-5 + 1.1e-6,
  |d|/|r| measured on the oracle's traces), and the BF16 / scaled-FP16
  snapshot gradients within their per-cell rounding bound.
* FWI, 240 x 600 grid, 400 receivers, 3000 steps at 0.8 ms: the
  global-coefficient launch (9-CTA clusters, 8 rows per thread, 320 threads),
  one particle and one source.
* svgd_step / ssvgd_step (Eq. 17, Eq. 22-25) on 600 particles of 36,000
  coordinates drawn from the 120 x 300 prior, with the bound reset: the
  updated particles of sampled rows against the oracle's update of those rows,
  for the three-piece BF16 Gram (rel-L2 1e-5) and the one-pass BF16 Gram (error
  stated, and bounded by the kernel-value error carried through Eq. 17).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle import fwi as ofwi
from oracle import svgd as osvgd
import paper_2310_13325_gb300 as vg
from gpu_common import (misfit_tolerance, oracle_gradients, oracle_map, oracle_sqdist, pair_job,
                        rel)

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U_BF16 = 2.0 ** -8     # unit roundoff of BF16 (8-bit significand)
U_FP16 = 2.0 ** -11    # unit roundoff of FP16 (11-bit significand)


def _t(a, dtype=torch.float32):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_13325_gb300 import build
    build.build()


def _subset_problem(name, sel, P, nt=None):
    """The named workload restricted to the sources sel (geometry of the full
    acquisition), P prior particles, and data = oracle traces of the true model
    plus seeded noise at the workload's sigma rule."""
    cfg = synth.config(name)
    if nt:
        cfg = cfg.with_(nt=nt)
    full = synth.geometry(cfg)
    geo = dict(full, src_iz=full["src_iz"][sel], src_ix=full["src_ix"][sel])
    sub = cfg.with_(nsrc=len(sel))
    g = ofwi.Geom.from_config(sub, geo)
    v_true = synth.true_model(cfg)
    lo, hi = synth.prior_bounds(cfg, v_true)
    V = synth.particles_from_prior(lo, hi, P, seed=2)
    clean = np.stack(oracle_map(pair_job, [(g, v_true, s, None, None)
                                           for s in range(len(sel))]))
    sigma = synth.sigma_from_traces(clean, cfg.sigma_rule)
    d_obs = clean + sigma * synth.unit_noise(clean.shape, seed=1)
    return sub, geo, g, V, d_obs, sigma


@pytest.fixture(scope="module")
def cfg3_case():
    sub, geo, g, V, d_obs, sigma = _subset_problem("cfg3", [0, 13], 1)
    J, G, M, tr = oracle_gradients(g, V, [0, 1], d_obs, sigma)
    return sub, geo, g, V, d_obs, sigma, J, G, M, tr


def test_cfg3_benchmark_launch_matches_oracle(cfg3_case):
    sub, geo, g, V, d_obs, sigma, J_ref, G_ref, M_ref, tr_ref = cfg3_case
    fwi = vg.Fwi.from_config(sub, geo)
    fwi.set_plan(4, 10, 352, coeff=1)
    plan = fwi.query_plan(1)
    assert (plan["cluster_ctas"], plan["rows_per_thread"], plan["threads"],
            plan["coefficients"]) == (4, 10, 352, "shared"), plan
    Vt, Dt = _t(V), _t(d_obs)
    seis = fwi.forward(Vt).cpu().numpy()
    for s in range(2):
        e = rel(seis[0, s], tr_ref[(0, s)])
        print("cfg3 traces, source %d: rel-L2 %.2e" % (s, e))
        assert e <= 1e-5, (s, e)
    J, G = fwi.gradient(Vt, Dt, sigma)
    assert fwi.last_status() == 0
    eg = rel(G.reshape(-1).cpu().numpy(), G_ref[0])
    jtol = misfit_tolerance(np.stack([tr_ref[(0, s)] for s in range(2)])[None], d_obs)
    eJ = abs(J.item() - J_ref[0]) / J_ref[0]
    print("cfg3 benchmark launch: gradient rel-L2 %.2e, misfit rel %.2e (tolerance %.2e)"
          % (eg, eJ, jtol))
    assert eg <= 1e-5
    assert eJ <= jtol


@pytest.mark.parametrize("prec,u", [(vg.FWI_CKPT_BF16, U_BF16), (vg.FWI_CKPT_FP16, U_FP16)])
def test_cfg3_reduced_precision_snapshots_within_rounding_bound(cfg3_case, prec, u):
    """Only the stored snapshot D is rounded; the forward and adjoint fields
    are the FP32 ones. Per cell, dJ/dv then moves by at most u times the sum
    of the magnitudes of its imaging terms (M, from the oracle), plus the
    different FP32 rounding of the two accumulations over N steps (2 N 2^-24
    of M), plus the final rounding (2 * 2^-24 of M). The FP16 values that fall
    below the normal range after the per-block scaling (below 2^-14 of the
    block's largest value) carry an absolute error under 2^-39 of that value:
    a slack of 1e-7 of the largest M covers it."""
    sub, geo, g, V, d_obs, sigma, J_ref, G_ref, M_ref, tr_ref = cfg3_case
    fwi = vg.Fwi.from_config(sub, geo)
    fwi.set_plan(4, 10, 352, coeff=1)
    Vt, Dt = _t(V), _t(d_obs)
    J32, G32 = fwi.gradient(Vt, Dt, sigma)
    G32 = G32.reshape(-1).double().cpu().numpy()
    J, G = fwi.gradient(Vt, Dt, sigma, precision=prec)
    G = G.reshape(-1).double().cpu().numpy()
    M = M_ref[0]
    N = sub.nt
    bound = (u + (2 * N + 2) * 2.0 ** -24) * M * 1.001 + 1e-7 * M.max()
    excess = np.abs(G - G32) / bound
    e_or = rel(G, G_ref[0])
    print("cfg3 snapshots %s: gradient rel-L2 vs oracle %.2e (FP32 path %.2e); largest "
          "|G - G_fp32| / bound %.3f; mean |G - G_fp32| / (u M) %.2e"
          % ("BF16" if prec == vg.FWI_CKPT_BF16 else "FP16", e_or, rel(G32, G_ref[0]),
             excess.max(), (np.abs(G - G32) / (u * M + 1e-300)).mean()))
    assert excess.max() <= 1.0
    assert abs(J.item() - J32.item()) <= 1e-12 * J32.item()   # forward sweep unchanged


def test_largest_grid_global_coefficient_launch_matches_oracle():
    sub, geo, g, V, d_obs, sigma = _subset_problem("cfg5", [20], 1)
    J_ref, G_ref, M_ref, tr_ref = oracle_gradients(g, V, [0], d_obs, sigma)
    fwi = vg.Fwi.from_config(sub, geo)
    fwi.set_plan(9, 8, 320, coeff=2)
    plan = fwi.query_plan(1)
    assert (plan["cluster_ctas"], plan["rows_per_thread"], plan["threads"],
            plan["coefficients"]) == (9, 8, 320, "global"), plan
    Vt, Dt = _t(V), _t(d_obs)
    seis = fwi.forward(Vt).cpu().numpy()
    et = rel(seis[0, 0], tr_ref[(0, 0)])
    J, G = fwi.gradient(Vt, Dt, sigma)
    assert fwi.last_status() == 0
    eg = rel(G.reshape(-1).cpu().numpy(), G_ref[0])
    eJ = abs(J.item() - J_ref[0]) / J_ref[0]
    print("240x600 global-coefficient launch: traces %.2e, gradient %.2e, misfit %.2e"
          % (et, eg, eJ))
    jtol = misfit_tolerance(tr_ref[(0, 0)][None], d_obs[0])
    assert et <= 1e-5 and eg <= 1e-5 and eJ <= jtol


# ---------------------------------------------------------------------------
ROWS = [0, 1, 137, 299, 300, 451, 598, 599]


@pytest.fixture(scope="module")
def svgd_case(tmp_path_factory):
    cfg = synth.config("cfg3")
    v = synth.true_model(cfg)
    lo, hi = synth.prior_bounds(cfg, v)
    lo, hi = lo.reshape(-1), hi.reshape(-1)
    X = synth.particles_from_prior(lo, hi, 600, seed=2).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(7)
    G = (rng.standard_normal(X.shape) * 1e-3).astype(np.float32).astype(np.float64)
    xi = rng.standard_normal(X.shape).astype(np.float32).astype(np.float64)
    D2 = oracle_sqdist(X)
    return X, G, xi, lo, hi, D2


def _eps(X, G, rows, D2, move):
    """Step size giving the sampled rows a largest move of `move` m/s."""
    phi, _, _ = osvgd.svgd_direction_rows(X, -G, rows, D2)
    return move / np.abs(phi).max()


def test_svgd_step_benchmark_shape_matches_oracle(svgd_case):
    X, G, xi, lo, hi, D2 = svgd_case
    eps = _eps(X, G, ROWS, D2, 300.0)
    ref, h2_ref = osvgd.svgd_step_rows(X, -G, eps, ROWS, D2, lo=lo, hi=hi)
    Xt = _t(X)
    ws, h2 = vg.svgd_step(Xt, _t(G), eps, lo=_t(lo), hi=_t(hi),
                          gram_precision=vg.VIP_GRAM_BF16X3, gscale=-1.0)
    assert vg.svgd_status(ws) == vg.VIP_OK
    got = Xt.double().cpu().numpy()[ROWS]
    ex = rel(got, ref)
    em = rel(got - X[ROWS], ref - X[ROWS])
    eh = abs(h2.item() / h2_ref - 1)
    print("svgd_step 600 x 36000, three-piece Gram: updated X %.2e, move %.2e, h2 %.2e"
          % (ex, em, eh))
    assert ex <= 1e-5 and em <= 1e-5 and eh <= 1e-6


def test_ssvgd_step_benchmark_shape_matches_oracle(svgd_case):
    X, G, xi, lo, hi, D2 = svgd_case
    eps = _eps(X, G, ROWS, D2, 300.0)
    ref, h2_ref, tau_ref = osvgd.ssvgd_step_rows(X, -G, eps, xi, ROWS, D2, lo=lo, hi=hi)
    Xt = _t(X)
    ws, h2, tau = vg.ssvgd_step(Xt, _t(G), eps, seed=0, it=0, xi=_t(xi), lo=_t(lo), hi=_t(hi),
                                gram_precision=vg.VIP_GRAM_BF16X3, gscale=-1.0)
    assert vg.svgd_status(ws) == vg.VIP_OK
    assert tau.item() == pytest.approx(tau_ref)
    got = Xt.double().cpu().numpy()[ROWS]
    em = rel(got - X[ROWS], ref - X[ROWS])
    print("ssvgd_step 600 x 36000, injected noise: updated X %.2e, move %.2e"
          % (rel(got, ref), em))
    assert rel(got, ref) <= 1e-5 and em <= 1e-5


def test_svgd_step_one_pass_bf16_gram_error_is_bounded(svgd_case):
    """One-pass BF16 Gram (the reduced-precision mode of the batched workload):
    only the kernel values K and the bandwidth h^2 change. Carried through
    Eq. 17, phi_i moves by at most
      e_K (1/n) sum_j |gscale G_j + (x_i - x_j)/h^2| + e_h (1/n) sum_j K_ij |x_i - x_j| / h^2
    per coordinate, e_K the largest kernel-value error and e_h the relative
    bandwidth error, both measured on the same particles through svgd_sqdist;
    2e-5 of the largest move covers the FP32 update itself."""
    X, G, xi, lo, hi, D2 = svgd_case
    n = X.shape[0]
    h2_ref = osvgd.median_bandwidth(D2)
    K_ref = osvgd.rbf(D2, h2_ref)
    D2g, h2g = vg.svgd_sqdist(_t(X), gram_precision=vg.VIP_GRAM_BF16)
    Kg = np.exp(-D2g.cpu().numpy() / (2 * h2g.item()))
    e_K = np.abs(Kg - K_ref).max()
    e_h = abs(h2g.item() / h2_ref - 1)
    eps = _eps(X, G, ROWS, D2, 300.0)
    phi_ref, _, _ = osvgd.svgd_direction_rows(X, -G, ROWS, D2)
    Xt = _t(X)
    ws, h2 = vg.svgd_step(Xt, _t(G), eps, gram_precision=vg.VIP_GRAM_BF16, gscale=-1.0)
    assert vg.svgd_status(ws) == vg.VIP_OK
    phi = (Xt.double().cpu().numpy()[ROWS] - X[ROWS]) / eps
    B = np.stack([np.abs(-G + (X[i][None, :] - X) / h2_ref).mean(axis=0) for i in ROWS])
    R = np.stack([(K_ref[i][:, None] * np.abs(X[i][None, :] - X)).mean(axis=0) / h2_ref
                  for i in ROWS])
    bound = 1.01 * (e_K * B + e_h * R) + 2e-5 * np.abs(phi_ref).max()
    print("one-pass BF16 Gram at 600 x 36000: Kbar max error %.2e, h2 %.2e, phi rel-L2 %.2e, "
          "largest |dphi| / bound %.3f" % (e_K, e_h, rel(phi, phi_ref),
                                            (np.abs(phi - phi_ref) / bound).max()))
    assert np.all(np.abs(phi - phi_ref) <= bound)
    assert e_K <= 1e-3


@pytest.mark.parametrize("K,prec", [(1, vg.FWI_FP32), (7, vg.FWI_CKPT_BF16),
                                    (1, vg.FWI_CKPT_FP16), (7, vg.FWI_CKPT_FP16)])
def test_fill_launch_on_idle_sms_changes_no_result(K, prec):
    """The benchmark's grid with more work items than 4-CTA clusters: a second
    launch of smaller global-coefficient clusters takes the SMs the main launch
    leaves idle and draws items from the same counter. Traces, gradients and
    misfits equal those of the main launch alone bit for bit, whichever launch
    computed an item (store-every-step FP32 snapshots, and restart checkpoints
    every 7 steps with BF16 snapshots, scaled FP16 snapshots, whose power-of-two
    scale belongs to the 4 cells of a task's row whatever the launch shape), in
    the forward, gradient, adjoint-only and source-minibatch calls."""
    sub, geo, g, V, d_obs, sigma = _subset_problem("cfg3", [0, 13], 48, nt=300)
    Vt, Dt = _t(V), _t(d_obs)
    out = {}
    for fill in (True, False):
        fwi = vg.Fwi.from_config(sub, geo)
        fwi.set_mode(vg.FWI_MODE_BATCHED, K)
        fwi.set_fill(fill)
        shape = fwi.query_fill(48, prec)
        if fill:
            print("fill launch:", shape, "main:", fwi.query_plan(48))
            assert shape["clusters"] >= 1 and shape["cluster_ctas"] < 4
        else:
            assert shape["clusters"] == 0
        S = fwi.forward(Vt).clone()
        J, G = fwi.gradient(Vt, Dt, sigma, precision=prec)
        J, G = J.clone(), G.clone()
        A = fwi.adjoint(Vt, S - Dt[None], precision=prec).clone()   # autograd backward
        Jm, Gm = fwi.gradient(Vt, Dt, sigma, precision=prec, sources=[1])   # minibatch
        out[fill] = (S, J, G, A, Jm.clone(), Gm.clone())
        assert fwi.last_status() == 0
        fwi.close()
    for a, b in zip(out[True], out[False]):
        assert torch.equal(a, b)


def test_svgd_step_largest_shape_matches_oracle_on_sampled_rows():
    """svgd_step at the largest workload's size (2000 particles of the 240x600
    prior, 144,000 coordinates) with the bound reset. With the bandwidth given
    (h2 > 0 skips the median), the updated particle i needs only the row
    D2[i, :], so the oracle computes those rows alone for the sampled
    particles."""
    cfg = synth.config("cfg5")
    v = synth.true_model(cfg)
    lo, hi = synth.prior_bounds(cfg, v)
    lo, hi = lo.reshape(-1), hi.reshape(-1)
    n = 2000
    X = synth.particles_from_prior(lo, hi, n, seed=2).astype(np.float32).astype(np.float64)
    G = (np.random.default_rng(17).standard_normal(X.shape) * 1e-3).astype(np.float32)
    G = G.astype(np.float64)
    rows = [0, 1, 777, 1000, 1998, 1999]
    D2 = np.zeros((n, n))
    D2[rows] = osvgd.sqdist_rows(X, rows)
    h2 = float(np.median(D2[rows])) / (2.0 * np.log(n + 1.0))
    phi, _, _ = osvgd.svgd_direction_rows(X, -G, rows, D2, h2)
    eps = 300.0 / np.abs(phi).max()
    ref, _ = osvgd.svgd_step_rows(X, -G, eps, rows, D2, h2=h2, lo=lo, hi=hi)
    Xt = _t(X)
    ws, h2_used = vg.svgd_step(Xt, _t(G), eps, h2=h2, lo=_t(lo), hi=_t(hi),
                               gram_precision=vg.VIP_GRAM_BF16X3, gscale=-1.0)
    assert vg.svgd_status(ws) == vg.VIP_OK
    assert h2_used.item() == pytest.approx(h2, rel=1e-7)
    got = Xt.double().cpu().numpy()[rows]
    ex, em = rel(got, ref), rel(got - X[rows], ref - X[rows])
    # per element, the move may differ by the FP32 rounding of the stored
    # particle (2^-24 of |x| before and after) plus the FP32 accumulation of
    # the n particles' terms of Eq. 17, at most (n + 6) 2^-24 times the sum of
    # their magnitudes A = (eps / n) sum_j k_ij (|G_j| + |x_i - x_j| / h^2)
    K = osvgd.rbf(D2[rows], h2)
    A = np.stack([(eps / n) * (K[k] @ np.abs(G) +
                               (K[k][:, None] * np.abs(X[i][None, :] - X)).sum(axis=0) / h2)
                  for k, i in enumerate(rows)])
    bound = 2.0 ** -24 * (np.abs(X[rows]) + np.abs(ref)) + (n + 6) * 2.0 ** -24 * A
    ratio = (np.abs(got - ref) / bound).max()
    print("svgd_step 2000 x 144000 (given bandwidth), sampled rows: updated X %.2e, move %.2e, "
          "largest |error| / per-element bound %.3f" % (ex, em, ratio))
    assert ex <= 1e-5 and ratio <= 1.0
