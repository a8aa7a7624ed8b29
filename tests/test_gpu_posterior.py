"""Posterior statistics after several iterations, GPU beside the FP64 oracle.

The 64 x 64 workload (8 particles, 4 sources, 32 receivers, 400 steps):
K iterations of gradient (Sec. 3, Eq. 26) -> SVGD update (Eq. 17) with the
bound reset, and of sSVGD (Eq. 22-25) with the same injected noise on both
sides, run by the library and by the oracle's own loop from the same seeded
particles. After every iteration the relative L2 error of the particle mean
and of the per-cell standard deviation against the oracle is printed for each
precision mode, and that of the mean's displacement from the starting
particles (what the iterations changed): FP32 snapshots with the three-piece BF16 Gram, BF16 snapshots,
scaled FP16 snapshots, the one-pass BF16 Gram, and BF16 snapshots with the
one-pass Gram together (the reduced-precision workload as a whole). The
iteration is chaotic in the particles, so these errors are reported, not
gated: the test asserts finite results and a loose sanity bound only.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import svgd as osvgd
import paper_2310_13325_gb300 as vg
from gpu_common import cfg1_case, oracle_gradients, rel

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
ITERS = 6
P = 8
MODES = [("FP32 snapshots, BF16x3 Gram", vg.FWI_FP32, vg.VIP_GRAM_BF16X3),
         ("BF16 snapshots", vg.FWI_CKPT_BF16, vg.VIP_GRAM_BF16X3),
         ("FP16 snapshots", vg.FWI_CKPT_FP16, vg.VIP_GRAM_BF16X3),
         ("one-pass BF16 Gram", vg.FWI_FP32, vg.VIP_GRAM_BF16),
         ("BF16 snapshots + BF16 Gram", vg.FWI_CKPT_BF16, vg.VIP_GRAM_BF16)]


def _t(a, dtype=torch.float32):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_13325_gb300 import build
    build.build()


def _noise(k, shape):
    return np.random.default_rng(500 + k).standard_normal(shape).astype(np.float32)


@pytest.fixture(scope="module")
def oracle_runs():
    """The oracle's own SVGD and sSVGD loops: particles after each iteration."""
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(P)
    lo, hi = lo.reshape(-1), hi.reshape(-1)
    X0 = V.astype(np.float32).astype(np.float64)
    _, G0, _, _ = oracle_gradients(g, X0, range(g.nsrc), d_obs, sigma)
    eps = 20.0 / np.abs(G0).max()          # first update moves the fastest cell ~20 m/s
    runs = {}
    for kind in ("svgd", "ssvgd"):
        X, hist = X0.copy(), []
        for k in range(ITERS):
            _, G, _, _ = oracle_gradients(g, X, range(g.nsrc), d_obs, sigma)
            if kind == "svgd":
                X, _ = osvgd.svgd_step(X, -G, eps, lo=lo, hi=hi)
            else:
                X, _, _ = osvgd.ssvgd_step(X, -G, eps, _noise(k, X.shape), lo=lo, hi=hi)
            hist.append(X.copy())
        runs[kind] = hist
    return eps, runs


def _gpu_run(kind, prec, gram, eps):
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(P)
    fwi = vg.Fwi.from_config(cfg, geo)
    X = _t(V.astype(np.float32))
    Dt, lo_t, hi_t = _t(d_obs), _t(lo.reshape(-1)), _t(hi.reshape(-1))
    hist = []
    ws = None
    for k in range(ITERS):
        _, G = fwi.gradient(X, Dt, sigma, precision=prec)
        assert fwi.last_status() == vg.VIP_OK
        G = G.reshape(P, -1)
        if kind == "svgd":
            ws, _ = vg.svgd_step(X, G, eps, lo=lo_t, hi=hi_t, gram_precision=gram, ws=ws,
                                 gscale=-1.0)
        else:
            ws, _, _ = vg.ssvgd_step(X, G, eps, seed=0, it=k, xi=_t(_noise(k, X.shape)),
                                     lo=lo_t, hi=hi_t, gram_precision=gram, ws=ws, gscale=-1.0)
        assert vg.svgd_status(ws) == vg.VIP_OK
        hist.append(X.double().cpu().numpy())
    return hist


@pytest.mark.parametrize("kind", ["svgd", "ssvgd"])
def test_posterior_mean_and_std_after_iterations(oracle_runs, kind):
    eps, runs = oracle_runs
    ref = runs[kind]
    x0 = cfg1_case(P)[4].astype(np.float32).astype(np.float64)
    modes = MODES if kind == "svgd" else MODES[:3]
    print("\n%s, %d particles, 64 x 64, eps %.3g: rel-L2 of the particle mean / per-cell "
          "std against the oracle after each iteration" % (kind, P, eps))
    for name, prec, gram in modes:
        hist = _gpu_run(kind, prec, gram, eps)
        em = [rel(h.mean(0), r.mean(0)) for h, r in zip(hist, ref)]
        es = [rel(h.std(0), r.std(0)) for h, r in zip(hist, ref)]
        # the mean's displacement from the starting particles: the part of the
        # mean the iterations changed, so its error is not diluted by the prior
        ed = [rel(h.mean(0) - x0.mean(0), r.mean(0) - x0.mean(0)) for h, r in zip(hist, ref)]
        print("  %-28s mean  %s" % (name, " ".join("%.1e" % e for e in em)))
        print("  %-28s drift %s" % ("", " ".join("%.1e" % e for e in ed)))
        print("  %-28s std   %s" % ("", " ".join("%.1e" % e for e in es)))
        assert all(np.isfinite(h).all() for h in hist)
        assert max(em) <= 1e-3 and max(es) <= 0.2 and max(ed) <= 0.2, (name, em, es, ed)
