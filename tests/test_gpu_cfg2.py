"""Differentiation check at the 128 x 128 grid (8 sources, 64 receivers, 800
steps at 1 ms) with restart checkpoints every 50 steps and recomputation:

* the autograd backward of the seismogram map (FwiSeis, i.e. fwi_adjoint)
  for the Gaussian misfit equals the FP64 oracle gradient (rel-L2 <= 1e-5) and
  fwi_gradient;
* linearisation dot product: <J dv, r> (central difference of fwi_forward,
  h = 0.5 m/s along dv) equals <dv, J^T r> (fwi_adjoint) to 2e-3, the FP32
  finite-difference noise at this step;
* the scratch memory of the checkpointed plan is reported and is smaller than
  storing every step.

The central differences of the misfit at h = 1e-3 m/s on single cells are
taken on the FP64 oracle (tests/test_oracle_fwi.py): in FP32 such a step is
below round-off.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle import fwi as ofwi
import paper_2310_13325_gb300 as vg
from gpu_common import problem, rel

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a, dtype=torch.float32):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


@pytest.fixture(scope="module")
def case():
    from paper_2310_13325_gb300 import build
    build.build()
    cfg = synth.config("cfg2")
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = problem(cfg, 1)
    J_ref, G_ref = ofwi.gradients(V, g, d_obs, sigma)
    return cfg, geo, g, V, d_obs, sigma, J_ref, G_ref


def test_autograd_with_checkpoints_matches_oracle(case):
    cfg, geo, g, V, d_obs, sigma, J_ref, G_ref = case
    fwi = vg.Fwi.from_config(cfg, geo)
    plan1 = fwi.query_plan(1)
    fwi.set_mode(vg.FWI_MODE_BATCHED, cfg.ckpt_every)
    planK = fwi.query_plan(1)
    print("scratch bytes: every step %.1f MB, checkpoint every %d steps %.1f MB"
          % (plan1["scratch_bytes"] / 1e6, planK["ckpt_every"], planK["scratch_bytes"] / 1e6))
    assert planK["ckpt_every"] == cfg.ckpt_every
    assert planK["scratch_bytes"] < plan1["scratch_bytes"]
    v = _t(V).reshape(1, cfg.nz, cfg.nx).requires_grad_(True)
    seis = vg.FwiSeis.apply(v, fwi)
    loss = 0.5 * (((seis - _t(d_obs)[None]) / sigma) ** 2).sum()
    loss.backward()
    g_auto = v.grad.reshape(-1).cpu().numpy()
    assert rel(g_auto, G_ref[0]) <= 1e-5, rel(g_auto, G_ref[0])
    J, G = fwi.gradient(_t(V), _t(d_obs), sigma)
    assert rel(G.reshape(-1).cpu().numpy(), G_ref[0]) <= 1e-5
    assert rel(g_auto, G.reshape(-1).cpu().numpy()) <= 1e-6
    assert abs(J.item() - J_ref[0]) <= 3e-5 * J_ref[0]


def test_linearisation_dot_product(case):
    cfg, geo, g, V, d_obs, sigma, J_ref, G_ref = case
    fwi = vg.Fwi.from_config(cfg, geo)
    fwi.set_mode(vg.FWI_MODE_BATCHED, cfg.ckpt_every)
    gen = torch.Generator(device=DEV).manual_seed(7)
    v = _t(V).reshape(1, cfg.nz, cfg.nx)
    dv = torch.randn(v.shape, generator=gen, device=DEV) * 5.0
    r = torch.randn((1, g.nsrc, g.nrec, g.nt), generator=gen, device=DEV)
    h = 0.5
    Jdv = (fwi.forward(v + h * dv) - fwi.forward(v - h * dv)).double() / (2 * h)
    lhs = float((Jdv * r.double()).sum())
    JTr = fwi.adjoint(v, r)
    rhs = float((JTr.double() * dv.double()).sum())
    assert abs(lhs - rhs) <= 2e-3 * abs(rhs), (lhs, rhs)
