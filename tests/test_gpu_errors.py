"""Error paths of the C ABI on the GPU, made to happen without any fault:

* VIP_ERR_NOMEM from a context whose workspace limit is too small, with the
  bytes a plan needs reported (fwi_query_plan, fwi_bytes_needed);
* VIP_ERR_NONFINITE from NaN velocities, NaN observed data, NaN particles and
  NaN gradients (fwi_last_status, svgd_status), the tensor-core update leaving
  the particles unchanged;
* VIP_ERR_TIMEOUT from the bounded mbarrier waits of the tensor-core Gram and
  update kernels: the test hook shortens the bound to about 10 microseconds
  and stops the copy producer, so the consumer's wait runs out by design; the
  kernels record the failure, free their tensor memory and return, and the
  context stays usable (the next step matches the oracle).
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import svgd as osvgd
import paper_2310_13325_gb300 as vg
from paper_2310_13325_gb300 import _lib
from gpu_common import cfg1_case, rel

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a, dtype=torch.float32):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_13325_gb300 import build
    build.build()


def test_workspace_limit_too_small_reports_bytes_needed():
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(2)
    small = 1 << 20
    fwi = vg.Fwi.from_config(cfg, geo, workspace_limit=small)
    with pytest.raises(vg.VipError) as e:
        fwi.gradient(_t(V), _t(d_obs), sigma)
    assert e.value.code == vg.VIP_ERR_NOMEM
    need = fwi.bytes_needed()
    assert need > small
    L = _lib.load()
    plan = (ctypes.c_int * 10)()
    nb = ctypes.c_size_t(0)
    assert L.fwi_query_plan(fwi._h, 2, vg.FWI_FP32, plan, ctypes.byref(nb)) == vg.VIP_ERR_NOMEM
    assert nb.value == need
    # granting the reported bytes makes the same call succeed
    ok = vg.Fwi.from_config(cfg, geo, workspace_limit=need)
    J, G = ok.gradient(_t(V), _t(d_obs), sigma)
    assert ok.last_status() == vg.VIP_OK and torch.isfinite(G).all()
    assert ok.bytes_needed() <= need


def test_nonfinite_velocity_and_data_are_reported():
    cfg, geo, g, v_true, V, d_obs, sigma, lo, hi = cfg1_case(2)
    fwi = vg.Fwi.from_config(cfg, geo)
    Vt, Dt = _t(V), _t(d_obs)
    bad = Vt.clone()
    bad[1, 7] = float("nan")
    fwi.gradient(bad, Dt, sigma)
    assert fwi.last_status() == vg.VIP_ERR_NONFINITE
    fwi.forward(bad)
    assert fwi.last_status() == vg.VIP_ERR_NONFINITE
    bad[1, 7] = float("inf")
    fwi.forward(bad)
    assert fwi.last_status() == vg.VIP_ERR_NONFINITE
    fwi.gradient(Vt, Dt, sigma)
    assert fwi.last_status() == vg.VIP_OK
    Dbad = Dt.clone()
    Dbad[0, 3, 50] = float("nan")
    J, _ = fwi.gradient(Vt, Dbad, sigma)
    assert fwi.last_status() == vg.VIP_ERR_NONFINITE
    assert not torch.isfinite(J).all()
    # the plain loop reports the same
    fwi.set_mode(vg.FWI_MODE_PLAIN, 1)
    fwi.gradient(bad, Dt, sigma)
    assert fwi.last_status() == vg.VIP_ERR_NONFINITE
    fwi.gradient(Vt, Dt, sigma)
    assert fwi.last_status() == vg.VIP_OK


@pytest.mark.parametrize("gp", [vg.VIP_GRAM_BF16X3, vg.VIP_GRAM_BF16, vg.VIP_GRAM_FP32])
def test_nonfinite_gradient_and_particles_are_reported(gp):
    rng = np.random.default_rng(3)
    n, d = 40, 3000
    X = _t(rng.standard_normal((n, d)))
    G = _t(rng.standard_normal((n, d)))
    Gbad = G.clone()
    Gbad[5, 1234] = float("nan")
    X0 = X.clone()
    ws, _ = vg.svgd_step(X, Gbad, 0.1, gram_precision=gp)
    assert vg.svgd_status(ws) == vg.VIP_ERR_NONFINITE
    if gp != vg.VIP_GRAM_FP32:
        # the tensor-core update leaves the particles as they were
        assert torch.equal(X, X0)
    Xbad = X0.clone()
    Xbad[2, 17] = float("inf")
    ws, _ = vg.svgd_step(Xbad, G, 0.1, gram_precision=gp, ws=ws)
    assert vg.svgd_status(ws) == vg.VIP_ERR_NONFINITE
    X = X0.clone()
    ws, _ = vg.svgd_step(X, G, 0.1, gram_precision=gp, ws=ws)
    assert vg.svgd_status(ws) == vg.VIP_OK
    assert torch.isfinite(X).all()


def test_expired_wait_reports_timeout_and_leaves_the_context_usable():
    L = _lib.load()
    rng = np.random.default_rng(4)
    n, d = 64, 2000
    X = rng.standard_normal((n, d)).astype(np.float32).astype(np.float64)
    G = rng.standard_normal((n, d)).astype(np.float32).astype(np.float64)
    Xt = _t(X)
    assert L.vip_test_set_wait(20000, 1) == 0          # ~10 us, producer stalled
    try:
        ws, h2 = vg.svgd_step(Xt, _t(G), 0.1, gram_precision=vg.VIP_GRAM_BF16X3)
        st = vg.svgd_status(ws)
    finally:
        assert L.vip_test_set_wait(0, 0) == 0
    assert st == vg.VIP_ERR_TIMEOUT
    assert np.isnan(h2.item())
    assert torch.isnan(Xt).all()                       # no half-updated particles
    assert L.vip_test_set_wait(-1, 0) == vg.VIP_ERR_ARG
    assert L.vip_test_set_wait(0, 2) == vg.VIP_ERR_ARG
    # same process, same context: the next step runs normally and is right
    # (step size with an O(1) move, so the FP32 rounding of the particles does
    # not mask the error of the move)
    phi0, _, _ = osvgd.svgd_direction(X, G)
    eps = 0.5 / np.abs(phi0).max()
    Xt = _t(X)
    ws, h2 = vg.svgd_step(Xt, _t(G), eps, gram_precision=vg.VIP_GRAM_BF16X3, ws=ws)
    assert vg.svgd_status(ws) == vg.VIP_OK
    X_ref, h2_ref = osvgd.svgd_step(X, G, eps)
    assert rel(Xt.cpu().numpy() - X, X_ref - X) <= 1e-5
    assert abs(h2.item() / h2_ref - 1) <= 1e-6
