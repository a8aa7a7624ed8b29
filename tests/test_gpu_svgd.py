"""GPU parity of the SVGD / sSVGD / ADVI updates against the FP64 oracle,
through the C ABI.

FP32 results (phi, updated particles) are held to relative L2 <= 1e-5; the
one-pass BF16 Gram is measured and held to the bound stated in its test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle import advi as oadvi
from oracle import philox as ophilox
from oracle import svgd as osvgd
import paper_2310_13325_gb300 as vg
from gpu_common import rel

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
EXACT_GRAMS = [vg.VIP_GRAM_BF16X3, vg.VIP_GRAM_FP32]


def _t(a, dtype=torch.float32):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_13325_gb300 import build
    build.build()


def _unit_case(n, d, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)).astype(np.float32).astype(np.float64)
    G = rng.standard_normal((n, d)).astype(np.float32).astype(np.float64)
    return X, G


@pytest.mark.parametrize("gp", EXACT_GRAMS)
@pytest.mark.parametrize("n,d", [(8, 4096), (3, 2), (1, 50), (130, 1000), (257, 3001)])
def test_svgd_step_matches_oracle(gp, n, d):
    X, G = _unit_case(n, d, seed=n + d)
    Xt = _t(X)
    # step size such that the update is O(1): the FP32 rounding of the new
    # particles then does not mask the error of phi
    phi0, _, _ = osvgd.svgd_direction(X, G)
    eps = 0.5 / np.abs(phi0).max()
    ws, h2 = vg.svgd_step(Xt, _t(G), eps, gram_precision=gp)
    X_ref, h2_ref = osvgd.svgd_step(X, G, eps)
    assert rel(Xt.cpu().numpy(), X_ref) <= 1e-5
    phi = (Xt.double().cpu().numpy() - X) / eps
    phi_ref = (X_ref - X) / eps
    assert rel(phi, phi_ref) <= 1e-5, rel(phi, phi_ref)
    assert abs(h2.item() - h2_ref) <= 1e-6 * h2_ref


def test_svgd_step_cfg1_particles_with_bounds():
    cfg = synth.config("cfg1")
    v = synth.true_model(cfg)
    lo, hi = synth.prior_bounds(cfg, v)
    X = synth.particles_from_prior(lo, hi, 8, seed=2).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(0)
    G = (rng.standard_normal(X.shape) * 0.5).astype(np.float32).astype(np.float64)
    eps = 400.0
    Xt = _t(X)
    vg.svgd_step(Xt, _t(G), eps, lo=_t(lo.reshape(-1)), hi=_t(hi.reshape(-1)))
    X_ref, _ = osvgd.svgd_step(X, G, eps, lo=lo.reshape(-1), hi=hi.reshape(-1))
    got = Xt.cpu().numpy()
    assert rel(got, X_ref) <= 1e-5
    assert np.all(got >= lo.reshape(1, -1) - 1e-3) and np.all(got <= hi.reshape(1, -1) + 1e-3)
    assert rel(got - X, X_ref - X) <= 1e-4


@pytest.mark.parametrize("gp", EXACT_GRAMS + [vg.VIP_GRAM_BF16])
def test_sqdist_and_median_bandwidth(gp):
    X, _ = _unit_case(200, 5000, seed=5)
    D2, h2 = vg.svgd_sqdist(_t(X), gram_precision=gp)
    D2_ref = osvgd.pairwise_sqdist(X)
    tol = 1e-6 if gp != vg.VIP_GRAM_BF16 else 2e-3
    off = ~np.eye(200, dtype=bool)
    e = np.abs(D2.cpu().numpy() - D2_ref)[off].max() / D2_ref[off].min()
    print("gram %d: max D2 error / min D2 = %.2e" % (gp, e))
    assert e <= tol
    assert np.all(np.diag(D2.cpu().numpy()) == 0)
    assert abs(h2.item() - osvgd.median_bandwidth(D2_ref)) <= tol * h2.item()


@pytest.mark.parametrize("n", [1, 2, 7, 8, 33])
def test_median_selection_is_exact_on_exact_distances(n):
    # integer coordinates: every Gram entry and squared distance is exact in
    # BF16 products with FP32 accumulation, so the selected median must equal
    # a plain sort of the oracle's distances exactly
    rng = np.random.default_rng(n)
    X = rng.integers(-6, 7, size=(n, 64)).astype(np.float64)
    if n > 3:
        X[3] = X[1]                       # a duplicate particle: zero distances
    D2_ref = osvgd.pairwise_sqdist(X)
    for gp in (vg.VIP_GRAM_BF16, vg.VIP_GRAM_FP32):
        # centring makes coordinates non-integers; compare the median of the
        # GPU's own D2 with the bandwidth it selected
        D2, h2 = vg.svgd_sqdist(_t(X), gram_precision=gp)
        D2 = D2.cpu().numpy()
        allv = np.sort(D2.reshape(-1))
        m = allv.size
        med = allv[m // 2] if m % 2 else 0.5 * (allv[m // 2 - 1] + allv[m // 2])
        expect = 1.0 if med < 1e-30 else med / (2 * np.log(n + 1.0))
        assert abs(h2.item() - expect) <= 1e-14 * max(expect, 1.0)
        # centring makes the coordinates non-integer unless n is a power of
        # two, so the one-piece BF16 image rounds them
        # (the duplicated particle's zero distance is recovered from
        # |x|^2 + |y|^2 - 2 x.y: its error scales with |x|^2, not with 0)
        tol = 3e-3 if gp == vg.VIP_GRAM_BF16 else 1e-5
        assert np.allclose(D2, D2_ref, rtol=tol, atol=tol * np.median(D2_ref))


def test_bf16_gram_kernel_error_is_bounded():
    """Velocity particles shaped like the batched workload (120 x 300 cells,
    prior band of 2 km/s): squared distances and kernel values of the one-pass
    BF16 Gram and of the three-piece split against the FP64 oracle."""
    cfg = synth.config("cfg3")
    v = synth.true_model(cfg)
    lo, hi = synth.prior_bounds(cfg, v)
    X = synth.particles_from_prior(lo, hi, 96, seed=2).astype(np.float32).astype(np.float64)
    D2_ref = osvgd.pairwise_sqdist(X)
    h2_ref = osvgd.median_bandwidth(D2_ref)
    K_ref = osvgd.rbf(D2_ref, h2_ref)
    off = ~np.eye(96, dtype=bool)
    res = {}
    for gp in (vg.VIP_GRAM_BF16, vg.VIP_GRAM_BF16X3):
        D2, h2 = vg.svgd_sqdist(_t(X), gram_precision=gp)
        D2 = D2.cpu().numpy()
        eD = np.abs(D2 - D2_ref)[off].max() / np.median(D2_ref[off])
        K = np.exp(-D2 / (2 * h2.item()))
        eK = np.abs(K - K_ref).max() / K_ref[off].max()
        res[gp] = (eD, eK, abs(h2.item() / h2_ref - 1))
    print("one-pass BF16: D2 %.2e, Kbar %.2e, h2 %.2e; three-piece: D2 %.2e, Kbar %.2e, "
          "h2 %.2e" % (res[0] + res[1]))
    assert res[vg.VIP_GRAM_BF16][0] <= 1e-3 and res[vg.VIP_GRAM_BF16][1] <= 1e-3
    assert res[vg.VIP_GRAM_BF16X3][0] <= 1e-6 and res[vg.VIP_GRAM_BF16X3][1] <= 1e-6


def test_ssvgd_step_injected_noise_matches_oracle():
    X, G = _unit_case(16, 3000, seed=8)
    xi = np.random.default_rng(9).standard_normal(X.shape).astype(np.float32).astype(np.float64)
    Xt = _t(X)
    eps = 0.05
    ws, h2, tau = vg.ssvgd_step(Xt, _t(G), eps, seed=0, it=0, xi=_t(xi))
    X_ref, h2_ref, tau_ref = osvgd.ssvgd_step(X, G, eps, xi)
    assert tau.item() == pytest.approx(tau_ref)
    assert rel(Xt.cpu().numpy() - X, X_ref - X) <= 1e-5


@pytest.mark.parametrize("n", [31, 32, 33, 65, 97])
def test_ssvgd_cholesky_panels_match_oracle(n):
    # the blocked Cholesky of Kbar + tau I works in 32-wide panels: one short
    # panel, exactly one, one plus a single row, several with a ragged last
    # one. The noise term sqrt(2 eps / n) Lk Xi of the move carries the factor.
    X, G = _unit_case(n, 1000, seed=40 + n)
    xi = np.random.default_rng(50 + n).standard_normal(X.shape).astype(np.float32)
    xi = xi.astype(np.float64)
    Xt = _t(X)
    eps = 0.05
    _, _, tau = vg.ssvgd_step(Xt, _t(G), eps, seed=0, it=0, xi=_t(xi))
    X_ref, _, tau_ref = osvgd.ssvgd_step(X, G, eps, xi)
    assert tau.item() == pytest.approx(tau_ref)
    assert rel(Xt.cpu().numpy() - X, X_ref - X) <= 1e-5


def test_ssvgd_step_philox_noise_matches_oracle_stream():
    X, G = _unit_case(12, 2049, seed=10)
    seed, it = 3, 17
    xi = ophilox.normal(12, 2049, seed, it)
    Xt = _t(X)
    eps = 0.05
    vg.ssvgd_step(Xt, _t(G), eps, seed=seed, it=it)
    X_ref, _, _ = osvgd.ssvgd_step(X, G, eps, xi)
    assert rel(Xt.cpu().numpy() - X, X_ref - X) <= 1e-5


def test_philox_normal_stream_matches_oracle():
    out = vg.philox_normal(33, 1027, seed=0x123456789, it=(5 << 32) + 7).cpu().numpy()
    ref = ophilox.normal(33, 1027, 0x123456789, (5 << 32) + 7)
    assert np.abs(out - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("bounded", [True, False])
def test_advi_sample_and_step_match_oracle(bounded):
    rng = np.random.default_rng(4)
    d, S = 5000, 64
    a = rng.uniform(1500, 2000, d) if bounded else None
    b = a + rng.uniform(500, 1500, d) if bounded else None
    mu = rng.standard_normal(d) * 0.5
    om = rng.standard_normal(d) * 0.2 - 1.0
    eta = rng.standard_normal((S, d))
    gm = rng.standard_normal((S, d)) * 1e-3
    f32 = lambda x: None if x is None else x.astype(np.float32).astype(np.float64)
    mu, om, eta, gm, a, b = map(f32, (mu, om, eta, gm, a, b))
    m_ref = oadvi.sample(mu, om, eta, a, b)
    m = vg.advi_sample(_t(mu), _t(om), _t(eta), None if a is None else _t(a),
                       None if b is None else _t(b))
    assert rel(m.cpu().numpy(), m_ref) <= 1e-6
    st = torch.zeros((4, d), device=DEV)
    mut, omt = _t(mu), _t(om)
    ref_state = tuple(np.zeros(d) for _ in range(4))
    mur, omr = mu.copy(), om.copy()
    for t in (1, 2, 3):
        vg.advi_step(mut, omt, st, t, _t(eta), _t(gm), 0.01, None if a is None else _t(a),
                     None if b is None else _t(b))
        mur, omr, ref_state = oadvi.advi_step(mur, omr, ref_state, t, eta, gm, 0.01, a, b)
    assert rel(mut.cpu().numpy(), mur) <= 1e-5
    assert rel(omt.cpu().numpy(), omr) <= 1e-5


# ---------------------------------------------------------------------------
# diagonal matrix-valued kernel (svgd_step_q, ssvgd_step_q, svgd_inverse_variance)

def _scaled_case(n, d, seed):
    """Particles whose coordinates have spreads from 0.1 to 20, so that the
    inverse-variance metric differs strongly from the Euclidean one."""
    rng = np.random.default_rng(seed)
    scale = rng.uniform(0.1, 20.0, size=(1, d))
    X = (rng.standard_normal((n, d)) * scale).astype(np.float32).astype(np.float64)
    G = (rng.standard_normal((n, d)) / scale).astype(np.float32).astype(np.float64)
    return X, G


@pytest.mark.parametrize("n,d,offset", [(9, 4096, 0.0), (2, 3, 0.0), (130, 1000, 0.0),
                                        (600, 2000, 3000.0)])
def test_inverse_variance_matches_oracle(n, d, offset):
    # offset: velocity-like coordinates, a spread of 0.1 to 20 on a mean of
    # 3000, where the deviations are small against the values
    X, _ = _scaled_case(n, d, seed=n)
    X = (X + offset).astype(np.float32).astype(np.float64)
    X[:, 0] = X[0, 0]                     # a coordinate without spread: q = 1
    q = vg.svgd_inverse_variance(_t(X)).cpu().numpy()
    ref = osvgd.inverse_variance(X)
    assert q[0] == 1.0
    assert np.allclose(q, ref, rtol=1e-6, atol=0)


@pytest.mark.parametrize("gp", EXACT_GRAMS)
@pytest.mark.parametrize("n,d", [(8, 4096), (3, 2), (130, 1000)])
def test_matrix_kernel_svgd_step_matches_oracle(gp, n, d):
    X, G = _scaled_case(n, d, seed=n + 2 * d)
    Xt = _t(X)
    q = vg.svgd_inverse_variance(Xt)
    qh = q.double().cpu().numpy()         # the same q on both sides
    phi0, _, _ = osvgd.svgd_direction_q(X, G, qh)
    eps = 0.5 / np.abs(phi0 / X.std(axis=0, keepdims=True).clip(1e-30)).max()
    ws, h2 = vg.svgd_step(Xt, _t(G), eps, gram_precision=gp, q=q)
    X_ref, h2_ref = osvgd.svgd_step_q(X, G, qh, eps)
    phi = (Xt.double().cpu().numpy() - X) / eps
    phi_ref = (X_ref - X) / eps
    assert rel(phi, phi_ref) <= 1e-5, rel(phi, phi_ref)
    # the Gram is accumulated in FP32: centred particles are strongly
    # anticorrelated at small n (G_ij ~ -|x|^2 / (n - 1)), and d/16 sequential
    # FP32 additions of partial sums of that size bound the relative error of
    # the median distance by 2 (d/16) 2^-24 |G| / med ~ 2e-6 for n = 8,
    # d = 4096 (measured 1.3e-6); 1e-5 is the FP32 bound used for phi
    assert abs(h2.item() - h2_ref) <= 1e-5 * h2_ref


def test_matrix_kernel_with_unit_q_equals_rbf_bit_for_bit():
    X, G = _unit_case(40, 2000, seed=21)
    xi = _t(np.random.default_rng(22).standard_normal(X.shape))
    ones = torch.ones(X.shape[1], device=DEV)
    A, B = _t(X), _t(X)
    vg.svgd_step(A, _t(G), 0.1)
    vg.svgd_step(B, _t(G), 0.1, q=ones)
    assert torch.equal(A, B)
    A, B = _t(X), _t(X)
    vg.ssvgd_step(A, _t(G), 0.05, seed=0, it=0, xi=xi)
    vg.ssvgd_step(B, _t(G), 0.05, seed=0, it=0, xi=xi, q=ones)
    assert torch.equal(A, B)


def test_matrix_kernel_ssvgd_step_injected_noise_matches_oracle():
    X, G = _scaled_case(16, 3000, seed=23)
    xi = np.random.default_rng(24).standard_normal(X.shape).astype(np.float32).astype(np.float64)
    Xt = _t(X)
    q = vg.svgd_inverse_variance(Xt)
    qh = q.double().cpu().numpy()
    eps = 0.05
    ws, h2, tau = vg.ssvgd_step(Xt, _t(G), eps, seed=0, it=0, xi=_t(xi), q=q)
    X_ref, h2_ref, tau_ref = osvgd.ssvgd_step_q(X, G, qh, eps, xi)
    assert tau.item() == pytest.approx(tau_ref)
    assert rel(Xt.cpu().numpy() - X, X_ref - X) <= 1e-5


# ---------------------------------------------------------------------------
# ADVI ascent rules (advi_step_opt) and SVGD in the unconstrained space

def _advi_case(d, S, seed, bounded):
    rng = np.random.default_rng(seed)
    a = rng.uniform(1500, 2000, d) if bounded else None
    b = a + rng.uniform(500, 1500, d) if bounded else None
    mu = rng.standard_normal(d) * 0.5
    om = rng.standard_normal(d) * 0.2 - 1.0
    eta = rng.standard_normal((S, d))
    gm = rng.standard_normal((S, d)) * 1e-3
    f32 = lambda x: None if x is None else x.astype(np.float32).astype(np.float64)
    return tuple(map(f32, (mu, om, eta, gm, a, b)))


@pytest.mark.parametrize("rule", [vg.ASCENT_SGD, vg.ASCENT_ADAGRAD, vg.ASCENT_ADADELTA,
                                  vg.ASCENT_ADAM])
def test_advi_ascent_rules_match_oracle(rule):
    d, S = 5000, 64
    mu, om, eta, gm, a, b = _advi_case(d, S, 31, True)
    lr = {vg.ASCENT_SGD: 0.5, vg.ASCENT_ADAGRAD: 0.01, vg.ASCENT_ADADELTA: 1.0,
          vg.ASCENT_ADAM: 0.01}[rule]
    st = torch.zeros((4, d), device=DEV)
    mut, omt = _t(mu), _t(om)
    state = tuple(np.zeros(d) for _ in range(4))
    mur, omr = mu.copy(), om.copy()
    for t in (1, 2, 3):
        vg.advi_step_opt(mut, omt, st, t, _t(eta), _t(gm), lr, rule, _t(a), _t(b))
        mur, omr, state = oadvi.advi_step_opt(mur, omr, state, t, eta, gm, lr, rule, a, b)
    # compare the moves (the particles' own FP32 rounding would mask them)
    assert rel(mut.double().cpu().numpy() - mu, mur - mu) <= 1e-5, rule
    assert rel(omt.double().cpu().numpy() - om, omr - om) <= 1e-5, rule


def test_advi_step_opt_adam_is_advi_step():
    d, S = 3000, 16
    mu, om, eta, gm, a, b = _advi_case(d, S, 32, True)
    st1, st2 = torch.zeros((4, d), device=DEV), torch.zeros((4, d), device=DEV)
    m1, o1, m2, o2 = _t(mu), _t(om), _t(mu), _t(om)
    for t in (1, 2):
        vg.advi_step(m1, o1, st1, t, _t(eta), _t(gm), 0.02, _t(a), _t(b))
        vg.advi_step_opt(m2, o2, st2, t, _t(eta), _t(gm), 0.02, vg.ASCENT_ADAM, _t(a), _t(b))
    assert torch.equal(m1, m2) and torch.equal(o1, o2) and torch.equal(st1, st2)


def test_unconstrained_transforms_match_oracle():
    rng = np.random.default_rng(33)
    n, d = 7, 3001
    a = rng.uniform(1500, 2000, d).astype(np.float32).astype(np.float64)
    b = (a + rng.uniform(500, 1500, d)).astype(np.float32).astype(np.float64)
    m = (a + (b - a) * rng.uniform(0.02, 0.98, (n, d))).astype(np.float32).astype(np.float64)
    gm = (rng.standard_normal((n, d)) * 1e-3).astype(np.float32).astype(np.float64)
    th = vg.to_unconstrained(_t(m), _t(a), _t(b))
    th_ref = osvgd.to_unconstrained(m, a, b)
    assert np.abs(th.cpu().numpy() - th_ref).max() <= 1e-5 * np.abs(th_ref).max()
    thh = th.double().cpu().numpy()
    m2 = vg.to_model(th, _t(a), _t(b))
    assert rel(m2.cpu().numpy(), osvgd.to_model(thh, a, b)) <= 1e-6
    g = vg.unconstrained_gradient(th, _t(gm), _t(a), _t(b), gscale=-1.0)
    assert rel(g.cpu().numpy(), osvgd.unconstrained_gradient(thh, -gm, a, b)) <= 1e-5


@pytest.mark.parametrize("stochastic", [False, True])
def test_svgd_in_unconstrained_space_matches_oracle(stochastic):
    """One update of theta = T(m) with the transformed gradient (strategy 2 of
    the uniform prior): vip_unconstrained_gradient then svgd_step /
    ssvgd_step without bounds, against the oracle."""
    rng = np.random.default_rng(34)
    n, d = 24, 2000
    a = rng.uniform(1500, 2000, d).astype(np.float32).astype(np.float64)
    b = (a + rng.uniform(500, 1500, d)).astype(np.float32).astype(np.float64)
    th = (rng.standard_normal((n, d)) * 1.5).astype(np.float32).astype(np.float64)
    gm = (rng.standard_normal((n, d)) * 1e-2).astype(np.float32).astype(np.float64)
    tht = _t(th)
    g = vg.unconstrained_gradient(tht, _t(gm), _t(a), _t(b))
    eps = 0.05
    if not stochastic:
        vg.svgd_step(tht, g, eps)
        ref, _ = osvgd.svgd_step_unconstrained(th, gm, eps, a, b)
    else:
        xi = rng.standard_normal((n, d)).astype(np.float32).astype(np.float64)
        vg.ssvgd_step(tht, g, eps, seed=0, it=0, xi=_t(xi))
        ref, _, _ = osvgd.ssvgd_step_unconstrained(th, gm, eps, xi, a, b)
    assert rel(tht.double().cpu().numpy() - th, ref - th) <= 1e-5


# ---------------------------------------------------------------------------
# low-rank-plus-diagonal ADVI

@pytest.mark.parametrize("bounded", [True, False])
def test_advi_lowrank_sample_and_step_match_oracle(bounded):
    d, S, r = 2000, 16, 4
    mu, om, eta, gm, a, b = _advi_case(d, S, 51, bounded)
    rng = np.random.default_rng(52)
    B = (rng.standard_normal((d, r)) * 0.05).astype(np.float32).astype(np.float64)
    eps = rng.standard_normal((S, r)).astype(np.float32).astype(np.float64)
    ta = None if a is None else _t(a)
    tb = None if b is None else _t(b)
    m = vg.advi_lowrank_sample(_t(mu), _t(om), _t(B), _t(eta), _t(eps), ta, tb)
    assert rel(m.cpu().numpy(), oadvi.sample_lowrank(mu, om, B, eta, eps, a, b)) <= 1e-6
    st = torch.zeros(4 * d + 2 * d * r, device=DEV)
    mut, omt, Bt = _t(mu), _t(om), _t(B)
    state = tuple(np.zeros_like(x) for x in (mu, mu, om, om, B, B))
    mur, omr, Br = mu.copy(), om.copy(), B.copy()
    work = None
    for t in (1, 2, 3):
        work = vg.advi_lowrank_step(mut, omt, Bt, st, t, _t(eta), _t(eps), _t(gm), 0.01, ta, tb,
                                    work=work)
        mur, omr, Br, state = oadvi.advi_lowrank_step(mur, omr, Br, state, t, eta, eps, gm, 0.01,
                                                      a, b)
    assert rel(mut.double().cpu().numpy() - mu, mur - mu) <= 1e-5
    assert rel(omt.double().cpu().numpy() - om, omr - om) <= 1e-5
    assert rel(Bt.double().cpu().numpy() - B, Br - B) <= 1e-5


def test_advi_lowrank_with_zero_B_is_meanfield_step():
    d, S, r = 3000, 16, 3
    mu, om, eta, gm, a, b = _advi_case(d, S, 53, True)
    eps = _t(np.random.default_rng(54).standard_normal((S, r)))
    st1 = torch.zeros((4, d), device=DEV)
    st2 = torch.zeros(4 * d + 2 * d * r, device=DEV)
    m1, o1, m2, o2 = _t(mu), _t(om), _t(mu), _t(om)
    Bz = torch.zeros((d, r), device=DEV)
    for t in (1, 2):
        vg.advi_step(m1, o1, st1, t, _t(eta), _t(gm), 0.02, _t(a), _t(b))
        vg.advi_lowrank_step(m2, o2, Bz.clone(), st2, t, _t(eta), eps, _t(gm), 0.02, _t(a), _t(b))
    assert rel(m2.double().cpu().numpy() - mu, m1.double().cpu().numpy() - mu) <= 1e-6
    assert rel(o2.double().cpu().numpy() - om, o1.double().cpu().numpy() - om) <= 1e-6
