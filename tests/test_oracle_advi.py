"""Pins of the FP64 mean-field ADVI oracle.

* logit transform: T^{-1}(T(m)) = m, and the chain-rule / log-det terms agree
  with finite differences of T^{-1} and log|dT^{-1}/dtheta|;
* one step: the Monte-Carlo ELBO gradients equal central differences of the
  ELBO estimator at fixed eta (Eq. 10-11 restricted to the diagonal);
* optimum: on a linear-Gaussian target the mean-field optimum is
  mu = posterior mean, sigma_i = 1 / sqrt(Lambda_ii) (closed form), reached
  by each ascent rule (SGD, ADAGRAD, ADADELTA, ADAM);
* first steps in closed form: ADAGRAD moves by lr sign(g); ADADELTA by
  sqrt(eps) g / sqrt((1 - rho) g^2 + eps); SGD by lr g.

Low-rank-plus-diagonal ADVI (Sigma = diag(e^{2 omega}) + B B^T):
* B = 0 reduces to the mean-field gradients;
* the gradients equal central differences of the ELBO estimator
  mean_s [log p(m_s) + log|J|] + 1/2 log|Sigma| at fixed eta, eps;
* on a Gaussian target whose covariance is diagonal plus rank one, rank-1
  ADVI recovers the mean and the full covariance.
"""
import numpy as np
import pytest

from oracle import advi


def test_transform_roundtrip_and_derivatives():
    rng = np.random.default_rng(0)
    a = rng.uniform(1000, 2000, 50)
    b = a + rng.uniform(500, 2000, 50)
    m = a + rng.uniform(0.01, 0.99, 50) * (b - a)
    assert np.allclose(advi.T_inv(advi.T(m, a, b), a, b), m, rtol=1e-13)
    th = rng.standard_normal(50) * 2
    e = 1e-6
    dm = (advi.T_inv(th + e, a, b) - advi.T_inv(th - e, a, b)) / (2 * e)
    s = 1 / (1 + np.exp(-th))
    assert np.allclose(dm, (b - a) * s * (1 - s), rtol=1e-8)

    def logdet(t):
        return np.log((advi.T_inv(t + 1e-5, a, b) - advi.T_inv(t - 1e-5, a, b))
                      / 2e-5)
    dld = (logdet(th + 1e-3) - logdet(th - 1e-3)) / 2e-3
    assert np.allclose(dld, 1 - 2 * s, rtol=1e-4, atol=1e-5)


def _gauss_target(d, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((d, d))
    Lam = B @ B.T + d * np.eye(d)
    mu = rng.standard_normal(d)
    return mu, Lam


def test_one_step_gradients_equal_fd_of_elbo_estimator():
    d, S = 4, 6
    rng = np.random.default_rng(1)
    a = np.full(d, -3.0)
    b = np.full(d, 4.0)
    mu_t, Lam = _gauss_target(d, 2)

    def logp(m):                       # Gaussian log density on m (unnormalised)
        r = m - mu_t[None, :]
        return -0.5 * np.einsum("si,ij,sj->s", r, Lam, r)

    def dlogp(m):
        return -(m - mu_t[None, :]) @ Lam.T

    eta = rng.standard_normal((S, d))
    mu = rng.standard_normal(d) * 0.3
    om = rng.standard_normal(d) * 0.2 - 0.5

    def elbo_hat(mu, om):
        th = mu[None, :] + np.exp(om)[None, :] * eta
        m = advi.T_inv(th, a[None, :], b[None, :])
        s = 1 / (1 + np.exp(-th))
        ld = np.log((b - a)[None, :] * s * (1 - s)).sum(axis=1)
        return np.mean(logp(m) + ld) + om.sum()

    m_s = advi.sample(mu, om, eta, a, b)
    gmu, gom = advi.elbo_gradients(mu, om, eta, dlogp(m_s), a, b)
    e = 1e-6
    for i in range(d):
        u = np.zeros(d)
        u[i] = e
        fmu = (elbo_hat(mu + u, om) - elbo_hat(mu - u, om)) / (2 * e)
        fom = (elbo_hat(mu, om + u) - elbo_hat(mu, om - u)) / (2 * e)
        assert np.isclose(gmu[i], fmu, rtol=1e-6, atol=1e-7)
        assert np.isclose(gom[i], fom, rtol=1e-6, atol=1e-7)


def test_adam_first_step_moves_by_lr():
    p = np.zeros(3)
    g = np.array([2.0, -0.5, 1e-3])
    p1, m1, m2 = advi.adam_ascent(p, g, np.zeros(3), np.zeros(3), 1, 0.1)
    # bias-corrected first step is lr * sign(g) up to the epsilon term
    assert np.allclose(p1, 0.1 * np.sign(g), rtol=1e-4)


def test_meanfield_optimum_linear_gaussian():
    d = 3
    mu_t, Lam = _gauss_target(d, 5)
    rng = np.random.default_rng(7)
    mu = np.zeros(d)
    om = np.zeros(d)
    st = tuple(np.zeros(d) for _ in range(4))
    S = 64
    for t in range(1, 3001):
        eta = rng.standard_normal((S, d))
        m = advi.sample(mu, om, eta)
        gm = -(m - mu_t[None, :]) @ Lam.T
        lr = 0.05 if t < 2000 else 0.005
        mu, om, st = advi.advi_step(mu, om, st, t, eta, gm, lr)
    assert np.allclose(mu, mu_t, atol=0.02)
    assert np.allclose(np.exp(om), 1 / np.sqrt(np.diag(Lam)), rtol=0.03)


def test_first_steps_of_the_ascent_rules():
    g = np.array([2.0, -0.5, 1e-3])
    z = np.zeros(3)
    p, s1, s2 = advi.ascend(z, g, z, z, 1, 0.1, advi.SGD)
    assert np.allclose(p, 0.1 * g, rtol=1e-15)
    p, s1, s2 = advi.ascend(z, g, z, z, 1, 0.1, advi.ADAGRAD)
    assert np.allclose(p, 0.1 * np.sign(g), rtol=1e-4)
    assert np.allclose(s1, g * g, rtol=1e-15)
    p, s1, s2 = advi.ascend(z, g, z, z, 1, 1.0, advi.ADADELTA)
    rho, e = advi.ADADELTA_RHO, advi.ADADELTA_EPS
    dx = np.sqrt(e) * g / np.sqrt((1 - rho) * g * g + e)
    assert np.allclose(p, dx, rtol=1e-13)
    assert np.allclose(s2, (1 - rho) * dx * dx, rtol=1e-13)


def test_every_ascent_rule_reaches_the_meanfield_optimum():
    d = 3
    mu_t, Lam = _gauss_target(d, 5)
    rates = {advi.SGD: (0.05, 0.005), advi.ADAGRAD: (0.5, 0.05),
             advi.ADADELTA: (1.0, 0.2), advi.ADAM: (0.05, 0.005)}
    for opt, (lr0, lr1) in rates.items():
        rng = np.random.default_rng(7)
        mu = np.zeros(d)
        om = np.zeros(d)
        st = tuple(np.zeros(d) for _ in range(4))
        for t in range(1, 3001):
            eta = rng.standard_normal((64, d))
            m = advi.sample(mu, om, eta)
            gm = -(m - mu_t[None, :]) @ Lam.T
            mu, om, st = advi.advi_step_opt(mu, om, st, t, eta, gm, lr0 if t < 2000 else lr1, opt)
        assert np.allclose(mu, mu_t, atol=0.02), opt
        assert np.allclose(np.exp(om), 1 / np.sqrt(np.diag(Lam)), rtol=0.03), opt


# ---------------------------------------------------------------------------
# low-rank-plus-diagonal ADVI

def test_lowrank_with_zero_B_is_meanfield():
    rng = np.random.default_rng(40)
    d, r, S = 6, 2, 5
    mu, om = rng.standard_normal(d), rng.standard_normal(d) * 0.3
    eta, eps = rng.standard_normal((S, d)), rng.standard_normal((S, r))
    gm = rng.standard_normal((S, d))
    a = rng.uniform(0, 1, d)
    b = a + rng.uniform(1, 2, d)
    g1 = advi.elbo_gradients_lowrank(mu, om, np.zeros((d, r)), eta, eps, gm, a, b)
    g0 = advi.elbo_gradients(mu, om, eta, gm, a, b)
    assert np.allclose(g1[0], g0[0], rtol=1e-13)
    assert np.allclose(g1[1], g0[1], rtol=1e-12)
    # with B = 0 the B-gradient is the sample covariance of g and eps alone
    sg = 1 / (1 + np.exp(-(mu[None, :] + np.exp(om)[None, :] * eta)))
    g = gm * (b - a)[None, :] * sg * (1 - sg) + (1 - 2 * sg)
    assert np.allclose(g1[2], g.T @ eps / S, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("bounded", [False, True])
def test_lowrank_gradients_equal_fd_of_elbo_estimator(bounded):
    rng = np.random.default_rng(41)
    d, r, S = 5, 2, 4
    mu, om = rng.standard_normal(d) * 0.3, rng.standard_normal(d) * 0.2
    B = rng.standard_normal((d, r)) * 0.4
    eta, eps = rng.standard_normal((S, d)), rng.standard_normal((S, r))
    c, prec = rng.standard_normal(d), np.diag(rng.uniform(0.5, 2.0, d))
    a = rng.uniform(-3, -2, d) if bounded else None
    b = rng.uniform(2, 3, d) if bounded else None

    def estimator(mu, om, B):
        th = mu[None, :] + np.exp(om)[None, :] * eta + eps @ B.T
        if bounded:
            m = advi.T_inv(th, a[None, :], b[None, :])
            sg = 1 / (1 + np.exp(-th))
            logj = np.log((b - a)[None, :] * sg * (1 - sg)).sum(axis=1)
        else:
            m, logj = th, 0.0
        logp = -0.5 * np.einsum("si,ij,sj->s", m - c, prec, m - c)
        Sigma = np.diag(np.exp(2 * om)) + B @ B.T
        return np.mean(logp + logj) + 0.5 * np.linalg.slogdet(Sigma)[1]

    th = mu[None, :] + np.exp(om)[None, :] * eta + eps @ B.T
    m = advi.T_inv(th, a[None, :], b[None, :]) if bounded else th
    gm = -(m - c) @ prec
    gmu, gom, gB = advi.elbo_gradients_lowrank(mu, om, B, eta, eps, gm, a, b)
    h = 1e-6
    for k in range(d):
        e = np.eye(d)[k] * h
        assert np.isclose(gmu[k], (estimator(mu + e, om, B) - estimator(mu - e, om, B)) / (2 * h),
                          rtol=1e-6, atol=1e-7)
        assert np.isclose(gom[k], (estimator(mu, om + e, B) - estimator(mu, om - e, B)) / (2 * h),
                          rtol=1e-6, atol=1e-7)
        for j in range(r):
            E = np.zeros((d, r)); E[k, j] = h
            fd = (estimator(mu, om, B + E) - estimator(mu, om, B - E)) / (2 * h)
            assert np.isclose(gB[k, j], fd, rtol=1e-6, atol=1e-7)


def test_lowrank_recovers_diagonal_plus_rank_one_posterior():
    rng = np.random.default_rng(42)
    d = 4
    c = rng.standard_normal(d)
    u = rng.standard_normal(d) * 0.8
    Sig_t = np.diag(rng.uniform(0.2, 0.5, d) ** 2) + np.outer(u, u)
    prec = np.linalg.inv(Sig_t)
    mu, om, B = np.zeros(d), np.zeros(d), rng.standard_normal((d, 1)) * 0.1
    st = tuple(np.zeros_like(x) for x in (mu, mu, om, om, B, B))
    for t in range(1, 6001):
        eta, eps = rng.standard_normal((64, d)), rng.standard_normal((64, 1))
        m = advi.sample_lowrank(mu, om, B, eta, eps)
        gm = -(m - c[None, :]) @ prec
        lr = 0.02 if t < 4000 else 0.002
        mu, om, B, st = advi.advi_lowrank_step(mu, om, B, st, t, eta, eps, gm, lr)
    Sig = np.diag(np.exp(2 * om)) + B @ B.T
    assert np.allclose(mu, c, atol=0.03)
    assert np.abs(Sig - Sig_t).max() <= 0.05 * np.abs(Sig_t).max()
