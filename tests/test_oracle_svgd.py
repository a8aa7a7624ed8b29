"""Pins of the FP64 SVGD / sSVGD oracle.

* brute force on tiny inputs: phi of Eq. (17) rebuilt from kernel values and
  finite-difference kernel gradients (pins the sign of grad k);
* median: a plain sort of all n^2 entries;
* n = 1 SVGD is gradient ascent and reaches the closed-form MAP of a
  linear-Gaussian toy;
* fixed point on a Gaussian target: the kernel-weighted particle mean equals
  the target mean; the repulsive terms sum to zero over particles;
* sSVGD with n = 1 is the unadjusted Langevin algorithm, whose stationary
  variance on N(mu, s^2) is s^2 / (1 - eps / (2 s^2));
* sSVGD noise covariance is (2 eps / n) (Kbar + tau I).

Diagonal matrix-valued kernel (Q = diag(q)):
* q = 1 reduces to the RBF kernel exactly;
* brute force: phi rebuilt from Q^{-1} k_Q and finite-difference gradients of
  k_Q (pins the Q^{-1} factor and the Q-metric);
* change of coordinates: the RBF SVGD / sSVGD of z = sqrt(q) m with
  gradients G / sqrt(q) and the same noise, mapped back by 1 / sqrt(q);
* n = 1 is preconditioned gradient ascent, phi = G / q;
* q from the particles is the inverse population variance.

Unconstrained (logit) space:
* T and T^{-1} invert each other; the transformed gradient equals central
  differences of log p(T^{-1}(theta)) + log|dT^{-1}/dtheta| for a Gaussian
  log p in m;
* one particle on a uniform target ascends the logistic density of theta to
  its mode theta = 0 (the middle of the box).
"""
import numpy as np

from oracle import svgd


def _rbf_scalar(a, b, h2):
    return np.exp(-np.sum((a - b) ** 2) / (2 * h2))


def test_phi_brute_force_tiny():
    rng = np.random.default_rng(0)
    n, d = 3, 2
    X = rng.standard_normal((n, d))
    G = rng.standard_normal((n, d))
    h2 = 0.7
    phi, h2u, K = svgd.svgd_direction(X, G, h2)
    assert h2u == h2
    e = 1e-6
    for i in range(n):
        acc = np.zeros(d)
        for j in range(n):
            acc += _rbf_scalar(X[j], X[i], h2) * G[j]
            # gradient of k(m_j, m_i) with respect to its first argument m_j
            for c in range(d):
                xp = X[j].copy()
                xm = X[j].copy()
                xp[c] += e
                xm[c] -= e
                acc[c] += (_rbf_scalar(xp, X[i], h2)
                           - _rbf_scalar(xm, X[i], h2)) / (2 * e)
        assert np.allclose(phi[i], acc / n, rtol=1e-8, atol=1e-10)
    for i in range(n):
        for j in range(n):
            assert np.isclose(K[i, j], _rbf_scalar(X[i], X[j], h2), rtol=1e-14)


def test_median_bandwidth_matches_sort():
    rng = np.random.default_rng(1)
    for n in (8, 7):
        X = rng.standard_normal((n, 5))
        D2 = svgd.pairwise_sqdist(X)
        allv = sorted(D2.reshape(-1).tolist())
        m = len(allv)
        med = allv[m // 2] if m % 2 else 0.5 * (allv[m // 2 - 1] + allv[m // 2])
        assert np.isclose(svgd.median_bandwidth(D2), med / (2 * np.log(n + 1)),
                          rtol=1e-15)
        # squared distances by explicit double loop
        for i in range(n):
            for j in range(n):
                assert np.isclose(D2[i, j], sum((X[i] - X[j]) ** 2), rtol=1e-13)
    assert svgd.median_bandwidth(np.zeros((4, 4))) == 1.0


def _linear_gaussian(d=3, m=5, seed=2):
    """y = A x + e, e ~ N(0, s^2 I), prior x ~ N(x0, P0). Returns the posterior
    mean, precision and a gradient function of the log posterior."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, d))
    x_true = rng.standard_normal(d)
    s = 0.3
    y = A @ x_true + s * rng.standard_normal(m)
    x0 = np.zeros(d)
    P0inv = np.eye(d) / 4.0
    Lam = A.T @ A / s ** 2 + P0inv
    mu = np.linalg.solve(Lam, A.T @ y / s ** 2 + P0inv @ x0)

    def grad_logp(X):
        return -(X - mu[None, :]) @ Lam.T
    return mu, Lam, grad_logp


def test_single_particle_svgd_reaches_map():
    mu, Lam, grad_logp = _linear_gaussian()
    X = np.zeros((1, mu.size))
    eps = 0.5 / np.linalg.eigvalsh(Lam).max()
    for _ in range(4000):
        X, _ = svgd.svgd_step(X, grad_logp(X), eps)
    assert np.allclose(X[0], mu, rtol=0, atol=1e-10)


def test_fixed_point_weighted_mean_and_zero_repulsion():
    rot = np.array([[np.cos(0.4), -np.sin(0.4)], [np.sin(0.4), np.cos(0.4)]])
    Lam = rot @ np.diag([1.0, 2.0]) @ rot.T
    mu = np.array([0.3, -0.2])

    def grad_logp(X):
        return -(X - mu[None, :]) @ Lam.T
    rng = np.random.default_rng(3)
    X = mu[None, :] + rng.standard_normal((6, 2))
    for _ in range(8000):
        X, _ = svgd.svgd_step(X, grad_logp(X), 0.25, h2=0.5)
    phi, h2, K = svgd.svgd_direction(X, grad_logp(X), 0.5)
    assert np.abs(phi).max() < 1e-9
    w = K.sum(axis=0)                              # sum_i k_ij
    resid = (w[:, None] * ((X - mu[None, :]) @ Lam.T)).sum(axis=0)
    assert np.abs(resid).max() < 1e-8
    # the particles do not collapse onto the mean
    assert svgd.pairwise_sqdist(X)[np.triu_indices(6, 1)].min() > 1e-2
    # sum over i of the repulsive terms is zero for any particle set
    Y = rng.standard_normal((5, 4))
    D2 = svgd.pairwise_sqdist(Y)
    Ky = svgd.rbf(D2, 1.3)
    rep = np.array([(Ky[i][:, None] * (Y[i][None, :] - Y)).sum(axis=0)
                    for i in range(5)])
    assert np.abs(rep.sum(axis=0)).max() < 1e-13


def test_single_particle_ssvgd_is_ula_with_known_variance():
    mu0, s2, eps = 0.3, 1.0, 0.5
    d = 20000
    rng = np.random.default_rng(4)
    x = np.full((1, d), mu0)
    samples = []
    for t in range(350):
        G = -(x - mu0) / s2
        x, _, tau = svgd.ssvgd_step(x, G, eps, rng.standard_normal((1, d)))
        if t >= 50:
            samples.append(x[0].copy())
    S = np.array(samples)
    var = S.var()
    expect = s2 / (1 - eps / (2 * s2)) * (1 + tau)
    # 3-sigma Monte-Carlo band; the chain decorrelates in ~2 steps
    n_eff = S.size / 4.0
    assert abs(var - expect) < 3 * expect * np.sqrt(2 / n_eff), (var, expect)
    assert abs(S.mean() - mu0) < 3 * np.sqrt(expect / n_eff)


def test_ssvgd_noise_covariance_is_scaled_kernel():
    rng = np.random.default_rng(6)
    n, d = 4, 200000
    X = rng.standard_normal((n, 3)) * 0.8
    # replicate the particle set along extra coordinates with zero spread so
    # that Kbar is unchanged while d grows
    Xd = np.concatenate([X, np.zeros((n, d - 3))], axis=1)
    G = np.zeros_like(Xd)
    eps = 0.01
    xi = rng.standard_normal((n, d))
    Xn, h2, tau = svgd.ssvgd_step(Xd, G, eps, xi, h2=1.1)
    Xs, _ = svgd.svgd_step(Xd, G, eps, h2=1.1)
    noise = Xn - Xs
    C = noise @ noise.T / d
    K = svgd.rbf(svgd.pairwise_sqdist(X), 1.1)
    target = 2 * eps / n * (K + tau * np.eye(n))
    assert np.abs(C - target).max() < 4 * (2 * eps / n) * np.sqrt(2.0 / d) * 2
    # the factor itself: L L^T = K + tau I and L lower triangular
    L, tau2 = svgd.jittered_cholesky(K)
    assert np.allclose(L @ L.T, K + tau2 * np.eye(n), rtol=0, atol=1e-14)
    assert np.all(np.triu(L, 1) == 0)


def test_clip_resets_to_nearest_bound():
    X = np.array([[0.5, 3.0, -2.0]])
    out = svgd.clip(X, np.array([0.0, 0.0, -1.0]), np.array([1.0, 2.0, 1.0]))
    assert np.array_equal(out, [[0.5, 2.0, -1.0]])


# ---------------------------------------------------------------------------
# diagonal matrix-valued kernel

def _case_q(n, d, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)) * rng.uniform(0.2, 5.0, size=(1, d))
    G = rng.standard_normal((n, d))
    q = svgd.inverse_variance(X)
    return X, G, q


def test_matrix_kernel_with_unit_q_is_the_rbf_kernel():
    X, G, _ = _case_q(5, 7, 1)
    q = np.ones(7)
    phi_q, h2_q, K_q = svgd.svgd_direction_q(X, G, q)
    phi, h2, K = svgd.svgd_direction(X, G)
    assert np.isclose(h2_q, h2, rtol=1e-14)
    assert np.allclose(phi_q, phi, rtol=1e-13, atol=1e-14)
    xi = np.random.default_rng(2).standard_normal(X.shape)
    a = svgd.ssvgd_step_q(X, G, q, 0.01, xi)[0]
    b = svgd.ssvgd_step(X, G, 0.01, xi)[0]
    assert np.allclose(a, b, rtol=1e-13, atol=1e-14)


def test_matrix_kernel_phi_brute_force_tiny():
    X, G, q = _case_q(3, 2, 3)
    phi, h2, _ = svgd.svgd_direction_q(X, G, q)
    n, d = X.shape

    def kq(a, b):
        return np.exp(-np.sum(q * (a - b) ** 2) / (2 * h2))

    ref = np.zeros_like(X)
    e = 1e-6
    for i in range(n):
        for j in range(n):
            grad = np.zeros(d)
            for c in range(d):
                dp = X[j].copy(); dp[c] += e
                dm = X[j].copy(); dm[c] -= e
                grad[c] = (kq(dp, X[i]) - kq(dm, X[i])) / (2 * e)
            # K_Q = Q^{-1} k_Q; its divergence in m_j is Q^{-1} grad k_Q
            ref[i] += (kq(X[j], X[i]) * G[j] + grad) / q
    ref /= n
    assert np.allclose(phi, ref, rtol=1e-7, atol=1e-9)


def test_matrix_kernel_is_rbf_svgd_in_scaled_coordinates():
    X, G, q = _case_q(6, 5, 4)
    s = np.sqrt(q)[None, :]
    phi_q, h2_q, _ = svgd.svgd_direction_q(X, G, q)
    phi_z, h2_z, _ = svgd.svgd_direction(X * s, G / s)
    assert np.isclose(h2_q, h2_z, rtol=1e-12)
    assert np.allclose(phi_q, phi_z / s, rtol=1e-10, atol=1e-12)
    xi = np.random.default_rng(5).standard_normal(X.shape)
    eps = 0.03
    Xq = svgd.ssvgd_step_q(X, G, q, eps, xi)[0]
    Zn = svgd.ssvgd_step(X * s, G / s, eps, xi)[0]
    assert np.allclose(Xq, Zn / s, rtol=1e-10, atol=1e-12)


def test_matrix_kernel_single_particle_is_preconditioned_ascent():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((1, 4))
    G = rng.standard_normal((1, 4))
    q = np.array([0.5, 2.0, 4.0, 10.0])
    phi, _, _ = svgd.svgd_direction_q(X, G, q)
    assert np.allclose(phi, G / q, rtol=1e-14)


def test_inverse_variance_is_population_variance():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((9, 6)) * 3.0
    X[:, 2] = 1.5                              # zero variance -> q = 1
    q = svgd.inverse_variance(X)
    var = np.var(X, axis=0)                    # numpy: population variance
    assert q[2] == 1.0
    m = np.arange(6) != 2
    assert np.allclose(q[m], 1.0 / var[m], rtol=1e-13)


# ---------------------------------------------------------------------------
# unconstrained (logit) space

def test_unconstrained_transform_and_gradient():
    rng = np.random.default_rng(8)
    d = 5
    a = rng.uniform(1000, 2000, d)
    b = a + rng.uniform(500, 3000, d)
    m = a + (b - a) * rng.uniform(0.05, 0.95, d)
    th = svgd.to_unconstrained(m, a, b)
    assert np.allclose(svgd.to_model(th, a, b), m, rtol=1e-13)
    c = a + 0.3 * (b - a)
    s2 = ((b - a) / 4) ** 2

    def logp_theta(t):
        mm = a + (b - a) / (1.0 + np.exp(-t))
        # log p(m) + log|dm/dtheta|, the Jacobian from central differences of m(theta)
        e = 1e-6
        dm = ((a + (b - a) / (1.0 + np.exp(-(t + e)))) - (a + (b - a) / (1.0 + np.exp(-(t - e))))) / (2 * e)
        return np.sum(-0.5 * (mm - c) ** 2 / s2) + np.sum(np.log(dm))

    gm = -(m - c) / s2
    g = svgd.unconstrained_gradient(th, gm, a, b)
    e = 1e-4
    fd = np.array([(logp_theta(th + e * np.eye(d)[k]) - logp_theta(th - e * np.eye(d)[k])) / (2 * e)
                   for k in range(d)])
    assert np.allclose(g, fd, rtol=1e-5, atol=1e-6)


def test_unconstrained_single_particle_uniform_target_reaches_mode():
    a = np.array([1500.0, 2000.0])
    b = np.array([3000.0, 2600.0])
    th = np.array([[2.5, -3.0]])
    for _ in range(400):
        th, _ = svgd.svgd_step_unconstrained(th, np.zeros_like(th), 0.5, a, b)
    assert np.allclose(th, 0.0, atol=1e-8)
    assert np.allclose(svgd.to_model(th, a, b), (a + b) / 2, rtol=1e-10)


def test_row_restricted_updates_equal_the_full_ones():
    """svgd_step_rows / ssvgd_step_rows evaluate the same sums as svgd_step /
    ssvgd_step for a subset of the particles (used where the full update of
    every particle is too slow for the oracle)."""
    rng = np.random.default_rng(21)
    n, d = 9, 40
    X = rng.standard_normal((n, d))
    G = rng.standard_normal((n, d))
    xi = rng.standard_normal((n, d))
    lo, hi = -np.full(d, 1.5), np.full(d, 1.5)
    rows = [0, 4, 8]
    D2 = svgd.pairwise_sqdist(X)
    brute = np.array([[((X[i] - X[j]) ** 2).sum() for j in range(n)] for i in range(n)])
    assert np.allclose(D2, brute, rtol=1e-14, atol=0)
    assert np.allclose(svgd.sqdist_rows(X, rows), brute[rows], rtol=1e-14, atol=0)
    full, h2 = svgd.svgd_step(X, G, 0.3, lo=lo, hi=hi)
    part, h2r = svgd.svgd_step_rows(X, G, 0.3, rows, D2, lo=lo, hi=hi)
    assert h2r == h2
    assert np.allclose(part, full[rows], rtol=1e-13, atol=1e-14)
    fulls, h2s, tau = svgd.ssvgd_step(X, G, 0.3, xi, lo=lo, hi=hi)
    parts, h2sr, taur = svgd.ssvgd_step_rows(X, G, 0.3, xi, rows, D2, lo=lo, hi=hi)
    assert taur == tau and h2sr == h2s
    assert np.allclose(parts, fulls[rows], rtol=1e-13, atol=1e-14)
