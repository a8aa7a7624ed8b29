"""FP64 oracle: SVGD (Eq. 13-17) and stochastic SVGD (Eq. 21-25), with the
RBF kernel or the diagonal matrix-valued kernel of the Discussion.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Particles X [n, d], gradients G [n, d] = grad log p(m_j | d_obs).

  RBF kernel (Eq. 16)   k(m, m') = exp(-|m - m'|^2 / (2 h^2))
  bandwidth             the paper calls h "a scale factor" and gives no rule;
                        the median heuristic is used: h^2 = med / (2 ln(n + 1)),
                        med the median of all n^2 squared distances including
                        the zero diagonal (mean of the two middle values when
                        n^2 is even); h^2 = 1 when med < 1e-30
  SVGD (Eq. 17)         phi(m_i) = 1/n sum_j [k(m_j, m_i) G_j + grad_{m_j} k(m_j, m_i)],
                        grad_{m_j} k(m_j, m_i) = k(m_j, m_i) (m_i - m_j) / h^2,
                        m_i <- m_i + eps phi(m_i)
  sSVGD (Eq. 22)        z <- z + eps [K grad log p + div K] + N(0, 2 eps K),
                        K = (1/n) Kbar (x) I_d; the drift equals phi above and
                        the noise is sqrt(2 eps / n) Lk Xi (Eq. 25) with
                        Lk = chol(Kbar) and Xi [n, d] standard normal; Kbar is
                        factorised with a jitter tau I (tau = 1e-6 n, times 10 on
                        failure, at most 3 retries)
  prior                 uniform bounds enforced by resetting to the nearest
                        bound (Sec. 3, first strategy)
"""
import numpy as np


def sqdist_rows(X, rows):
    """D2[rows, :] with D2[i, j] = sum_c (X[i, c] - X[j, c])^2, taken directly."""
    X = np.asarray(X, dtype=np.float64)
    rows = list(rows)
    D2 = np.zeros((len(rows), X.shape[0]))
    for k, i in enumerate(rows):
        diff = X - X[i][None, :]
        D2[k] = np.einsum("jc,jc->j", diff, diff)
    return D2


def pairwise_sqdist(X):
    """D2[i, j] = sum_c (X[i, c] - X[j, c])^2, taken directly."""
    X = np.asarray(X, dtype=np.float64)
    return sqdist_rows(X, range(X.shape[0]))


def median_bandwidth(D2):
    """h^2 from the median of all n^2 entries of D2."""
    n = D2.shape[0]
    med = float(np.median(D2.reshape(-1)))
    if med < 1e-30:
        return 1.0
    return med / (2.0 * np.log(n + 1.0))


def rbf(D2, h2):
    """Kbar[i, j] = k(m_i, m_j) (Eq. 16)."""
    return np.exp(-D2 / (2.0 * h2))


def svgd_direction(X, G, h2=None):
    """phi [n, d] of Eq. (17), with the bandwidth used and Kbar."""
    X = np.asarray(X, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    n = X.shape[0]
    D2 = pairwise_sqdist(X)
    if h2 is None or h2 <= 0:
        h2 = median_bandwidth(D2)
    K = rbf(D2, h2)
    attract = K @ G                       # sum_j k(m_j, m_i) G_j
    repulse = np.zeros_like(X)
    for i in range(n):                    # sum_j k(m_j, m_i) (m_i - m_j) / h^2
        repulse[i] = (K[i][:, None] * (X[i][None, :] - X)).sum(axis=0) / h2
    return (attract + repulse) / n, h2, K


def svgd_direction_rows(X, G, rows, D2, h2=None):
    """phi(m_i) of Eq. (17) for the particles i in rows only, given the full
    squared-distance matrix D2 (pairwise_sqdist): the same sums over j as
    svgd_direction, evaluated for those i. Returns (phi [len(rows), d], h2, K)."""
    X = np.asarray(X, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    n = X.shape[0]
    if h2 is None or h2 <= 0:
        h2 = median_bandwidth(D2)
    K = rbf(D2, h2)
    phi = np.zeros((len(rows), X.shape[1]))
    for k, i in enumerate(rows):
        attract = K[i] @ G                                   # sum_j k(m_j, m_i) G_j
        repulse = (K[i][:, None] * (X[i][None, :] - X)).sum(axis=0) / h2
        phi[k] = (attract + repulse) / n
    return phi, h2, K


def svgd_step_rows(X, G, eps, rows, D2, h2=None, lo=None, hi=None):
    """Rows of svgd_step: the updated particles i in rows."""
    X = np.asarray(X, dtype=np.float64)
    phi, h2u, _ = svgd_direction_rows(X, G, rows, D2, h2)
    lo_ = None if lo is None else np.asarray(lo, dtype=np.float64).reshape(-1)
    hi_ = None if hi is None else np.asarray(hi, dtype=np.float64).reshape(-1)
    return clip(X[list(rows)] + eps * phi, lo_, hi_), h2u


def ssvgd_step_rows(X, G, eps, xi, rows, D2, h2=None, lo=None, hi=None):
    """Rows of ssvgd_step: the updated particles i in rows, with the noise
    sqrt(2 eps / n) (Lk xi)_i of Eq. (25) (Lk from the full kernel matrix).
    Returns (X_new[rows], h2, tau)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    phi, h2u, K = svgd_direction_rows(X, G, rows, D2, h2)
    L, tau = jittered_cholesky(K)
    xi = np.asarray(xi, dtype=np.float64)
    noise = np.sqrt(2.0 * eps / n) * np.stack([L[i] @ xi for i in rows])
    lo_ = None if lo is None else np.asarray(lo, dtype=np.float64).reshape(-1)
    hi_ = None if hi is None else np.asarray(hi, dtype=np.float64).reshape(-1)
    return clip(X[list(rows)] + eps * phi + noise, lo_, hi_), h2u, tau


def clip(X, lo, hi):
    if lo is None and hi is None:
        return X
    lo = -np.inf if lo is None else np.asarray(lo, dtype=np.float64).reshape(1, -1)
    hi = np.inf if hi is None else np.asarray(hi, dtype=np.float64).reshape(1, -1)
    return np.minimum(np.maximum(X, lo), hi)


def svgd_step(X, G, eps, h2=None, lo=None, hi=None):
    """One SVGD update (Eq. 17) followed by the bound reset."""
    phi, h2u, _ = svgd_direction(X, G, h2)
    return clip(np.asarray(X, dtype=np.float64) + eps * phi, lo, hi), h2u


def jittered_cholesky(K):
    """Lower Cholesky factor of K + tau I, tau = 1e-6 n, x10 per failure, at
    most 3 retries. Returns (L, tau)."""
    n = K.shape[0]
    tau = 1e-6 * n
    for _ in range(4):
        try:
            return np.linalg.cholesky(K + tau * np.eye(n)), tau
        except np.linalg.LinAlgError:
            tau *= 10.0
    raise np.linalg.LinAlgError("kernel matrix not positive definite")


def ssvgd_step(X, G, eps, xi, h2=None, lo=None, hi=None):
    """One stochastic SVGD update (Eq. 22 with the noise of Eq. 25).

    xi [n, d] standard normal draws (Xi). Returns (X_new, h2, tau)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    phi, h2u, K = svgd_direction(X, G, h2)
    L, tau = jittered_cholesky(K)
    noise = np.sqrt(2.0 * eps / n) * (L @ np.asarray(xi, dtype=np.float64))
    return clip(X + eps * phi + noise, lo, hi), h2u, tau


# ---------------------------------------------------------------------------
# Diagonal matrix-valued kernel (Discussion of the paper; Wang et al. 2019).
#
# With a positive diagonal preconditioner Q = diag(q), the kernel is the
# matrix K_Q(m', m) = Q^{-1} k_Q(m', m), where k_Q is the RBF kernel in the
# Q-metric, k_Q(m', m) = exp(-(m' - m)^T Q (m' - m) / (2 h^2)), and h^2 follows
# the median rule on the Q-weighted squared distances. The SVGD direction
# (Eq. 17 with this kernel) is
#   phi(m_i) = 1/n sum_j [K_Q(m_j, m_i) G_j + div_{m_j} K_Q(m_j, m_i)],
# the divergence taken over the columns of K_Q: for a diagonal constant Q it
# is Q^{-1} grad_{m_j} k_Q(m_j, m_i). The paper sets q to the inverse of the
# variance of each coordinate across the particles (population variance
# here; coordinates with zero variance get q = 1). For sSVGD the diffusion
# matrix becomes (1/n) Kbar (x) Q^{-1}, whose square root is
# (1/sqrt(n)) Lk (x) Q^{-1/2}.

def inverse_variance(X):
    """q [d]: 1 / Var_j(X[j, c]) (population variance over the particles),
    1 where the variance is zero."""
    X = np.asarray(X, dtype=np.float64)
    var = ((X - X.mean(axis=0, keepdims=True)) ** 2).mean(axis=0)
    q = np.ones_like(var)
    pos = var > 0
    q[pos] = 1.0 / var[pos]
    return q


def pairwise_sqdist_q(X, q):
    """D2[i, j] = sum_c q_c (X[i, c] - X[j, c])^2, taken directly."""
    X = np.asarray(X, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64).reshape(1, -1)
    n = X.shape[0]
    D2 = np.zeros((n, n))
    for i in range(n):
        diff = X - X[i][None, :]
        D2[i] = (q * diff * diff).sum(axis=1)
    return D2


def svgd_direction_q(X, G, q, h2=None):
    """phi [n, d] with the diagonal matrix-valued kernel, the bandwidth used
    and the scalar factor k_Q as Kbar."""
    X = np.asarray(X, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    n = X.shape[0]
    D2 = pairwise_sqdist_q(X, q)
    if h2 is None or h2 <= 0:
        h2 = median_bandwidth(D2)
    K = rbf(D2, h2)                        # k_Q(m_i, m_j)
    qinv = 1.0 / q
    phi = np.zeros_like(X)
    for i in range(n):
        for j in range(n):
            # K_Q(m_j, m_i) G_j = Q^{-1} k_Q G_j
            drive = qinv * (K[i, j] * G[j])
            # grad_{m_j} k_Q(m_j, m_i) = k_Q Q (m_i - m_j) / h^2, times Q^{-1}
            grad_k = K[i, j] * q * (X[i] - X[j]) / h2
            phi[i] += drive + qinv * grad_k
    return phi / n, h2, K


def svgd_step_q(X, G, q, eps, h2=None, lo=None, hi=None):
    """One SVGD update with the diagonal matrix-valued kernel, then the bound
    reset."""
    phi, h2u, _ = svgd_direction_q(X, G, q, h2)
    return clip(np.asarray(X, dtype=np.float64) + eps * phi, lo, hi), h2u


def ssvgd_step_q(X, G, q, eps, xi, h2=None, lo=None, hi=None):
    """One stochastic SVGD update with the diagonal matrix-valued kernel:
    drift phi above, noise sqrt(2 eps / n) (Lk Xi) Q^{-1/2} (column c scaled
    by 1/sqrt(q_c)). Returns (X_new, h2, tau)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    phi, h2u, K = svgd_direction_q(X, G, q, h2)
    L, tau = jittered_cholesky(K)
    noise = np.sqrt(2.0 * eps / n) * (L @ np.asarray(xi, dtype=np.float64))
    noise = noise / np.sqrt(np.asarray(q, dtype=np.float64))[None, :]
    return clip(X + eps * phi + noise, lo, hi), h2u, tau


# ---------------------------------------------------------------------------
# SVGD / sSVGD in the unconstrained space (Sec. 3, second strategy for the
# uniform prior): the particles are theta = T(m) with the logit transform of
# Eq. (12), T(m) = log(m - a) - log(b - m), m = T^{-1}(theta) =
# a + (b - a) / (1 + e^{-theta}), and the target is the density of theta,
# p(m(theta)) |dm/dtheta|. Its gradient, by the chain rule and the derivative
# of the log-Jacobian log((b - a) s (1 - s)), s = sigmoid(theta), is
#   grad_theta = grad_m log p * (b - a) s (1 - s) + (1 - 2 s).
# The update runs on theta without a bound reset.

def to_unconstrained(m, a, b):
    m = np.asarray(m, dtype=np.float64)
    return np.log(m - a) - np.log(b - m)


def to_model(theta, a, b):
    theta = np.asarray(theta, dtype=np.float64)
    return a + (b - a) / (1.0 + np.exp(-theta))


def unconstrained_gradient(theta, gm, a, b):
    """grad_theta log p_theta from gm = grad_m log p at m = T^{-1}(theta)."""
    s = 1.0 / (1.0 + np.exp(-np.asarray(theta, dtype=np.float64)))
    return np.asarray(gm, dtype=np.float64) * (b - a) * s * (1.0 - s) + (1.0 - 2.0 * s)


def svgd_step_unconstrained(theta, gm, eps, a, b, h2=None):
    """One SVGD update of theta (Eq. 17) for the transformed target."""
    g = unconstrained_gradient(theta, gm, a, b)
    return svgd_step(theta, g, eps, h2)


def ssvgd_step_unconstrained(theta, gm, eps, xi, a, b, h2=None):
    """One sSVGD update of theta (Eq. 22, 25) for the transformed target."""
    g = unconstrained_gradient(theta, gm, a, b)
    return ssvgd_step(theta, g, eps, xi, h2)
