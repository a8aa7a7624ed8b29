"""FP64 oracle: SVGD (Eq. 13-17) and stochastic SVGD (Eq. 21-25).

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


def pairwise_sqdist(X):
    """D2[i, j] = sum_c (X[i, c] - X[j, c])^2, taken directly."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    D2 = np.zeros((n, n))
    for i in range(n):
        diff = X - X[i][None, :]
        D2[i] = np.einsum("jc,jc->j", diff, diff)
    return D2


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
