"""FP64 oracle: mean-field ADVI (Eq. 7-12) with Adam ascent.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Unconstrained variable theta = T(m), T the logit transform of Eq. (12):
  theta = log(m - a) - log(b - m),   m = T^{-1}(theta) = a + (b - a) / (1 + e^{-theta}).
Mean-field Gaussian q(theta) = N(mu, diag(e^{2 omega})), i.e. the Cholesky
factor L of Eq. (8) restricted to its diagonal, L_ii = e^{omega_i} (the
diagonal-covariance option of Sec. 5). With theta_s = mu + e^omega * eta_s,
eta_s ~ N(0, I), Eq. (10)-(11) become, per coordinate,

  g_s        = dlogp/dm(m_s) * dm/dtheta + d log|det J|/dtheta
             = dlogp/dm(m_s) * (b - a) s (1 - s) + (1 - 2 s),   s = sigmoid(theta_s)
  grad_mu    = mean_s g_s
  grad_omega = mean_s g_s eta_s e^omega + 1      ((L^{-1})^T on the diagonal,
                                                  times dL/domega = e^omega)

When a, b are None the transform is the identity (g_s = dlogp/dm).
The ELBO is ascended with Adam (beta1 0.9, beta2 0.999, eps 1e-8).
"""
import numpy as np

BETA1, BETA2, ADAM_EPS = 0.9, 0.999, 1e-8


def T(m, a, b):
    return np.log(m - a) - np.log(b - m)


def T_inv(theta, a, b):
    return a + (b - a) / (1.0 + np.exp(-theta))


def sample(mu, omega, eta, a=None, b=None):
    """m_s = T^{-1}(mu + e^omega eta_s), eta [S, d] -> [S, d]."""
    theta = mu[None, :] + np.exp(omega)[None, :] * eta
    if a is None:
        return theta
    return T_inv(theta, a[None, :], b[None, :])


def elbo_gradients(mu, omega, eta, gm, a=None, b=None):
    """Monte-Carlo grad_mu, grad_omega of the ELBO from S samples.

    gm [S, d] = d log p / dm at m_s."""
    theta = mu[None, :] + np.exp(omega)[None, :] * eta
    if a is None:
        g = np.asarray(gm, dtype=np.float64)
    else:
        s = 1.0 / (1.0 + np.exp(-theta))
        g = gm * (b - a)[None, :] * s * (1.0 - s) + (1.0 - 2.0 * s)
    grad_mu = g.mean(axis=0)
    grad_omega = (g * eta * np.exp(omega)[None, :]).mean(axis=0) + 1.0
    return grad_mu, grad_omega


def adam_ascent(p, grad, m1, m2, t, lr):
    """One Adam step that increases the objective; returns new (p, m1, m2)."""
    m1 = BETA1 * m1 + (1.0 - BETA1) * grad
    m2 = BETA2 * m2 + (1.0 - BETA2) * grad * grad
    mhat = m1 / (1.0 - BETA1 ** t)
    vhat = m2 / (1.0 - BETA2 ** t)
    return p + lr * mhat / (np.sqrt(vhat) + ADAM_EPS), m1, m2


def advi_step(mu, omega, state, t, eta, gm, lr, a=None, b=None):
    """One mean-field ADVI iteration.

    state = (m_mu, v_mu, m_omega, v_omega), the Adam moments; t >= 1 the step
    number. Returns (mu, omega, state)."""
    gmu, gom = elbo_gradients(mu, omega, eta, gm, a, b)
    m_mu, v_mu, m_om, v_om = state
    mu, m_mu, v_mu = adam_ascent(mu, gmu, m_mu, v_mu, t, lr)
    omega, m_om, v_om = adam_ascent(omega, gom, m_om, v_om, t, lr)
    return mu, omega, (m_mu, v_mu, m_om, v_om)
