"""FP64 oracle: mean-field ADVI (Eq. 7-12) with Adam ascent (and the SGD,
ADAGRAD and ADADELTA rules the paper also lists).

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


# ---------------------------------------------------------------------------
# The other ascent rules of Sec. 5 (the paper lists SGD, ADAGRAD, ADADELTA and
# ADAM for the ELBO), written from their published definitions (Duchi et al.
# 2011, diagonal form; Zeiler 2012), each increasing the objective:
#   SGD       p <- p + lr g
#   ADAGRAD   G <- G + g^2;  p <- p + lr g / (sqrt(G) + eps)            eps 1e-8
#   ADADELTA  E[g^2] <- rho E[g^2] + (1 - rho) g^2
#             dx = sqrt(E[dx^2] + eps) / sqrt(E[g^2] + eps) g
#             E[dx^2] <- rho E[dx^2] + (1 - rho) dx^2;  p <- p + lr dx  rho 0.95, eps 1e-6
#                                                                     (lr = 1 is Zeiler's rule)
#   ADAM      adam_ascent above
# Each keeps two state arrays per variable (s1, s2): unused (SGD), (G, -)
# (ADAGRAD), (E[g^2], E[dx^2]) (ADADELTA), (m, v) (ADAM).

SGD, ADAGRAD, ADADELTA, ADAM = 0, 1, 2, 3
ADAGRAD_EPS = 1e-8
ADADELTA_RHO, ADADELTA_EPS = 0.95, 1e-6


def sgd_ascent(p, grad, lr):
    return p + lr * grad


def adagrad_ascent(p, grad, acc, lr):
    acc = acc + grad * grad
    return p + lr * grad / (np.sqrt(acc) + ADAGRAD_EPS), acc


def adadelta_ascent(p, grad, eg2, edx2, lr):
    eg2 = ADADELTA_RHO * eg2 + (1.0 - ADADELTA_RHO) * grad * grad
    dx = np.sqrt(edx2 + ADADELTA_EPS) / np.sqrt(eg2 + ADADELTA_EPS) * grad
    edx2 = ADADELTA_RHO * edx2 + (1.0 - ADADELTA_RHO) * dx * dx
    return p + lr * dx, eg2, edx2


def ascend(p, grad, s1, s2, t, lr, opt):
    """One step of the chosen rule; returns (p, s1, s2)."""
    if opt == SGD:
        return sgd_ascent(p, grad, lr), s1, s2
    if opt == ADAGRAD:
        p, s1 = adagrad_ascent(p, grad, s1, lr)
        return p, s1, s2
    if opt == ADADELTA:
        return adadelta_ascent(p, grad, s1, s2, lr)
    if opt == ADAM:
        return adam_ascent(p, grad, s1, s2, t, lr)
    raise ValueError("unknown optimizer %r" % (opt,))


def advi_step_opt(mu, omega, state, t, eta, gm, lr, opt, a=None, b=None):
    """advi_step with the ascent rule opt (SGD, ADAGRAD, ADADELTA, ADAM);
    state = (s1_mu, s2_mu, s1_omega, s2_omega)."""
    gmu, gom = elbo_gradients(mu, omega, eta, gm, a, b)
    s1m, s2m, s1o, s2o = state
    mu, s1m, s2m = ascend(mu, gmu, s1m, s2m, t, lr, opt)
    omega, s1o, s2o = ascend(omega, gom, s1o, s2o, t, lr, opt)
    return mu, omega, (s1m, s2m, s1o, s2o)


# ---------------------------------------------------------------------------
# Full-rank ADVI restricted to a low-rank-plus-diagonal covariance (Eq. 7-11;
# the full d x d factor L is out of reach at d = 36,000-144,000):
#   theta = mu + e^omega * eta + B eps,   eta ~ N(0, I_d), eps ~ N(0, I_r),
#   Sigma = diag(e^{2 omega}) + B B^T   (B [d, r]).
# With g_s the per-sample gradient of log p(T^{-1}(theta)) + log|det J| as in
# the mean-field case, the ELBO = E[...] + 1/2 log|Sigma| + const has
#   grad_mu    = mean_s g_s
#   grad_omega = mean_s g_s eta_s e^omega + diag(Sigma^{-1}) e^{2 omega}
#   grad_B     = mean_s g_s eps_s^T + Sigma^{-1} B
# (d/domega_i of 1/2 log|Sigma| = 1/2 tr(Sigma^{-1} dSigma/domega_i) and
# d/dB of 1/2 log|Sigma| = Sigma^{-1} B). Here Sigma^{-1} is formed and
# inverted densely: plain and slow, for small d only.

def sample_lowrank(mu, omega, B, eta, eps, a=None, b=None):
    """m_s = T^{-1}(mu + e^omega eta_s + B eps_s); eta [S, d], eps [S, r]."""
    theta = mu[None, :] + np.exp(omega)[None, :] * eta + eps @ B.T
    if a is None:
        return theta
    return T_inv(theta, a[None, :], b[None, :])


def elbo_gradients_lowrank(mu, omega, B, eta, eps, gm, a=None, b=None):
    """Monte-Carlo (grad_mu, grad_omega, grad_B)."""
    theta = mu[None, :] + np.exp(omega)[None, :] * eta + eps @ B.T
    if a is None:
        g = np.asarray(gm, dtype=np.float64)
    else:
        s = 1.0 / (1.0 + np.exp(-theta))
        g = gm * (b - a)[None, :] * s * (1.0 - s) + (1.0 - 2.0 * s)
    S = g.shape[0]
    Sigma = np.diag(np.exp(2.0 * omega)) + B @ B.T
    Sinv = np.linalg.inv(Sigma)
    grad_mu = g.mean(axis=0)
    grad_omega = (g * eta * np.exp(omega)[None, :]).mean(axis=0) + np.diag(Sinv) * np.exp(2.0 * omega)
    grad_B = g.T @ eps / S + Sinv @ B
    return grad_mu, grad_omega, grad_B


def advi_lowrank_step(mu, omega, B, state, t, eta, eps, gm, lr, a=None, b=None):
    """One low-rank-plus-diagonal ADVI iteration with Adam on mu, omega, B.
    state = (m_mu, v_mu, m_omega, v_omega, m_B, v_B)."""
    gmu, gom, gB = elbo_gradients_lowrank(mu, omega, B, eta, eps, gm, a, b)
    m_mu, v_mu, m_om, v_om, m_B, v_B = state
    mu, m_mu, v_mu = adam_ascent(mu, gmu, m_mu, v_mu, t, lr)
    omega, m_om, v_om = adam_ascent(omega, gom, m_om, v_om, t, lr)
    B, m_B, v_B = adam_ascent(B, gB, m_B, v_B, t, lr)
    return mu, omega, B, (m_mu, v_mu, m_om, v_om, m_B, v_B)
