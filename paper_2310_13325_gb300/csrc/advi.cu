// Mean-field ADVI (Eq. 7-12 with a diagonal Cholesky factor L = diag(e^omega),
// the paper's mean-field option, Sec. 5) and Adam ascent of the ELBO.
//   sample:  theta_s = mu + e^omega eta_s,  m_s = T^{-1}(theta_s)
//            T^{-1}(theta) = a + (b - a) / (1 + e^{-theta})   (Eq. 12)
//   gradient per coordinate from S samples (Eq. 10-11 on the diagonal):
//            g_s = gm_s (b - a) s (1 - s) + (1 - 2 s),  s = sigmoid(theta_s)
//            grad_mu = mean_s g_s,  grad_omega = mean_s g_s eta_s e^omega + 1
//   Adam (beta1 0.9, beta2 0.999, eps 1e-8), ascent; advi_step_opt also
//   offers the other rules the paper lists (Sec. 5): SGD, ADAGRAD (Duchi et
//   al. 2011, eps 1e-8) and ADADELTA (Zeiler 2012, rho 0.95, eps 1e-6).
// With a == b == NULL the transform is the identity (g_s = gm_s).
//
// The same transform serves SVGD / sSVGD in the unconstrained space (Sec. 3,
// second strategy for the uniform prior): to_unconstrained, to_model and the
// gradient of the transformed density, grad_m log p (b - a) s (1 - s) +
// (1 - 2 s), elementwise over [n][d].
#include "common.cuh"

namespace vip {

__global__ void advi_sample_kernel(const float *mu, const float *om, const float *eta, int S,
                                   int d, const float *a, const float *b, float *m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d) return;
  const float mi = mu[i], si = expf(om[i]);
  const float ai = a ? a[i] : 0.f, wi = a ? b[i] - a[i] : 0.f;
  for (int s = 0; s < S; ++s) {
    const float th = fmaf(si, eta[(size_t)s * d + i], mi);
    m[(size_t)s * d + i] = a ? fmaf(wi, 1.f / (1.f + expf(-th)), ai) : th;
  }
}

// Monte-Carlo ELBO gradients of coordinate i (Eq. 10-11 on the diagonal).
__device__ __forceinline__ void advi_grads(const float *mu, const float *om, const float *eta,
                                           const float *gm, float gscale, int S, int d,
                                           const float *a, const float *b, int i,
                                           float &gm_mu, float &gm_om) {
  const float mi = mu[i], si = expf(om[i]);
  const float wi = a ? b[i] - a[i] : 0.f;
  double gmu = 0.0, gom = 0.0;
  for (int s = 0; s < S; ++s) {
    const float e = eta[(size_t)s * d + i];
    float g = gscale * gm[(size_t)s * d + i];
    if (a) {
      const float th = fmaf(si, e, mi);
      const float sg = 1.f / (1.f + expf(-th));
      g = fmaf(g * wi, sg * (1.f - sg), 1.f - 2.f * sg);
    }
    gmu += (double)g;
    gom += (double)g * (double)e;
  }
  gm_mu = (float)(gmu / S);
  gm_om = (float)(gom / S * (double)si + 1.0);
}

__global__ void advi_step_kernel(float *mu, float *om, float *st, int t, const float *eta,
                                 const float *gm, float gscale, int S, int d, const float *a,
                                 const float *b, float lr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d) return;
  const float mi = mu[i];
  float gm_mu, gm_om;
  advi_grads(mu, om, eta, gm, gscale, S, d, a, b, i, gm_mu, gm_om);
  const float b1 = 0.9f, b2 = 0.999f, ae = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  float *m_mu = st, *v_mu = st + d, *m_om = st + 2 * (size_t)d, *v_om = st + 3 * (size_t)d;
  float m1 = fmaf(b1, m_mu[i], (1.f - b1) * gm_mu);
  float m2 = fmaf(b2, v_mu[i], (1.f - b2) * gm_mu * gm_mu);
  m_mu[i] = m1; v_mu[i] = m2;
  mu[i] = mi + lr * (m1 / c1) / (sqrtf(m2 / c2) + ae);
  m1 = fmaf(b1, m_om[i], (1.f - b1) * gm_om);
  m2 = fmaf(b2, v_om[i], (1.f - b2) * gm_om * gm_om);
  m_om[i] = m1; v_om[i] = m2;
  om[i] = om[i] + lr * (m1 / c1) / (sqrtf(m2 / c2) + ae);
}

enum AscentRule { AR_SGD = 0, AR_ADAGRAD = 1, AR_ADADELTA = 2, AR_ADAM = 3 };

// One ascent step of p with gradient g; s1, s2 the rule's two state values.
template <int RULE>
__device__ __forceinline__ float ascend(float p, float g, float &s1, float &s2, float c1,
                                        float c2, float lr) {
  if (RULE == AR_SGD) return fmaf(lr, g, p);
  if (RULE == AR_ADAGRAD) {
    s1 = fmaf(g, g, s1);
    return p + lr * g / (sqrtf(s1) + 1e-8f);
  }
  if (RULE == AR_ADADELTA) {
    const float rho = 0.95f, e = 1e-6f;
    s1 = fmaf(rho, s1, (1.f - rho) * g * g);
    const float dx = sqrtf(s2 + e) / sqrtf(s1 + e) * g;
    s2 = fmaf(rho, s2, (1.f - rho) * dx * dx);
    return fmaf(lr, dx, p);
  }
  // Adam, as advi_step_kernel
  const float b1 = 0.9f, b2 = 0.999f, ae = 1e-8f;
  s1 = fmaf(b1, s1, (1.f - b1) * g);
  s2 = fmaf(b2, s2, (1.f - b2) * g * g);
  return p + lr * (s1 / c1) / (sqrtf(s2 / c2) + ae);
}

template <int RULE>
__global__ void advi_step_opt_kernel(float *mu, float *om, float *st, int t, const float *eta,
                                     const float *gm, float gscale, int S, int d, const float *a,
                                     const float *b, float lr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d) return;
  float gm_mu, gm_om;
  advi_grads(mu, om, eta, gm, gscale, S, d, a, b, i, gm_mu, gm_om);
  const float c1 = 1.f - powf(0.9f, (float)t), c2 = 1.f - powf(0.999f, (float)t);
  float *s1m = st, *s2m = st + d, *s1o = st + 2 * (size_t)d, *s2o = st + 3 * (size_t)d;
  float x = s1m[i], y = s2m[i];
  mu[i] = ascend<RULE>(mu[i], gm_mu, x, y, c1, c2, lr);
  s1m[i] = x; s2m[i] = y;
  x = s1o[i]; y = s2o[i];
  om[i] = ascend<RULE>(om[i], gm_om, x, y, c1, c2, lr);
  s1o[i] = x; s2o[i] = y;
}

// Eq. (12) elementwise over [n][d]; a, b per column.
__global__ void to_unconstrained_kernel(const float *m, const float *a, const float *b, size_t nd,
                                        int d, float *theta) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nd) return;
  const int c = (int)(k % d);
  theta[k] = logf(m[k] - a[c]) - logf(b[c] - m[k]);
}

__global__ void to_model_kernel(const float *theta, const float *a, const float *b, size_t nd,
                                int d, float *m) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nd) return;
  const int c = (int)(k % d);
  m[k] = fmaf(b[c] - a[c], 1.f / (1.f + expf(-theta[k])), a[c]);
}

__global__ void unconstrained_gradient_kernel(const float *theta, const float *gm, float gscale,
                                              const float *a, const float *b, size_t nd, int d,
                                              float *g) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nd) return;
  const int c = (int)(k % d);
  const float sg = 1.f / (1.f + expf(-theta[k]));
  g[k] = fmaf(gscale * gm[k] * (b[c] - a[c]), sg * (1.f - sg), 1.f - 2.f * sg);
}

}  // namespace vip

using namespace vip;

extern "C" {

int advi_sample(const float *mu, const float *omega, const float *eta, int S, int d,
                const float *a, const float *b, float *m_out, vip_stream_t stream) {
  if (!mu || !omega || !eta || !m_out || S < 1 || d < 1 || (!a) != (!b)) return VIP_ERR_ARG;
  advi_sample_kernel<<<idiv_up(d, 256), 256, 0, stream>>>(mu, omega, eta, S, d, a, b, m_out);
  VIP_CHECK_LAUNCH();
  return VIP_OK;
}

int advi_step(float *mu, float *omega, float *adam_state, int t, const float *eta,
              const float *gm, float gscale, int S, int d, const float *a, const float *b,
              float lr, vip_stream_t stream) {
  if (!mu || !omega || !adam_state || !eta || !gm || S < 1 || d < 1 || t < 1 ||
      (!a) != (!b))
    return VIP_ERR_ARG;
  advi_step_kernel<<<idiv_up(d, 256), 256, 0, stream>>>(mu, omega, adam_state, t, eta, gm, gscale,
                                                        S, d, a, b, lr);
  VIP_CHECK_LAUNCH();
  return VIP_OK;
}

int advi_step_opt(float *mu, float *omega, float *state, int t, const float *eta,
                  const float *gm, float gscale, int S, int d, const float *a, const float *b,
                  float lr, int rule, vip_stream_t stream) {
  if (!mu || !omega || !state || !eta || !gm || S < 1 || d < 1 || t < 1 || (!a) != (!b) ||
      rule < VIP_ASCENT_SGD || rule > VIP_ASCENT_ADAM)
    return VIP_ERR_ARG;
  const dim3 g(idiv_up(d, 256)), blk(256);
  switch (rule) {
    case VIP_ASCENT_SGD:
      advi_step_opt_kernel<AR_SGD><<<g, blk, 0, stream>>>(mu, omega, state, t, eta, gm, gscale, S,
                                                          d, a, b, lr);
      break;
    case VIP_ASCENT_ADAGRAD:
      advi_step_opt_kernel<AR_ADAGRAD><<<g, blk, 0, stream>>>(mu, omega, state, t, eta, gm,
                                                              gscale, S, d, a, b, lr);
      break;
    case VIP_ASCENT_ADADELTA:
      advi_step_opt_kernel<AR_ADADELTA><<<g, blk, 0, stream>>>(mu, omega, state, t, eta, gm,
                                                               gscale, S, d, a, b, lr);
      break;
    default:
      advi_step_opt_kernel<AR_ADAM><<<g, blk, 0, stream>>>(mu, omega, state, t, eta, gm, gscale,
                                                           S, d, a, b, lr);
  }
  VIP_CHECK_LAUNCH();
  return VIP_OK;
}

int vip_to_unconstrained(const float *m, const float *a, const float *b, int n, int d,
                         float *theta, vip_stream_t stream) {
  if (!m || !a || !b || !theta || n < 1 || d < 1) return VIP_ERR_ARG;
  const size_t nd = (size_t)n * d;
  to_unconstrained_kernel<<<(unsigned)((nd + 255) / 256), 256, 0, stream>>>(m, a, b, nd, d, theta);
  VIP_CHECK_LAUNCH();
  return VIP_OK;
}

int vip_to_model(const float *theta, const float *a, const float *b, int n, int d, float *m,
                 vip_stream_t stream) {
  if (!m || !a || !b || !theta || n < 1 || d < 1) return VIP_ERR_ARG;
  const size_t nd = (size_t)n * d;
  to_model_kernel<<<(unsigned)((nd + 255) / 256), 256, 0, stream>>>(theta, a, b, nd, d, m);
  VIP_CHECK_LAUNCH();
  return VIP_OK;
}

int vip_unconstrained_gradient(const float *theta, const float *gm, float gscale, const float *a,
                               const float *b, int n, int d, float *g, vip_stream_t stream) {
  if (!theta || !gm || !a || !b || !g || n < 1 || d < 1) return VIP_ERR_ARG;
  const size_t nd = (size_t)n * d;
  unconstrained_gradient_kernel<<<(unsigned)((nd + 255) / 256), 256, 0, stream>>>(
      theta, gm, gscale, a, b, nd, d, g);
  VIP_CHECK_LAUNCH();
  return VIP_OK;
}

}  // extern "C"
