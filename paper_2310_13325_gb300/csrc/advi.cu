// Mean-field ADVI (Eq. 7-12 with a diagonal Cholesky factor L = diag(e^omega),
// the paper's mean-field option, Sec. 5) and Adam ascent of the ELBO.
//   sample:  theta_s = mu + e^omega eta_s,  m_s = T^{-1}(theta_s)
//            T^{-1}(theta) = a + (b - a) / (1 + e^{-theta})   (Eq. 12)
//   gradient per coordinate from S samples (Eq. 10-11 on the diagonal):
//            g_s = gm_s (b - a) s (1 - s) + (1 - 2 s),  s = sigmoid(theta_s)
//            grad_mu = mean_s g_s,  grad_omega = mean_s g_s eta_s e^omega + 1
//   Adam (beta1 0.9, beta2 0.999, eps 1e-8), ascent.
// With a == b == NULL the transform is the identity (g_s = gm_s).
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

__global__ void advi_step_kernel(float *mu, float *om, float *st, int t, const float *eta,
                                 const float *gm, float gscale, int S, int d, const float *a,
                                 const float *b, float lr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d) return;
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
  const float gm_mu = (float)(gmu / S);
  const float gm_om = (float)(gom / S * (double)si + 1.0);
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

}  // extern "C"
