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

// ---------------------------------------------------------------------------
// Low-rank-plus-diagonal ADVI: theta = mu + e^omega eta + B eps, Sigma =
// D + B B^T with D = diag(e^{2 omega}), B [d][r] row-major, eps [S][r].
// The entropy terms need Sigma^{-1} only through M = I + B^T D^{-1} B (r x r):
//   Sigma^{-1} B = D^{-1} B M^{-1}                       (Woodbury)
//   diag(Sigma^{-1})_i = (1 - B_i M^{-1} B_i^T / D_i) / D_i
// so grad_omega_i = mean_s g eta e^omega + 1 - B_i M^{-1} B_i^T / D_i and
// grad_B_i = mean_s g eps^T + B_i M^{-1} / D_i.

__global__ void lowrank_sample_kernel(const float *mu, const float *om, const float *B, int r,
                                      const float *eta, const float *eps, int S, int d,
                                      const float *a, const float *b, float *m) {
  extern __shared__ float es[];   // eps [S][r]
  for (int q = threadIdx.x; q < S * r; q += blockDim.x) es[q] = eps[q];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d) return;
  float Bi[VIP_ADVI_MAX_RANK];
  for (int k = 0; k < r; ++k) Bi[k] = B[(size_t)i * r + k];
  const float mi = mu[i], si = expf(om[i]);
  const float ai = a ? a[i] : 0.f, wi = a ? b[i] - a[i] : 0.f;
  for (int s = 0; s < S; ++s) {
    float th = fmaf(si, eta[(size_t)s * d + i], mi);
    for (int k = 0; k < r; ++k) th = fmaf(Bi[k], es[s * r + k], th);
    m[(size_t)s * d + i] = a ? fmaf(wi, 1.f / (1.f + expf(-th)), ai) : th;
  }
}

// M_kl = delta_kl + sum_i B_ik B_il e^{-2 omega_i}: one block per (k, l <= k)
// pair, FP64, fixed reduction order.
__global__ void lowrank_m_kernel(const float *om, const float *B, int r, int d, double *M) {
  __shared__ double red[32];
  int p = blockIdx.x, k = 0;
  while (p > k) { p -= k + 1; ++k; }
  const int l = p;
  double acc = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x)
    acc += (double)B[(size_t)i * r + k] * (double)B[(size_t)i * r + l] * exp(-2.0 * (double)om[i]);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    if (k == l) t += 1.0;
    M[k * r + l] = t;
    M[l * r + k] = t;
  }
}

// Minv = M^{-1} for the symmetric positive definite r x r M (one thread:
// Cholesky M = L L^T, then columns of L^{-T} L^{-1}).
__global__ void lowrank_minv_kernel(const double *M, int r, double *Minv) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double L[VIP_ADVI_MAX_RANK * VIP_ADVI_MAX_RANK];
  for (int q = 0; q < r * r; ++q) L[q] = 0.0;
  for (int j = 0; j < r; ++j) {
    double s = M[j * r + j];
    for (int k = 0; k < j; ++k) s -= L[j * r + k] * L[j * r + k];
    const double ljj = sqrt(s > 0.0 ? s : 1e-300);
    L[j * r + j] = ljj;
    for (int i = j + 1; i < r; ++i) {
      double t = M[i * r + j];
      for (int k = 0; k < j; ++k) t -= L[i * r + k] * L[j * r + k];
      L[i * r + j] = t / ljj;
    }
  }
  double y[VIP_ADVI_MAX_RANK];
  for (int c = 0; c < r; ++c) {
    for (int i = 0; i < r; ++i) {           // L y = e_c
      double t = i == c ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) t -= L[i * r + k] * y[k];
      y[i] = t / L[i * r + i];
    }
    for (int i = r - 1; i >= 0; --i) {      // L^T x = y
      double t = y[i];
      for (int k = i + 1; k < r; ++k) t -= L[k * r + i] * Minv[k * r + c];
      Minv[i * r + c] = t / L[i * r + i];
    }
  }
}

__global__ void lowrank_step_kernel(float *mu, float *om, float *B, int r, float *st,
                                    const double *Minv, int t, const float *eta,
                                    const float *eps, const float *gm, float gscale, int S,
                                    int d, const float *a, const float *b, float lr) {
  extern __shared__ float smem_lr[];
  float *es = smem_lr;                                       // eps [S][r]
  double *Mi = reinterpret_cast<double *>(smem_lr + ((S * r + 1) & ~1));   // [r][r]
  for (int q = threadIdx.x; q < S * r; q += blockDim.x) es[q] = eps[q];
  for (int q = threadIdx.x; q < r * r; q += blockDim.x) Mi[q] = Minv[q];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d) return;
  float Bi[VIP_ADVI_MAX_RANK];
  double gB[VIP_ADVI_MAX_RANK];
  for (int k = 0; k < r; ++k) { Bi[k] = B[(size_t)i * r + k]; gB[k] = 0.0; }
  const float mi = mu[i], si = expf(om[i]);
  const float wi = a ? b[i] - a[i] : 0.f;
  double gmu = 0.0, gom = 0.0;
  for (int s = 0; s < S; ++s) {
    const float e = eta[(size_t)s * d + i];
    float th = fmaf(si, e, mi);
    for (int k = 0; k < r; ++k) th = fmaf(Bi[k], es[s * r + k], th);
    float g = gscale * gm[(size_t)s * d + i];
    if (a) {
      const float sg = 1.f / (1.f + expf(-th));
      g = fmaf(g * wi, sg * (1.f - sg), 1.f - 2.f * sg);
    }
    gmu += (double)g;
    gom += (double)g * (double)e;
    for (int k = 0; k < r; ++k) gB[k] += (double)g * (double)es[s * r + k];
  }
  // entropy terms through M^{-1}
  const double Di = exp(2.0 * (double)om[i]);
  double q = 0.0;
  double BM[VIP_ADVI_MAX_RANK];
  for (int k = 0; k < r; ++k) {
    double t2 = 0.0;
    for (int l = 0; l < r; ++l) t2 += (double)Bi[l] * Mi[l * r + k];
    BM[k] = t2;
    q += t2 * (double)Bi[k];
  }
  const float g_mu = (float)(gmu / S);
  const float g_om = (float)(gom / S * (double)si + 1.0 - q / Di);
  const float b1 = 0.9f, b2 = 0.999f, ae = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  float *m_mu = st, *v_mu = st + d, *m_om = st + 2 * (size_t)d, *v_om = st + 3 * (size_t)d;
  float *m_B = st + 4 * (size_t)d, *v_B = m_B + (size_t)d * r;
  float m1 = fmaf(b1, m_mu[i], (1.f - b1) * g_mu);
  float m2 = fmaf(b2, v_mu[i], (1.f - b2) * g_mu * g_mu);
  m_mu[i] = m1; v_mu[i] = m2;
  mu[i] = mi + lr * (m1 / c1) / (sqrtf(m2 / c2) + ae);
  m1 = fmaf(b1, m_om[i], (1.f - b1) * g_om);
  m2 = fmaf(b2, v_om[i], (1.f - b2) * g_om * g_om);
  m_om[i] = m1; v_om[i] = m2;
  om[i] = om[i] + lr * (m1 / c1) / (sqrtf(m2 / c2) + ae);
  for (int k = 0; k < r; ++k) {
    const size_t o = (size_t)i * r + k;
    const float g_b = (float)(gB[k] / S + BM[k] / Di);
    m1 = fmaf(b1, m_B[o], (1.f - b1) * g_b);
    m2 = fmaf(b2, v_B[o], (1.f - b2) * g_b * g_b);
    m_B[o] = m1; v_B[o] = m2;
    B[o] = Bi[k] + lr * (m1 / c1) / (sqrtf(m2 / c2) + ae);
  }
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

int advi_lowrank_sample(const float *mu, const float *omega, const float *B, int r,
                        const float *eta, const float *eps, int S, int d, const float *a,
                        const float *b, float *m_out, vip_stream_t stream) {
  if (!mu || !omega || !B || !eta || !eps || !m_out || S < 1 || d < 1 || r < 1 ||
      r > VIP_ADVI_MAX_RANK || (!a) != (!b) || (size_t)S * r * 4 > 48 * 1024)
    return VIP_ERR_ARG;
  lowrank_sample_kernel<<<idiv_up(d, 128), 128, (size_t)S * r * 4, stream>>>(
      mu, omega, B, r, eta, eps, S, d, a, b, m_out);
  VIP_CHECK_LAUNCH();
  return VIP_OK;
}

int advi_lowrank_step(float *mu, float *omega, float *B, int r, float *state, double *work,
                      int t, const float *eta, const float *eps, const float *gm,
                      float gscale, int S, int d, const float *a, const float *b, float lr,
                      vip_stream_t stream) {
  const size_t smem = (size_t)((S * r + 1) & ~1) * 4 + (size_t)r * r * 8;
  if (!mu || !omega || !B || !state || !work || !eta || !eps || !gm || S < 1 || d < 1 ||
      r < 1 || r > VIP_ADVI_MAX_RANK || t < 1 || (!a) != (!b) || smem > 48 * 1024)
    return VIP_ERR_ARG;
  double *M = work, *Minv = work + (size_t)r * r;
  lowrank_m_kernel<<<r * (r + 1) / 2, 256, 0, stream>>>(omega, B, r, d, M);
  VIP_CHECK_LAUNCH();
  lowrank_minv_kernel<<<1, 32, 0, stream>>>(M, r, Minv);
  VIP_CHECK_LAUNCH();
  lowrank_step_kernel<<<idiv_up(d, 128), 128, smem, stream>>>(
      mu, omega, B, r, state, Minv, t, eta, eps, gm, gscale, S, d, a, b, lr);
  VIP_CHECK_LAUNCH();
  return VIP_OK;
}

}  // extern "C"
