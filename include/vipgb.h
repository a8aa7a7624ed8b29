/*
 * vipgb.h - C ABI of libvipgb: the data-parallel hot path of variational
 * Bayesian full-waveform inversion (Zhang & Curtis, "VIP - Variational
 * Inversion Package", arXiv 2310.13325) on one NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every entry point
 *  - All array arguments are DEVICE pointers unless marked "host".
 *  - The caller owns every buffer it passes; the library never frees them.
 *    An fwi_ctx owns only its scratch memory, CUDA graphs and tuning cache.
 *  - Arrays are row-major with the last index fastest. A velocity model
 *    v[nz][nx] has x (horizontal) fastest; particle sets are X[n][d] with
 *    d = nz * nx.
 *  - Calls are asynchronous and ordered on the given stream (NULL = legacy
 *    default stream) unless stated otherwise. A return of VIP_OK means the
 *    work was enqueued; a negative return is an error code and nothing was
 *    enqueued unless stated otherwise. vip_strerror() names each code.
 *  - Units: velocity m/s, grid spacing m, time s.
 */
#ifndef VIPGB_H
#define VIPGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *vip_stream_t; /* same type as cudaStream_t */

/* ---- status codes ---------------------------------------------------- */
#define VIP_OK            0
#define VIP_ERR_ARG      -1  /* invalid argument (shape, pointer, range)     */
#define VIP_ERR_CFL      -2  /* max(v) dt / dx above the 8th-order limit     */
#define VIP_ERR_NOMEM    -3  /* workspace too small / device allocation fail */
#define VIP_ERR_CUDA     -4  /* a CUDA runtime call failed                  */
#define VIP_ERR_TIMEOUT  -5  /* a bounded device-side wait gave up          */
#define VIP_ERR_NOTPD    -6  /* kernel matrix not positive definite          */
#define VIP_ERR_UNSUPPORTED -7 /* no feasible launch plan on this device      */
#define VIP_ERR_NONFINITE -8 /* a NaN or infinity among the inputs          */

const char *vip_strerror(int code);

/* Text of the first CUDA runtime failure recorded on the calling host
 * thread since the last vip_clear_error() ("" if none). Diagnostics only. */
const char *vip_last_error(void);
void vip_clear_error(void);

/* ======================================================================
 * Full-waveform inversion forward / adjoint (paper Sec. 3 and Sec. 4.2)
 *
 * The paper simulates data with "a time-domain finite difference method"
 * and a 10 Hz Ricker wavelet and obtains velocity gradients "using the
 * adjoint method" (Sec. 4.2); the scheme is fixed here as
 *   a^{n+1} = g [2 a^n + w (L a^n + s^n)] - g^2 a^{n-1},  w = vpad^2 dt^2,
 * L the 8th-order 5-arm Laplacian with zero values outside the padded grid,
 * vpad the model edge-replicated into an nsponge-cell sponge on all sides,
 * g the Cerjan taper exp(-(alpha*i)^2) exp(-(alpha*j)^2) (i, j = cells into
 * the sponge), s^n = f(n dt)/dx^2 at the source node with the Ricker
 * f(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2), and the trace
 * sample d[r][n] = a^{n+1} at receiver r (n = 0 .. nt-1).
 * The misfit is the negative log of the Gaussian likelihood (Eq. 26),
 *   J = 1/2 sum_{s,r,n} ((d - d_obs) / sigma)^2,
 * and gradients are those of the exact discrete adjoint of the recurrence,
 * folded from the padded grid onto the physical cells.
 *
 * Batches: fwi_forward, fwi_gradient, fwi_gradient_sources and fwi_adjoint
 * take P >= 0 models. P = 0 is an empty batch (a rank or minibatch that holds
 * no particles): the other arguments are still checked, the P-sized pointers
 * may be NULL, and the call returns VIP_OK without any device work. P < 0 is
 * VIP_ERR_ARG.
 * ====================================================================== */

typedef struct {
    int   nz, nx;          /* physical grid                                  */
    float dx;              /* grid spacing (m), square cells                 */
    float dt;              /* time step (s)                                  */
    int   nt;              /* number of time steps = samples per trace       */
    int   nsponge;         /* sponge width in cells (20)                     */
    float sponge_alpha;    /* Cerjan decay constant (0.015)                  */
    float f0;              /* Ricker peak frequency (Hz)                     */
    float t0;              /* Ricker delay (s); <= 0 selects 1/f0            */
    int   nsrc;            /* number of sources S                            */
    const int *src_iz;     /* host [S] physical row of each source           */
    const int *src_ix;     /* host [S] physical column of each source        */
    int   nrec;            /* number of receivers R                          */
    const int *rec_iz;     /* host [R] physical row of each receiver         */
    const int *rec_ix;     /* host [R] physical column of each receiver      */
} fwi_geom;

/* An fwi_ctx is not thread-safe: calls on one context (its scratch memory,
 * graphs, tuning cache and, during fwi_gradient_sources, its source tables)
 * must come from one host thread at a time; separate contexts are
 * independent. */
typedef struct fwi_ctx fwi_ctx;

/* Precision of the stored forward wavefield snapshots that the imaging
 * condition reads back during the adjoint sweep. The stencil itself always
 * runs in FP32; restart checkpoints (checkpoint interval > 1) are FP32. */
#define FWI_FP32       0
#define FWI_CKPT_BF16  1
#define FWI_CKPT_FP16  2   /* FP16 with a power-of-two scale per row of 4 cells */

/* Execution modes. BATCHED: every (particle, source) pair of a call runs in
 * one persistent thread-block-cluster launch that keeps the wavefields in
 * shared memory for all time steps (replayed from a CUDA graph; setting the
 * environment variable VIPGB_GRAPHS=0 before fwi_create launches the same
 * kernels directly instead, e.g. under profilers).
 * PLAIN: one (particle, source) pair at a time, one kernel launch per time
 * step, wavefields in global memory, no graph - the comparison baseline. */
#define FWI_MODE_BATCHED 0
#define FWI_MODE_PLAIN   1

/* Create a context for one acquisition geometry. Copies *geom (and the host
 * index arrays). workspace_limit_bytes caps the device scratch the context
 * may allocate (0 = 85% of free device memory at each call).
 * Errors: VIP_ERR_ARG (bad sizes, indices outside the physical grid,
 * duplicate receiver cells), VIP_ERR_CUDA. Synchronous. */
int  fwi_create(const fwi_geom *geom, size_t workspace_limit_bytes,
                fwi_ctx **out);
void fwi_destroy(fwi_ctx *ctx);

/* Select the execution mode (FWI_MODE_*) and the restart-checkpoint interval
 * K (1 = store every snapshot, no recomputation; K > 1 = store the state
 * every K steps and recompute each K-step segment during the adjoint sweep;
 * 0 = choose automatically from the workspace limit). */
int  fwi_set_mode(fwi_ctx *ctx, int mode, int ckpt_every);

/* Autotuning of the batched launch (cluster size, rows per thread, threads
 * per block). When enabled, the first batched call with a new (P, mode,
 * precision, number of sources) times short runs (48 steps, one wave of clusters) of the
 * candidate launches on the caller's own inputs, synchronously, and caches
 * the fastest in the context; later calls reuse it. Without tuning a cost
 * model picks the launch. fwi_autotune(ctx, P, precision) enables tuning. */
int  fwi_autotune(fwi_ctx *ctx, int P, int precision);

/* Force the batched launch shape: Q CTAs per cluster (1..16, 0 = any), V
 * rows per thread (0 = any), T threads per CTA (multiple of 32,
 * 0 = any), the number of sources one cluster processes per work item
 * (0 = any) and where the model coefficients w' and the gradient
 * accumulator live: coeff 1 = shared memory next to the wavefield, 2 =
 * global memory (only the two time levels stay in shared memory, so taller
 * bands and smaller clusters fit large grids), 0 = any. V is one of 4, 5, 8,
 * 10 (10 only with coeff 1). All zeros restore automatic choice. A shape that
 * does not fit the device makes later calls return VIP_ERR_UNSUPPORTED.
 * Traces and misfits do not depend on the shape; gradients do not depend on
 * Q, V, T or coeff (every cell update and accumulation is evaluated
 * identically) and are deterministic for any split of the sources. */
int  fwi_set_plan(fwi_ctx *ctx, int Q, int V, int T, int sources_per_item, int coeff);
int  fwi_set_autotune(fwi_ctx *ctx, int enable);

/* Fill launch. Clusters of the batched launch's shape cannot be placed on
 * every SM (on the GB300, 36 clusters of 4 CTAs take 144 of the 152 SMs).
 * With filling enabled (the default) and an automatically chosen plan with
 * more work items than clusters, a second launch of smaller clusters (the
 * global-coefficient layout, whose taller band fits shared memory) runs on
 * the SMs left idle, at a lower priority, and both launches draw the work
 * items from one counter. Results do not depend on which launch computed an
 * item (every cell update, accumulation and per-receiver misfit sum is
 * evaluated identically). fwi_set_fill(ctx, 0) disables it; forced plans
 * (fwi_set_plan) never fill. fwi_query_fill writes 4 ints to fill_out
 * (host): {cluster_ctas, rows_per_thread, threads, clusters} of the fill
 * launch a gradient call for P particles would add, or zeros. */
int  fwi_set_fill(fwi_ctx *ctx, int enable);
int  fwi_query_fill(fwi_ctx *ctx, int P, int precision, int *fill_out);

/* Describe the plan chosen for P particles: writes 10 ints to plan_out
 * (host): {cluster_ctas, rows_per_thread, threads, band_rows, concurrent
 * pairs, ckpt_every, work_items, sources_per_item, coeff (1 shared, 2
 * global memory), shared-memory bytes per CTA}, and the device bytes the
 * context holds after planning to bytes_out (host, may be NULL). When no
 * plan fits the workspace limit it returns VIP_ERR_NOMEM and writes to
 * bytes_out the smallest scratch any plan tried would need (the limit a
 * caller would have to grant at the current checkpoint setting). */
int  fwi_query_plan(fwi_ctx *ctx, int P, int precision, int *plan_out,
                    size_t *bytes_out);

/* Device scratch bytes the last planned call on this context needed, or, if
 * that call returned VIP_ERR_NOMEM, the smallest footprint it tried and
 * could not fit under the workspace limit (host, synchronous, no device
 * call). 0 before the first call. */
size_t fwi_bytes_needed(fwi_ctx *ctx);

/* Seismograms for P models.
 *   v    [P][nz][nx] velocities (m/s)
 *   seis [P][S][R][nt] output traces
 * Errors: VIP_ERR_ARG, VIP_ERR_NOMEM, VIP_ERR_CUDA. The stability bound is
 * checked on the device and reported by fwi_last_status(). */
int  fwi_forward(fwi_ctx *ctx, const float *v, int P, float *seis,
                 vip_stream_t stream);

/* Misfit and its velocity gradient for P models (the data-parallel hot path).
 *   v      [P][nz][nx] velocities
 *   dobs   [S][R][nt] observed traces
 *   sigma  scalar data standard deviation (Eq. 26 with sigma_i = sigma)
 *   misfit [P] output, J per model, accumulated in FP64
 *   grad   [P][nz][nx] output dJ/dv (J >= 0; grad log p = -grad inside the
 *          uniform prior's bounds)
 *   precision FWI_FP32 | FWI_CKPT_BF16 | FWI_CKPT_FP16 */
int  fwi_gradient(fwi_ctx *ctx, const float *v, int P, const float *dobs,
                  double sigma, double *misfit, float *grad, int precision,
                  vip_stream_t stream);

/* fwi_gradient over a minibatch of the sources (the stochastic gradients of
 * sSVGD from uniformly drawn data subsets, Sec. 3 after Eq. 22): misfit and
 * gradient are the sums over the nb sources listed in sources (host array of
 * distinct indices in [0, S)), so (S / nb) times them is an unbiased estimate
 * of the full-data values (pass that factor as gscale to ssvgd_step). The
 * listed sources' traces are gathered from dobs [S][R][nt] into context
 * memory in stream order before the launch. Batched mode only
 * (VIP_ERR_UNSUPPORTED in plain mode); other errors as fwi_gradient. */
int  fwi_gradient_sources(fwi_ctx *ctx, const float *v, int P, const float *dobs,
                          double sigma, const int *sources, int nb, double *misfit,
                          float *grad, int precision, vip_stream_t stream);

/* Backward of the seismogram map (the autograd rule of fwi_forward):
 *   dseis [P][S][R][nt] upstream sensitivity dL/dseis
 *   grad  [P][nz][nx]   output dL/dv */
int  fwi_adjoint(fwi_ctx *ctx, const float *v, int P, const float *dseis,
                 float *grad, int precision, vip_stream_t stream);

/* Device-side status of the last call on this context (synchronises the
 * stream it last used): VIP_OK; VIP_ERR_NONFINITE if some velocity was NaN
 * or infinite, or a misfit came out non-finite (e.g. NaN observed data);
 * otherwise VIP_ERR_CFL if some model violated max(v) dt/dx <= 0.5547 (the
 * 2-D stability bound of the 8th-order leapfrog scheme). After either error
 * the outputs of that call are undefined. */
int  fwi_last_status(fwi_ctx *ctx);

/* ======================================================================
 * SVGD, Eq. (13)-(17):
 *   phi(m_i) = 1/n sum_j [k(m_j, m_i) G_j + k(m_j, m_i) (m_i - m_j) / h^2],
 *   m_i <- clip(m_i + eps phi(m_i), lo, hi)
 * with the RBF kernel of Eq. (16), k = exp(-|m - m'|^2 / (2 h^2)). The paper
 * leaves h free ("a scale factor"); h2 <= 0 selects the median rule
 *   h^2 = med / (2 ln(n + 1)),
 * med the median of all n^2 squared distances (zero diagonal included, mean
 * of the two middle values for even n^2; h^2 = 1 if med < 1e-30). The bound
 * reset is the paper's first uniform-prior strategy (Sec. 3).
 *   X   [n][d] particles, updated in place
 *   G   [n][d] gradient at each particle; grad log p = gscale * G (pass
 *       gscale = 1 for log-posterior gradients, -1 for the misfit gradients
 *       dJ/dv of fwi_gradient: inside a uniform prior's box grad log p = -dJ/dv)
 *   lo, hi [d] per-coordinate bounds, or NULL for none
 *   gram_precision: how |m_i - m_j|^2 is formed (VIP_GRAM_*)
 *   ws, ws_bytes: caller scratch of at least svgd_workspace_size() bytes,
 *           256-byte aligned
 *   h2_used [1] device double, the bandwidth used (may be NULL)
 * ====================================================================== */
#define VIP_GRAM_BF16    0  /* one BF16 tensor-core Gram, FP32 accumulate  */
#define VIP_GRAM_BF16X3  1  /* three-piece BF16 split, six tensor-core products:
                               FP32-class accuracy (dropped terms < 2^-24) */
#define VIP_GRAM_FP32    2  /* SIMT FP32 Gram without tensor cores (reference) */

size_t svgd_workspace_size(int n, int d, int gram_precision, int stochastic);

/* Device-side status of the last svgd_step / ssvgd_step / svgd_step_q /
 * ssvgd_step_q / svgd_sqdist that used the workspace ws (its first 16 bytes
 * hold the status words; synchronises stream):
 *   VIP_OK
 *   VIP_ERR_TIMEOUT    a bounded wait inside a tensor-core kernel expired
 *                      (the Gram: h2_used is NaN and so are the particles;
 *                      the update: every particle is set to NaN)
 *   VIP_ERR_NONFINITE  X or G held a NaN or infinity. With the tensor-core
 *                      update (VIP_GRAM_BF16, VIP_GRAM_BF16X3) the particles
 *                      are left unchanged; with the FP32 reference update
 *                      they are undefined.
 * Errors of its own: VIP_ERR_ARG (ws NULL or not 256-byte aligned),
 * VIP_ERR_CUDA. */
int  svgd_status(const void *ws, vip_stream_t stream);

/* Rows a9-a10 of one step on their own: the centred Gram on the tensor cores
 * (or SIMT), the squared distances D2 [n][n] (device, FP64, zero diagonal,
 * clamped at 0) and the median bandwidth h2_used [1] (device double, as in
 * svgd_step with h2 <= 0). ws as for svgd_step (stochastic = 0). */
int  svgd_sqdist(const float *X, int n, int d, int gram_precision, double *D2,
                 double *h2_used, void *ws, size_t ws_bytes, vip_stream_t stream);

int  svgd_step(float *X, const float *G, float gscale, int n, int d, float eps,
               float h2, const float *lo, const float *hi, int gram_precision,
               void *ws, size_t ws_bytes, double *h2_used,
               vip_stream_t stream);

/* svgd_step without a workspace argument and without any device memory
 * allocation, for callers that cannot allocate GPU memory themselves: for
 * example a plug-in that a host application calls with device pointers but
 * no allocator, a process whose device memory is entirely owned by another
 * framework's memory pool, or a latency-critical loop that must not call
 * cudaMalloc/cudaFree (which can synchronise the device). The paper has no
 * counterpart; this is a deployment variant of svgd_step.
 *
 * Scratch comes from one fixed array of VIP_NOALLOC_SCRATCH_BYTES (64 MiB)
 * in device memory, reserved on every GPU that loads the library until the
 * process exits. Problems whose svgd_workspace_size(n, d, gram_precision, 0)
 * exceeds that size are rejected with VIP_ERR_NOMEM before any device call
 * (with VIP_GRAM_BF16X3: n = 8 particles up to d = 53,376, n = 64 up to
 * d = 45,248, n = 600 up to d = 5,119).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture. All calls share the array and it keeps the
 * previous call's contents: every call rewrites what it reads, so no state
 * leaks between calls, but calls that overlap on the GPU (different
 * streams, or host threads, without ordering between them) race on the
 * scratch and give wrong results. Arguments and results are those of
 * svgd_step. */
#define VIP_NOALLOC_SCRATCH_BYTES (64u << 20)
int  svgd_step_noalloc(float *X, const float *G, float gscale, int n, int d,
                       float eps, float h2, const float *lo, const float *hi,
                       int gram_precision, double *h2_used,
                       vip_stream_t stream);

/* Stochastic SVGD, Eq. (22) with the noise of Eq. (25):
 *   m_i <- clip(m_i + eps phi(m_i) + sqrt(2 eps / n) sum_j Lk_ij xi_j, lo, hi),
 * Lk the lower Cholesky factor of Kbar + tau I (Kbar_ij = k(m_i, m_j),
 * tau = 1e-6 n, multiplied by 10 on failure, at most 3 retries; the factor
 * is FP32). xi [n][d] is either the caller's standard-normal array or, when
 * xi == NULL, drawn on the device from Philox-4x32-10 keyed by (seed, iter)
 * (counter = (column/4, row, iter)). tau_used [1] device double (may be
 * NULL). Synchronises the stream once to read the factorisation status.
 * Errors: as svgd_step, VIP_ERR_NOTPD if every retry failed. */
int  ssvgd_step(float *X, const float *G, float gscale, int n, int d, float eps,
                float h2, const float *lo, const float *hi, int gram_precision,
                void *ws, size_t ws_bytes, double *h2_used,
                uint64_t seed, uint64_t iter, const float *xi,
                double *tau_used, vip_stream_t stream);

/* SVGD and sSVGD with the diagonal matrix-valued kernel (Discussion
 * section; Wang et al. 2019): K_Q(m', m) = Q^{-1} k_Q(m', m), Q = diag(q),
 * k_Q(m', m) = exp(-(m' - m)^T Q (m' - m) / (2 h^2)), h^2 by the median rule
 * on the Q-weighted squared distances. The direction is
 *   phi(m_i) = 1/n sum_j k_Q(m_j, m_i) [G_j / q + (m_i - m_j) / h^2]
 * and the sSVGD noise sqrt(2 eps / n) (Lk Xi) Q^{-1/2}. q: device [d],
 * positive (typically 1 / the variance of each coordinate across the
 * particles, svgd_inverse_variance). All other arguments, the workspace
 * size and the errors are those of svgd_step / ssvgd_step; q = NULL is
 * VIP_ERR_ARG. With q = 1 the results equal svgd_step / ssvgd_step bit for
 * bit. */
int  svgd_step_q(float *X, const float *G, float gscale, const float *q, int n,
                 int d, float eps, float h2, const float *lo, const float *hi,
                 int gram_precision, void *ws, size_t ws_bytes, double *h2_used,
                 vip_stream_t stream);
int  ssvgd_step_q(float *X, const float *G, float gscale, const float *q, int n,
                  int d, float eps, float h2, const float *lo, const float *hi,
                  int gram_precision, void *ws, size_t ws_bytes,
                  double *h2_used, uint64_t seed, uint64_t iter,
                  const float *xi, double *tau_used, vip_stream_t stream);

/* q_c = 1 / Var_j(X[j][c]) for the particles X [n][d] (device, FP32 in,
 * two-pass population variance, FP64-class: compensated FP32 sums per
 * thread, FP64 across threads), 1 where the variance is zero; the
 * choice of Q the Discussion section gives. q: device [d], caller-owned. */
int  svgd_inverse_variance(const float *X, int n, int d, float *q,
                           vip_stream_t stream);

/* ======================================================================
 * Mean-field ADVI (Eq. 7-12 with a diagonal Cholesky factor, Sec. 5):
 * theta = mu + e^omega * eta, m = T^{-1}(theta) with the logit transform of
 * Eq. (12) when a, b are given (identity when a == b == NULL).
 * ====================================================================== */

/* m_out[s][i] = T^{-1}(mu_i + e^{omega_i} eta[s][i]) for S samples. */
int  advi_sample(const float *mu, const float *omega, const float *eta,
                 int S, int d, const float *a, const float *b, float *m_out,
                 vip_stream_t stream);

/* One ELBO ascent step (Eq. 10-11 on the diagonal) with Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8):
 *   g_s = gm[s] dm/dtheta + d log|det J|/dtheta,
 *   grad_mu = mean_s g_s, grad_omega = mean_s g_s eta_s e^omega + 1.
 *   adam_state [4][d]: first and second moments of mu, then of omega,
 *              zero before the first step; t >= 1 the step number.
 *   gm [S][d] gradient at m_s = advi_sample(...), with d log p / dm =
 *      gscale * gm (1 for log-density gradients, -1 for misfit gradients). */
int  advi_step(float *mu, float *omega, float *adam_state, int t,
               const float *eta, const float *gm, float gscale, int S, int d,
               const float *a, const float *b, float lr,
               vip_stream_t stream);

/* advi_step with a choice of ascent rule among those the paper lists for the
 * ELBO (Sec. 5): VIP_ASCENT_SGD (p += lr g), VIP_ASCENT_ADAGRAD (Duchi et al.
 * 2011, diagonal: G += g^2, p += lr g / (sqrt(G) + 1e-8)), VIP_ASCENT_ADADELTA
 * (Zeiler 2012, rho 0.95, eps 1e-6; lr multiplies the step, 1 is Zeiler's
 * rule) and VIP_ASCENT_ADAM (exactly advi_step). state: device [4][d],
 * zero before the first step: two values per variable, (s1_mu, s2_mu,
 * s1_omega, s2_omega); unused by SGD. Errors: VIP_ERR_ARG for an unknown
 * rule, otherwise as advi_step. */
#define VIP_ASCENT_SGD      0
#define VIP_ASCENT_ADAGRAD  1
#define VIP_ASCENT_ADADELTA 2
#define VIP_ASCENT_ADAM     3
int  advi_step_opt(float *mu, float *omega, float *state, int t,
                   const float *eta, const float *gm, float gscale, int S, int d,
                   const float *a, const float *b, float lr, int rule,
                   vip_stream_t stream);

/* Full-rank ADVI (Eq. 7-11) with the covariance restricted to low rank plus
 * diagonal, Sigma = diag(e^{2 omega}) + B B^T, because the full d x d factor
 * L is out of reach at d = 36,000-144,000:
 *   theta_s = mu + e^omega eta_s + B eps_s,  m_s = T^{-1}(theta_s)  (Eq. 12)
 *   grad_mu    = mean_s g_s
 *   grad_omega = mean_s g_s eta_s e^omega + diag(Sigma^{-1}) e^{2 omega}
 *   grad_B     = mean_s g_s eps_s^T + Sigma^{-1} B
 * with g_s as in advi_step and Sigma^{-1} applied through the r x r matrix
 * M = I + B^T diag(e^{-2 omega}) B (Woodbury); Adam ascent on mu, omega, B.
 *   B      [d][r] (row-major, r <= VIP_ADVI_MAX_RANK)
 *   eta    [S][d], eps [S][r] standard normal draws
 *   state  [4 d + 2 d r] zero before the first step: Adam moments of mu,
 *          omega (as advi_step) then of B ([d][r] each)
 *   work   [2 r r] FP64 scratch (M and its inverse), caller-owned
 * advi_lowrank_sample writes m_out [S][d]. With B = 0 the step equals
 * advi_step up to rounding. Errors: VIP_ERR_ARG (sizes, r, S r too large for
 * shared memory). */
#define VIP_ADVI_MAX_RANK 32
int  advi_lowrank_sample(const float *mu, const float *omega, const float *B, int r,
                         const float *eta, const float *eps, int S, int d,
                         const float *a, const float *b, float *m_out,
                         vip_stream_t stream);
int  advi_lowrank_step(float *mu, float *omega, float *B, int r, float *state,
                       double *work, int t, const float *eta, const float *eps,
                       const float *gm, float gscale, int S, int d, const float *a,
                       const float *b, float lr, vip_stream_t stream);

/* SVGD / sSVGD in the unconstrained space (Sec. 3, second strategy for the
 * uniform prior): particles theta = T(m) with the transform of Eq. (12),
 * T(m) = log(m - a) - log(b - m), T^{-1}(theta) = a + (b - a) / (1 + e^-theta),
 * updated by svgd_step / ssvgd_step (without bounds) with the gradient of
 * the transformed density,
 *   g_theta = gscale gm (b - a) s (1 - s) + (1 - 2 s),  s = sigmoid(theta),
 * gm = grad_m of the log-likelihood (or log posterior) at m = T^{-1}(theta).
 * All arrays device [n][d] (a, b: [d]); elementwise, in place allowed for
 * the transforms. Errors: VIP_ERR_ARG for NULL pointers or n, d < 1. */
int  vip_to_unconstrained(const float *m, const float *a, const float *b, int n,
                          int d, float *theta, vip_stream_t stream);
int  vip_to_model(const float *theta, const float *a, const float *b, int n,
                  int d, float *m, vip_stream_t stream);
int  vip_unconstrained_gradient(const float *theta, const float *gm, float gscale,
                                const float *a, const float *b, int n, int d,
                                float *g, vip_stream_t stream);

/* Standard normals out[rows][cols] from the Philox-4x32-10 stream used by
 * ssvgd_step (same counter layout), for the ADVI draws eta. */
int  vip_philox_normal(float *out, int rows, int cols, uint64_t seed,
                       uint64_t iter, vip_stream_t stream);

/* ======================================================================
 * Travel-time tomography (Sec. 4.1): group travel times between stations
 * from the first-order upwind discretisation of the eikonal equation
 * |grad T| = 1/v (the system fast marching solves, Rawlinson & Sambridge
 * 2004), and the gradient of the Gaussian misfit (Eq. 26, one sigma per
 * travel time) from rays traced through the travel-time field (Sec. 3).
 *
 * Units of this block: velocity km/s, spacing km, time s. Velocity lives on
 * the nodes of a regular ny x nx grid, V[P][ny][nx] with x fastest; stations
 * are node indices i * nx + j. Station s < ns - 1 is the source of the pairs
 * (s, r), r > s; data arrays hold the ns (ns - 1) / 2 pairs s-major, pair
 * (s, r) at s * ns - s (s + 1) / 2 + r - s - 1.
 *
 * Rays start at the receiver node and step half a node spacing against the
 * bilinearly interpolated nodal travel-time gradient (central differences
 * inside the grid, one-sided on its edge), clipped to the grid, until they
 * are within half a spacing of the source (or after 8 (ny + nx) steps), then
 * join it with a straight segment. Each segment adds its length times the
 * bilinear weights of its midpoint to the ray's slowness kernel.
 * ====================================================================== */
typedef struct tomo_ctx tomo_ctx;

/* stations: host array of n_stations distinct node indices (copied).
 * Errors: VIP_ERR_ARG (ny, nx < 2, h <= 0, fewer than 2 stations, an index
 * outside the grid or repeated), VIP_ERR_UNSUPPORTED (the grid does not fit
 * one CTA's shared memory: 2 (ny + 2) floor((nx + 3) / 2) + 4 ny nx floats),
 * VIP_ERR_CUDA.
 * Synchronous. The context is used by one host thread at a time. */
int  tomo_create(int ny, int nx, double h, int n_stations, const int *stations,
                 tomo_ctx **out);
int  tomo_destroy(tomo_ctx *ctx);
int  tomo_pair_count(const tomo_ctx *ctx);

/* Predicted travel times T[P][npairs] for P velocity maps V[P][ny][nx].
 * Errors: VIP_ERR_ARG (NULL with P > 0, P < 0), VIP_ERR_CUDA. */
int  tomo_traveltimes(tomo_ctx *ctx, const float *V, int P, float *T,
                      vip_stream_t stream);

/* Misfit J[p] = sum_i (T_i - dobs_i)^2 / (2 sigma_i^2) (FP64, summed over
 * sources in order) and grad[P][ny][nx] = dJ/dv from the rays, for P maps.
 *   dobs, sigma [npairs]; T [P][npairs] optional output (NULL to skip).
 * grad is overwritten (zeroed on the stream first, then accumulated with
 * atomics, so its last bits may vary between runs). Scratch of P (ns - 1)
 * doubles is owned by the context and grown on demand (the growth
 * synchronises the stream), so calls on different streams must not overlap. Errors: VIP_ERR_ARG, VIP_ERR_NOMEM,
 * VIP_ERR_CUDA. */
int  tomo_gradient(tomo_ctx *ctx, const float *V, int P, const float *dobs,
                   const float *sigma, double *misfit, float *grad, float *T,
                   vip_stream_t stream);

/* tomo_gradient over a minibatch of the source stations (the stochastic
 * gradients of sSVGD from uniformly drawn data subsets, Sec. 3 after Eq. 22):
 * misfit and gradient sum the pairs (s, r > s) of the nb distinct source
 * stations listed in sources (host array, values in [0, ns - 2], copied in
 * stream order), so ((ns - 1) / nb) times them estimates the full-data values
 * without bias. The list is staged in context memory, so two such calls on
 * different streams must not overlap. Errors: as tomo_gradient, VIP_ERR_ARG
 * for a bad list. */
int  tomo_gradient_sources(tomo_ctx *ctx, const float *V, int P, const float *dobs,
                           const float *sigma, const int *sources, int nb,
                           double *misfit, float *grad, vip_stream_t stream);

/* Device status of the last call (synchronises its stream): VIP_OK,
 * VIP_ERR_ARG if some velocity was not positive and finite, VIP_ERR_TIMEOUT
 * if a travel-time field did not settle within ny * nx relaxation sweeps;
 * the outputs of that call are then undefined. */
int  tomo_last_status(tomo_ctx *ctx);

/* ======================================================================
 * Test hook (no counterpart in the paper)
 *
 * Every wait on an mbarrier inside the tensor-core kernels (the Gram and the
 * update of svgd_step / ssvgd_step) is bounded: when the bound expires the
 * kernel records the failure in its status word, waits (bounded) for the
 * copies it has issued, frees its tensor memory and returns, so the CUDA
 * context stays usable and svgd_status() reports VIP_ERR_TIMEOUT.
 * vip_test_set_wait sets, for the launches that follow in this process, the
 * bound in SM clock cycles (0 restores the default of 2e9, about one second)
 * and, with stall_producer = 1, stops the copy producer of those kernels
 * from issuing anything, so that the consumer's wait expires by design
 * (tests of the error path; nothing faults). Not thread-safe; reset with
 * vip_test_set_wait(0, 0). Errors: VIP_ERR_ARG (negative cycles,
 * stall_producer not 0 or 1). Host only, synchronous. */
int  vip_test_set_wait(long long cycles, int stall_producer);

#ifdef __cplusplus
}
#endif
#endif /* VIPGB_H */
