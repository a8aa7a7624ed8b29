// Travel-time tomography (Sec. 4.1): station-to-station travel times by
// solving the first-order upwind eikonal discretisation, and the misfit
// gradient by tracing rays through the travel-time field (Sec. 3, Sec. 4.1).
//
// One CTA owns one (particle, source station) pair for the whole call. It
// stages the slowness map and an inf-padded travel-time field in shared
// memory and relaxes the upwind equations in red-black order until nothing
// changes (the fixed point is the same discrete solution fast marching
// reaches in heap order). The field is split by colour into two arrays
// ((i + j) even / odd, each row holding every other node), so a warp reading
// the neighbours of consecutive nodes of one colour reads consecutive words
// of the other array. Then each thread traces one ray from a receiver
// station back to the source and adds its weighted slowness kernel to a
// shared accumulator, which the CTA finally adds to the particle's gradient.
//
// Layout: V[P][ny][nx] km/s, x fastest; stations are node indices i*nx + j;
// data are ordered by (s, r), s < r, s-major.
#include "common.cuh"
#include <math_constants.h>

namespace {

constexpr int kTomoThreads = 256;
constexpr int kSlots = 3;                 // register-held nodes per thread and colour
constexpr float kRayStep = 0.5f;         // ray step, node spacings

struct TomoArgs {
  const float *V;
  const int *sta;
  const float *dobs, *sigma;
  float *Tout;        // [P][npairs] or null
  double *mpart;      // [P][nsrc] or null
  const int *slist;   // source stations of the launch (null: 0 .. ns-2)
  int nsrc;           // sources per particle in the launch
  float *grad;        // [P][ny*nx] or null
  int ny, nx, ns, npairs, P, maxit, maxsteps;
  float h;
  int *status;
};

__device__ __forceinline__ int pair_index(int s, int r, int ns) {
  return s * ns - s * (s + 1) / 2 + (r - s - 1);
}

// Upwind time of one node from its smaller neighbour times a, b along the
// two axes and f = h / v: the root t >= max of ((t-a)^+)^2 + ((t-b)^+)^2 = f^2.
// The two-sided root takes its square root as q * rsqrt(q) (q >= f^2 > 0 there;
// relative error a few 1e-7, far inside the travel-time tolerance).
__device__ __forceinline__ float upwind(float a, float b, float f) {
  const float lo = fminf(a, b), hi = fmaxf(a, b);
  if (!(lo < CUDART_INF_F)) return CUDART_INF_F;
  const float dd = hi - lo;
  if (dd >= f) return lo + f;
  const float q = 2.f * f * f - dd * dd;
  return 0.5f * (lo + hi + q * rsqrtf(q));
}

// Node k of colour c ((i + j) & 1 == c), k counted row-major within the colour.
__device__ __forceinline__ bool colour_node(int k, int c, int ny, int nx, int &i, int &j) {
  const int pr = k / nx, rem = k - pr * nx;    // two rows hold nx nodes of a colour
  const int n0 = (nx - c + 1) >> 1;            // colour-c nodes of the even row
  if (rem < n0) { i = 2 * pr;     j = c + 2 * rem; }
  else          { i = 2 * pr + 1; j = (1 - c) + 2 * (rem - n0); }
  return i < ny;
}

struct Bilin { int i0, j0; float fy, fx; };

__device__ __forceinline__ Bilin bilin(float y, float x, int ny, int nx) {
  Bilin b;
  b.i0 = min((int)y, ny - 2);                  // y, x >= 0: truncation is floor
  b.j0 = min((int)x, nx - 2);
  b.fy = y - (float)b.i0;
  b.fx = x - (float)b.j0;
  return b;
}

__device__ __forceinline__ float interp(const float *F, const Bilin &b, int nx) {
  const float *r0 = F + b.i0 * nx + b.j0, *r1 = r0 + nx;
  return (1.f - b.fy) * ((1.f - b.fx) * r0[0] + b.fx * r0[1]) +
         b.fy * ((1.f - b.fx) * r1[0] + b.fx * r1[1]);
}

// Adds w * (length of the segment p -> q) * bilinear weights of its midpoint.
__device__ __forceinline__ void add_segment(float *K, float py, float px, float qy, float qx,
                                            float w, int ny, int nx) {
  const float dy = qy - py, dx = qx - px;
  const float wl = w * sqrtf(dy * dy + dx * dx);
  const Bilin b = bilin(0.5f * (py + qy), 0.5f * (px + qx), ny, nx);
  float *r0 = K + b.i0 * nx + b.j0, *r1 = r0 + nx;
  atomicAdd(r0,     wl * (1.f - b.fy) * (1.f - b.fx));
  atomicAdd(r0 + 1, wl * (1.f - b.fy) * b.fx);
  atomicAdd(r1,     wl * b.fy * (1.f - b.fx));
  atomicAdd(r1 + 1, wl * b.fy * b.fx);
}

template <bool GRAD>
__global__ void __launch_bounds__(kTomoThreads, 6)
tomo_kernel(TomoArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ny = a.ny, nx = a.nx, n = ny * nx, ns = a.ns;
  const int ks = blockIdx.x % a.nsrc, p = blockIdx.x / a.nsrc;
  const int s = a.slist ? a.slist[ks] : ks;
  const int tid = threadIdx.x;
  const int Wc = (nx + 3) >> 1;                           // words per row and colour
  const int PS = (ny + 2) * Wc;
  double *red = (double *)smem_raw;                       // [32]
  float *C0 = (float *)(smem_raw + 32 * sizeof(double));  // [(ny+2)][Wc] colour 0
  float *C1 = C0 + PS;                                    // [(ny+2)][Wc] colour 1
  float *F = C1 + PS;                                     // [ny][nx] h / v
  float *GY = F + n, *GX = GY + n, *K = GX + n;           // GRAD only
  // travel time of node (i, j), -1 <= i <= ny, -1 <= j <= nx (the halo is inf)
  auto T = [&](int i, int j) -> float {
    const int I = i + 1, J = j + 1;
    return (((I + J) & 1) ? C1 : C0)[I * Wc + (J >> 1)];
  };

  const float *v = a.V + (size_t)p * n;
  bool bad = false;
  for (int k = tid; k < n; k += kTomoThreads) {
    const float vk = v[k];
    bad |= !(vk > 0.f && vk < CUDART_INF_F);
    F[k] = a.h / vk;
    if constexpr (GRAD) K[k] = 0.f;
  }
  for (int k = tid; k < 2 * PS; k += kTomoThreads) C0[k] = CUDART_INF_F;
  if (bad) atomicOr(a.status, 2);
  __syncthreads();
  const int src = a.sta[s];
  const int si = src / nx, sj = src - si * nx;
  if (tid == 0) {
    const int I = si + 1, J = sj + 1;
    (((I + J) & 1) ? C1 : C0)[I * Wc + (J >> 1)] = 0.f;
  }
  __syncthreads();

  // red-black relaxation of the upwind equations from T = inf (monotone:
  // every accepted change lowers a time, so the sweep ends at the fixed point)
  const int half = (n + 1) >> 1;                // colour-0 count bounds colour 1
  int it = 0;
  if (half <= kSlots * kTomoThreads) {
    // grids up to 2 kSlots x 256 nodes: each thread keeps the offsets of its
    // nodes in their colour array (times two, plus the column parity) and
    // their h / v in registers for the whole relaxation
    int off[2][kSlots];
    float fv[2][kSlots];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int m = 0; m < kSlots; ++m) {
        const int k = tid + m * kTomoThreads;
        int i, j;
        off[c][m] = -1;
        fv[c][m] = 0.f;
        if (k < half && colour_node(k, c, ny, nx, i, j)) {
          const int I = i + 1, J = j + 1;
          off[c][m] = ((I * Wc + (J >> 1)) << 1) | (J & 1);
          fv[c][m] = F[i * nx + j];
        }
      }
    for (; it < a.maxit; ++it) {
      int changed = 0;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        float *Tc = c ? C1 : C0;
        const float *Tn = c ? C0 : C1;
#pragma unroll
        for (int m = 0; m < kSlots; ++m) {
          if (off[c][m] < 0) continue;
          const int o = off[c][m] >> 1, pj = off[c][m] & 1;
          // left, right: the other colour's words o-1+pj, o+pj; up, down: o -/+ Wc
          const float *q = Tn + o;
          const float tn = upwind(fminf(q[pj - 1], q[pj]), fminf(q[-Wc], q[Wc]), fv[c][m]);
          if (tn < Tc[o]) { Tc[o] = tn; changed = 1; }
        }
        if (c == 0) __syncthreads();
      }
      if (!__syncthreads_or(changed)) break;
    }
  } else {
    for (; it < a.maxit; ++it) {
      int changed = 0;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        float *Tc = c ? C1 : C0;
        const float *Tn = c ? C0 : C1;
        for (int k = tid; k < half; k += kTomoThreads) {
          int i, j;
          if (!colour_node(k, c, ny, nx, i, j)) continue;
          const int I = i + 1, J = j + 1, o = I * Wc + (J >> 1), pj = J & 1;
          const float *q = Tn + o;
          const float tn = upwind(fminf(q[pj - 1], q[pj]), fminf(q[-Wc], q[Wc]), F[i * nx + j]);
          if (tn < Tc[o]) { Tc[o] = tn; changed = 1; }
        }
        if (c == 0) __syncthreads();
      }
      if (!__syncthreads_or(changed)) break;
    }
  }
  if (it == a.maxit && tid == 0) atomicOr(a.status, 1);

  const int nr = ns - 1 - s;                    // receivers r = s+1 .. ns-1
  const int pbase = pair_index(s, s + 1, ns);
  if (a.Tout) {
    for (int k = tid; k < nr; k += kTomoThreads) {
      const int r = a.sta[s + 1 + k];
      const int ri = r / nx, rj = r - ri * nx;
      a.Tout[(size_t)p * a.npairs + pbase + k] = T(ri, rj);
    }
  }
  if constexpr (GRAD) {
    // nodal gradients: central differences inside, one-sided on the edge
    for (int k = tid; k < n; k += kTomoThreads) {
      const int i = k / nx, j = k - i * nx;
      const float t0 = T(i, j);
      GX[k] = (j == 0) ? T(i, 1) - t0 : (j == nx - 1) ? t0 - T(i, j - 1)
                                       : 0.5f * (T(i, j + 1) - T(i, j - 1));
      GY[k] = (i == 0) ? T(1, j) - t0 : (i == ny - 1) ? t0 - T(i - 1, j)
                                       : 0.5f * (T(i + 1, j) - T(i - 1, j));
    }
    __syncthreads();

    double J = 0.0;
    for (int k = tid; k < nr; k += kTomoThreads) {
      const int r = a.sta[s + 1 + k];
      const int ri = r / nx, rj = r - ri * nx;
      const int pi = pbase + k;
      const float res = T(ri, rj) - a.dobs[pi];
      const float sg = a.sigma[pi];
      const float w = res / (sg * sg);
      J += 0.5 * (double)res * (double)res / ((double)sg * (double)sg);
      const float sy = (float)si, sx = (float)sj;
      float py = (float)ri, px = (float)rj;
      for (int st = 0; st < a.maxsteps; ++st) {
        const float dy = py - sy, dx = px - sx;
        if (dy * dy + dx * dx <= kRayStep * kRayStep) break;
        const Bilin b = bilin(py, px, ny, nx);
        const float gy = interp(GY, b, nx), gx = interp(GX, b, nx);
        const float g2 = gy * gy + gx * gx;
        if (g2 == 0.f) break;
        const float sc = kRayStep * rsqrtf(g2);       // step / |grad T|
        const float qy = fminf(fmaxf(py - sc * gy, 0.f), (float)(ny - 1));
        const float qx = fminf(fmaxf(px - sc * gx, 0.f), (float)(nx - 1));
        add_segment(K, py, px, qy, qx, w, ny, nx);
        py = qy;
        px = qx;
      }
      add_segment(K, py, px, sy, sx, w, ny, nx);
    }

    // CTA sum of the misfit terms, one FP64 partial per (particle, source)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) J += __shfl_xor_sync(0xffffffffu, J, o);
    if ((tid & 31) == 0) red[tid >> 5] = J;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int wi = 0; wi < kTomoThreads / 32; ++wi) t += red[wi];
      a.mpart[(size_t)p * a.nsrc + ks] = t;
    }
    // dJ/dv_k = -h K_k / v_k^2
    float *g = a.grad + (size_t)p * n;
    for (int k = tid; k < n; k += kTomoThreads) {
      const float kk = K[k];
      if (kk != 0.f) {
        const float vk = v[k];
        atomicAdd(g + k, -a.h * kk / (vk * vk));
      }
    }
  }
}

// misfit[p] = sum over sources of the partials, in source order
__global__ void tomo_misfit_kernel(const double *mpart, int P, int nsrc, double *misfit) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double t = 0.0;
  for (int s = 0; s < nsrc; ++s) t += mpart[(size_t)p * nsrc + s];
  misfit[p] = t;
}

size_t tomo_smem(int ny, int nx, bool grad) {
  const size_t n = (size_t)ny * nx;
  const size_t wc = (size_t)(nx + 3) / 2;
  return 32 * sizeof(double) + (2 * (size_t)(ny + 2) * wc + n * (grad ? 4 : 1)) * sizeof(float);
}

}  // namespace

struct tomo_ctx {
  int ny, nx, ns, npairs, maxit, maxsteps;
  float h;
  int *d_sta = nullptr;
  int *d_slist = nullptr;     // minibatch source list
  int *d_status = nullptr;
  double *d_mpart = nullptr;
  size_t mpart_cap = 0;
  cudaStream_t last_stream = nullptr;
};

extern "C" {

int tomo_create(int ny, int nx, double h, int n_stations, const int *stations,
                tomo_ctx **out) {
  if (!out) return VIP_ERR_ARG;
  *out = nullptr;
  if (ny < 2 || nx < 2 || !(h > 0.0) || n_stations < 2 || !stations) return VIP_ERR_ARG;
  if ((long long)ny * nx > (1 << 24)) return VIP_ERR_ARG;
  for (int k = 0; k < n_stations; ++k) {
    if (stations[k] < 0 || stations[k] >= ny * nx) return VIP_ERR_ARG;
    for (int m = 0; m < k; ++m)
      if (stations[m] == stations[k]) return VIP_ERR_ARG;
  }
  int dev = 0, optin = 0;
  VIP_TRY(cudaGetDevice(&dev));
  VIP_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (tomo_smem(ny, nx, true) > (size_t)optin) return VIP_ERR_UNSUPPORTED;
  VIP_TRY(cudaFuncSetAttribute(tomo_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tomo_smem(ny, nx, true)));
  VIP_TRY(cudaFuncSetAttribute(tomo_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tomo_smem(ny, nx, false)));
  tomo_ctx *c = new tomo_ctx;
  c->ny = ny;
  c->nx = nx;
  c->ns = n_stations;
  c->npairs = n_stations * (n_stations - 1) / 2;
  c->h = (float)h;
  c->maxit = ny * nx;                              // bounds the dependency depth
  c->maxsteps = (int)(4 * (ny + nx) / kRayStep);
  if (cudaMalloc(&c->d_sta, sizeof(int) * n_stations) != cudaSuccess ||
      cudaMalloc(&c->d_slist, sizeof(int) * n_stations) != cudaSuccess ||
      cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess ||
      cudaMemcpy(c->d_sta, stations, sizeof(int) * n_stations, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess) {
    cudaFree(c->d_sta);
    cudaFree(c->d_slist);
    cudaFree(c->d_status);
    delete c;
    return VIP_ERR_CUDA;
  }
  *out = c;
  return VIP_OK;
}

int tomo_destroy(tomo_ctx *c) {
  if (!c) return VIP_OK;
  cudaDeviceSynchronize();
  cudaFree(c->d_sta);
  cudaFree(c->d_slist);
  cudaFree(c->d_status);
  cudaFree(c->d_mpart);
  delete c;
  return VIP_OK;
}

int tomo_pair_count(const tomo_ctx *c) { return c ? c->npairs : VIP_ERR_ARG; }

static TomoArgs tomo_args(tomo_ctx *c, const float *V, int P) {
  TomoArgs a{};
  a.V = V;
  a.sta = c->d_sta;
  a.ny = c->ny;
  a.nx = c->nx;
  a.ns = c->ns;
  a.npairs = c->npairs;
  a.P = P;
  a.maxit = c->maxit;
  a.maxsteps = c->maxsteps;
  a.h = c->h;
  a.status = c->d_status;
  a.slist = nullptr;
  a.nsrc = c->ns - 1;
  return a;
}

int tomo_traveltimes(tomo_ctx *c, const float *V, int P, float *T, vip_stream_t stream) {
  if (!c || P < 0 || (P > 0 && (!V || !T))) return VIP_ERR_ARG;
  if ((long long)P * (c->ns - 1) > 0x7fffffffLL) return VIP_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  VIP_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int), st));
  if (P == 0) return VIP_OK;
  TomoArgs a = tomo_args(c, V, P);
  a.Tout = T;
  tomo_kernel<false><<<P * (c->ns - 1), kTomoThreads, tomo_smem(c->ny, c->nx, false), st>>>(a);
  VIP_CHECK_LAUNCH();
  return VIP_OK;
}

static int tomo_run_gradient(tomo_ctx *c, const float *V, int P, const float *dobs,
                             const float *sigma, const int *slist, int nsrc, double *misfit,
                             float *grad, float *T, cudaStream_t st) {
  const size_t need = (size_t)P * nsrc;
  if (need > c->mpart_cap) {
    VIP_TRY(cudaStreamSynchronize(st));
    cudaFree(c->d_mpart);
    c->d_mpart = nullptr;
    c->mpart_cap = 0;
    if (cudaMalloc(&c->d_mpart, need * sizeof(double)) != cudaSuccess) return VIP_ERR_NOMEM;
    c->mpart_cap = need;
  }
  VIP_TRY(cudaMemsetAsync(grad, 0, sizeof(float) * (size_t)P * c->ny * c->nx, st));
  TomoArgs a = tomo_args(c, V, P);
  a.dobs = dobs;
  a.sigma = sigma;
  a.Tout = T;
  a.mpart = c->d_mpart;
  a.grad = grad;
  a.slist = slist;
  a.nsrc = nsrc;
  tomo_kernel<true><<<P * nsrc, kTomoThreads, tomo_smem(c->ny, c->nx, true), st>>>(a);
  VIP_CHECK_LAUNCH();
  tomo_misfit_kernel<<<(P + 127) / 128, 128, 0, st>>>(c->d_mpart, P, nsrc, misfit);
  VIP_CHECK_LAUNCH();
  return VIP_OK;
}

int tomo_gradient(tomo_ctx *c, const float *V, int P, const float *dobs, const float *sigma,
                  double *misfit, float *grad, float *T, vip_stream_t stream) {
  if (!c || P < 0 || (P > 0 && (!V || !dobs || !sigma || !misfit || !grad))) return VIP_ERR_ARG;
  if ((long long)P * (c->ns - 1) > 0x7fffffffLL) return VIP_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  VIP_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int), st));
  if (P == 0) return VIP_OK;
  return tomo_run_gradient(c, V, P, dobs, sigma, nullptr, c->ns - 1, misfit, grad, T, st);
}

int tomo_gradient_sources(tomo_ctx *c, const float *V, int P, const float *dobs,
                          const float *sigma, const int *sources, int nb, double *misfit,
                          float *grad, vip_stream_t stream) {
  if (!c || P < 0 || (P > 0 && (!V || !dobs || !sigma || !misfit || !grad))) return VIP_ERR_ARG;
  if (!sources || nb < 1 || nb > c->ns - 1) return VIP_ERR_ARG;
  for (int k = 0; k < nb; ++k) {
    if (sources[k] < 0 || sources[k] >= c->ns - 1) return VIP_ERR_ARG;
    for (int m = 0; m < k; ++m)
      if (sources[m] == sources[k]) return VIP_ERR_ARG;
  }
  if ((long long)P * nb > 0x7fffffffLL) return VIP_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  VIP_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int), st));
  if (P == 0) return VIP_OK;
  // a copy from pageable host memory returns once the list has been staged,
  // and the launch that reads it follows in stream order
  VIP_TRY(cudaMemcpyAsync(c->d_slist, sources, sizeof(int) * nb, cudaMemcpyHostToDevice, st));
  return tomo_run_gradient(c, V, P, dobs, sigma, c->d_slist, nb, misfit, grad, nullptr, st);
}

int tomo_last_status(tomo_ctx *c) {
  if (!c) return VIP_ERR_ARG;
  if (cudaStreamSynchronize(c->last_stream) != cudaSuccess) return VIP_ERR_CUDA;
  int h = 0;
  if (cudaMemcpy(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return VIP_ERR_CUDA;
  if (h & 2) return VIP_ERR_ARG;
  if (h & 1) return VIP_ERR_TIMEOUT;
  return VIP_OK;
}

}  // extern "C"
