// SVGD (Eq. 13-17) and stochastic SVGD (Eq. 21-25) particle updates.
//
// Pipeline of one step on X [n][d], G [n][d] (all kernels below):
//   1. centre      mean over particles (FP64-class: compensated FP32 sums
//                  per thread, FP64 across threads), Xc = X - mean (FP32) and
//                  its BF16 image (one piece, or the three-piece split
//                  xc ~ h + m + l for FP32-class accuracy)
//   2. norms       |xc_i|^2, FP64-class the same way
//   3. gram        partial Xc Xc^T over K-splits (tcgen05 BF16 tensor cores,
//                  or a SIMT FP32 reference path)
//   4. finish      D2_ij = |xc_i|^2 + |xc_j|^2 - 2 Gram_ij in FP64, clamped at
//                  0, zero diagonal; upper triangle collected as sort keys
//   5. median      radix selection of the middle element(s) of all n^2
//                  entries -> h^2 = med / (2 ln(n+1))
//   6. kernel      Kbar_ij = exp(-D2_ij / (2 h^2)), row sums r_i
//   7. (sSVGD)     Lk = chol(Kbar + tau I) (blocked, FP32), noise draws
//   8. update      one fused GEMM pass over column tiles:
//                  phi_i = [ (Kbar G)_i + (r_i xc_i - (Kbar Xc)_i) / h^2 ] / n,
//                  x_i <- clip(x_i + eps phi_i + sqrt(2 eps/n) (Lk Xi)_i, lo, hi)
// The repulsive term uses the identity sum_j k_ij (m_i - m_j) =
// r_i xc_i - (Kbar Xc)_i, exact in real arithmetic because the particle
// mean cancels; centring keeps it well conditioned in FP32.
//
// FP64 runs at a small fraction of the FP32 rate on this GPU (conversions
// between float and double included), so no step does FP64 arithmetic per
// element of X: per-element sums use error-free FP32 transformations (the
// compensated summation and dot product of Ogita, Rump and Oishi, 2005), and
// FP64 only combines the per-thread partial sums and forms the per-pair
// distances of step 4.
//
// Diagonal matrix-valued kernel K_Q = Q^{-1} k_Q, Q = diag(q) (Discussion
// section): step 1 stores the centred particles scaled by sqrt(q), so steps
// 2-6 see the Q-metric; the update divides the driving term K G by q and the
// repulsive term and the sSVGD noise by sqrt(q), column by column (the
// repulsion is formed from the scaled Xc, whose factor sqrt(q) it removes).
#include "common.cuh"
#include "gram.cuh"
#include "philox.cuh"

#include <math_constants.h>
#include <cmath>
#include <mutex>

namespace vip {

struct SvgdWs {
  double *mean;
  float *qf;   // [2][dp] matrix-valued kernel: 1/q_c and 1/sqrt(q_c) per column (FP32)
  float *Xc;
  __nv_bfloat16 *Xh, *Xm, *Xl;   // BF16 pieces: x ~ h + m + l
  double *nrm;
  unsigned int *done;       // blocks of a radix-pass histogram that have finished
  float *parts;
  double *D2;
  unsigned long long *keys;
  unsigned int *hist;       // [2][256]
  unsigned long long *sel;  // prefix[2], mask, k[2], zero[2] (as u64)
  double *h2;
  int *flag;
  float *K, *rs;
  float *Lk, *Xi;
  float *L11;               // [32][32] the current Cholesky panel's diagonal factor
  // tensor-core update: A = [Kbar | Lk] and B = [Y | Z]^T as BF16 pieces
  __nv_bfloat16 *Ua[3], *Ub[3];
  float *rcoef;
  int np, dp, splits, M;
  int unp, udp, uKp;
  bool tcu;
};

// Splits of the coordinate axis for the Gram: as many CTAs as fit one wave
// (two Gram CTAs per SM on the 152 SMs: 97 KB of shared memory and 128 TMEM
// columns each), never more, so no CTA waits for a second wave.
static int gram_splits(int n, int d, int gp) {
  const int np = (n + 127) / 128 * 128;
  const int t = np / 128;
  const int tiles = gp == VIP_GRAM_FP32 ? ((n + 63) / 64) * ((n + 63) / 64 + 1) / 2
                                        : t * (t + 1) / 2;
  int s = 304 / tiles;
  const int kmax = std::max(1, d / 1024);
  return std::max(1, std::min(s, kmax));
}

static size_t layout(int n, int d, int gp, int stochastic, bool tcu, void *base, size_t cap,
                     SvgdWs &w) {
  Carve cv(base, cap);
  // status words first (offset 0): [0] Cholesky failure, [1] Gram wait
  // expired, [2] update wait expired, [3] non-finite input (bit 0 X, bit 1 G)
  w.flag = cv.take<int>(4);
  w.np = (n + 127) / 128 * 128;
  w.dp = (d + 63) / 64 * 64;
  w.splits = gram_splits(n, d, gp);
  w.M = n * (n - 1) / 2;
  w.mean = cv.take<double>(d);
  w.qf = cv.take<float>((size_t)2 * w.dp);
  w.Xc = cv.take<float>((size_t)n * d);
  const bool tc = gp != VIP_GRAM_FP32;
  w.Xh = cv.take<__nv_bfloat16>(tc ? (size_t)w.np * w.dp : 0);
  w.Xm = cv.take<__nv_bfloat16>(tc && gp == VIP_GRAM_BF16X3 ? (size_t)w.np * w.dp : 0);
  w.Xl = cv.take<__nv_bfloat16>(tc && gp == VIP_GRAM_BF16X3 ? (size_t)w.np * w.dp : 0);
  w.nrm = cv.take<double>(n);
  w.done = cv.take<unsigned int>(1);
  w.parts = cv.take<float>((size_t)w.splits * w.np * w.np);
  w.D2 = cv.take<double>((size_t)n * n);
  w.keys = cv.take<unsigned long long>(std::max(w.M, 1));
  w.hist = cv.take<unsigned int>(512);
  w.sel = cv.take<unsigned long long>(8);
  w.h2 = cv.take<double>(2);
  w.K = cv.take<float>((size_t)n * n);
  w.rs = cv.take<float>(n);
  w.Lk = cv.take<float>(stochastic ? (size_t)n * n : 0);
  w.L11 = cv.take<float>(stochastic ? 32 * 32 : 0);
  w.Xi = cv.take<float>(stochastic ? (size_t)n * d : 0);
  w.tcu = tcu;
  w.unp = (n + 127) / 128 * 128;
  w.udp = (d + 127) / 128 * 128;
  w.uKp = ((stochastic ? 2 * n : n) + 63) / 64 * 64;
  for (int k = 0; k < 3; ++k) {
    w.Ua[k] = cv.take<__nv_bfloat16>(tcu ? (size_t)w.unp * w.uKp : 0);
    w.Ub[k] = cv.take<__nv_bfloat16>(tcu ? (size_t)w.udp * w.uKp : 0);
  }
  w.rcoef = cv.take<float>(tcu ? n : 0);
  return cv.off;
}

// ---------------------------------------------------------------------------
// Error-free transformations in FP32: s + e == a + b exactly (Knuth's
// TwoSum) and p + e == a * b exactly (the product's rounding error from one
// FMA). Every operation is rounded explicitly, so none is contracted.
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
  return s;
}

// Compensated running sum (s, c): s the FP32 sum, c the accumulated rounding
// errors; s + c carries about twice the FP32 precision (Sum2 / Dot2 of
// Ogita, Rump and Oishi): the error of (double)s + (double)c is at most
// gamma_m^2 times the sum of magnitudes for m terms, gamma_m ~ m 2^-24.
struct Comp {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float e;
    s = two_sum(s, x, e);
    c = __fadd_rn(c, e);
  }
  __device__ __forceinline__ void add_sq(float x) {
    const float p = __fmul_rn(x, x);
    const float pe = __fmaf_rn(x, x, -p);
    float e;
    s = two_sum(s, p, e);
    c = __fadd_rn(c, __fadd_rn(e, pe));
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Column means and the centred particles. A block owns 32 columns: its 8
// warps sum interleaved sets of rows of them (each warp reads whole 128-byte
// row segments) with compensated FP32 sums, the 8 partial sums of a column
// are added in FP64 in a fixed order (so the mean does not depend on timing),
// and then the warps write the centred rows, FP32 Xc and its BF16 pieces.
// Xc = x - m is formed from the mean held as two floats mh + ml: x - mh
// exactly (TwoSum), then one rounding of its sum with -ml, which is within
// 2^-48 |m| of the exact difference. With the matrix-valued kernel (q
// given) that difference is multiplied by sqrt(q_c) rounded to FP32 (so q = 1
// gives the RBF path's values bit for bit), and 1/q_c and 1/sqrt(q_c) are
// kept in FP32 for the update, which then needs no FP64 division per element.
constexpr int kCentreRows = 8;
__global__ void __launch_bounds__(32 * kCentreRows) centre_kernel(
    const float *__restrict__ X, const float *__restrict__ q, int n, int d, int dp, int np,
    double *mean, float *Xc, __nv_bfloat16 *Xh, __nv_bfloat16 *Xm, __nv_bfloat16 *Xl,
    float *qf, int *nonfinite) {
  __shared__ double part[kCentreRows][32];
  __shared__ float mhc[32], mlc[32], sqc[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + tx;
  const bool live = c < d;
  Comp acc;
  if (live)
    for (int i = ty; i < n; i += kCentreRows) acc.add(X[(size_t)i * d + c]);
  part[ty][tx] = acc.value();
  __syncthreads();
  if (ty == 0 && live) {
    double t = 0.0;
    for (int r = 0; r < kCentreRows; ++r) t += part[r][tx];
    if (!isfinite(t)) atomicOr(nonfinite, 1);   // a NaN or infinity in the column
    const double m = t / n;
    mean[c] = m;
    const float mh = (float)m;
    mhc[tx] = mh;
    mlc[tx] = (float)(m - (double)mh);
    const double sq = q ? sqrt((double)q[c]) : 1.0;   // Q-metric scale of the column
    sqc[tx] = (float)sq;
    if (q) {
      qf[c] = (float)(1.0 / (double)q[c]);
      qf[dp + c] = (float)(1.0 / sq);
    }
  }
  __syncthreads();
  const int nblk = (d + 31) / 32;   // blocks holding live columns
  const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
  if ((int)blockIdx.x >= nblk) {    // padding columns only
    for (int i = ty; i < np; i += kCentreRows) {
      if (Xh) Xh[(size_t)i * dp + c] = z;
      if (Xm) { Xm[(size_t)i * dp + c] = z; Xl[(size_t)i * dp + c] = z; }
    }
    return;
  }
  const float nmh = live ? -mhc[tx] : 0.f, ml = live ? mlc[tx] : 0.f;
  const float sqf = live ? sqc[tx] : 1.f;
  for (int i = ty; i < n; i += kCentreRows) {
    const size_t g = (size_t)i * d + c;
    float xc = 0.f;
    if (live) {
      float e;
      const float s = two_sum(X[g], nmh, e);
      xc = __fadd_rn(s, __fsub_rn(e, ml));
      if (q) xc = __fmul_rn(xc, sqf);
      Xc[g] = xc;
    }
    if (Xh) {
      // three-piece BF16 split: each remainder is exact in FP32
      const __nv_bfloat16 h = __float2bfloat16_rn(xc);
      Xh[(size_t)i * dp + c] = h;
      if (Xm) {
        const float r1 = xc - __bfloat162float(h);
        const __nv_bfloat16 mm = __float2bfloat16_rn(r1);
        Xm[(size_t)i * dp + c] = mm;
        Xl[(size_t)i * dp + c] = __float2bfloat16_rn(r1 - __bfloat162float(mm));
      }
    }
  }
  if (Xh)
    for (int i = n + ty; i < np; i += kCentreRows) {
      Xh[(size_t)i * dp + c] = z;
      if (Xm) { Xm[(size_t)i * dp + c] = z; Xl[(size_t)i * dp + c] = z; }
    }
}

// q_c = 1 / Var_j(x_jc), the population variance over the particles, and 1
// where the variance is zero (every particle equal in the column, found
// from the column's minimum and maximum, exactly). A block owns 32 columns
// and its 8 warps interleaved rows, as in centre_kernel: the mean from
// compensated FP32 sums (FP64 across the warps, in a fixed order), then the
// squared deviations x - m (formed as in centre_kernel) summed the same way.
__global__ void __launch_bounds__(32 * kCentreRows) inverse_variance_kernel(
    const float *__restrict__ X, int n, int d, float *q) {
  __shared__ double part[kCentreRows][32];
  __shared__ float mhc[32], mlc[32];
  __shared__ float lo_s[kCentreRows][32], hi_s[kCentreRows][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + tx;
  const bool live = c < d;
  Comp acc;
  float lo = CUDART_INF_F, hi = -CUDART_INF_F;
  if (live)
    for (int i = ty; i < n; i += kCentreRows) {
      const float x = X[(size_t)i * d + c];
      acc.add(x);
      lo = fminf(lo, x);
      hi = fmaxf(hi, x);
    }
  part[ty][tx] = acc.value();
  lo_s[ty][tx] = lo;
  hi_s[ty][tx] = hi;
  __syncthreads();
  if (ty == 0 && live) {
    double t = 0.0;
    for (int r = 0; r < kCentreRows; ++r) t += part[r][tx];
    const double m = t / n;
    const float mh = (float)m;
    mhc[tx] = mh;
    mlc[tx] = (float)(m - (double)mh);
  }
  __syncthreads();
  Comp sq;
  if (live) {
    const float nmh = -mhc[tx], ml = mlc[tx];
    for (int i = ty; i < n; i += kCentreRows) {
      float e;
      const float s = two_sum(X[(size_t)i * d + c], nmh, e);
      sq.add_sq(__fadd_rn(s, __fsub_rn(e, ml)));
    }
  }
  __syncthreads();   // every thread has read part[][] of the first pass
  part[ty][tx] = sq.value();
  __syncthreads();
  if (ty == 0 && live) {
    double v = 0.0;
    float cl = lo_s[0][tx], ch = hi_s[0][tx];
    for (int r = 0; r < kCentreRows; ++r) {
      v += part[r][tx];
      cl = fminf(cl, lo_s[r][tx]);
      ch = fmaxf(ch, hi_s[r][tx]);
    }
    v /= n;
    q[c] = (cl == ch || !(v > 0.0)) ? 1.f : (float)(1.0 / v);
  }
}

__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// |xc_i|^2: a compensated FP32 dot product per thread (16-byte loads where
// the rows are 16-byte aligned), the threads' sums added in FP64.
__global__ void norms_kernel(const float *__restrict__ Xc, int d, double *nrm) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  const float *row = Xc + (size_t)i * d;
  Comp acc;
  if ((d & 3) == 0) {
    const float4 *r4 = reinterpret_cast<const float4 *>(row);
    for (int c = threadIdx.x; c < d / 4; c += blockDim.x) {
      const float4 v = r4[c];
      acc.add_sq(v.x);
      acc.add_sq(v.y);
      acc.add_sq(v.z);
      acc.add_sq(v.w);
    }
  } else {
    for (int c = threadIdx.x; c < d; c += blockDim.x) acc.add_sq(row[c]);
  }
  const double t = block_sum(acc.value(), red);
  if (threadIdx.x == 0) nrm[i] = t;
}

// SIMT FP32 Gram partials (reference path): 64x64 upper-triangle tiles.
__global__ void gram_simt_kernel(const float *__restrict__ Xc, int n, int d, int np, int kchunk,
                                 float *parts) {
  __shared__ float As[32][65], Bs[32][65];
  const int T = (n + 63) / 64;
  int t = blockIdx.x, ti = 0;
  while (t >= T - ti) { t -= T - ti; ++ti; }
  const int tj = ti + t;
  const int i0 = ti * 64, j0 = tj * 64;
  const int k0 = blockIdx.y * kchunk, k1 = min(d, k0 + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  for (int kb = k0; kb < k1; kb += 32) {
    for (int q = threadIdx.x; q < 64 * 32; q += 256) {
      const int r = q >> 5, kk = q & 31;
      const int k = kb + kk;
      As[kk][r] = (i0 + r < n && k < k1) ? Xc[(size_t)(i0 + r) * d + k] : 0.f;
      Bs[kk][r] = (j0 + r < n && k < k1) ? Xc[(size_t)(j0 + r) * d + k] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      float a[4], b[4];
      for (int u = 0; u < 4; ++u) { a[u] = As[kk][ty * 4 + u]; b[u] = Bs[kk][tx * 4 + u]; }
      for (int u = 0; u < 4; ++u)
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
  float *P = parts + (size_t)blockIdx.y * np * np;
  for (int u = 0; u < 4; ++u)
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty * 4 + u, j = j0 + tx * 4 + v;
      if (i < n && j < n) P[(size_t)i * np + j] = acc[u][v];
    }
}

__global__ void copy_d2_kernel(const double *D2, size_t nn, double *out) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nn) out[q] = D2[q];
}

__global__ void d2_finish_kernel(const float *__restrict__ parts, int splits, int n, int np,
                                 const double *nrm, double *D2, unsigned long long *keys) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= n || j < i) return;
  double v = 0.0;
  if (i != j) {
    double g = 0.0;
    for (int s = 0; s < splits; ++s) g += (double)parts[(size_t)s * np * np + (size_t)i * np + j];
    v = nrm[i] + nrm[j] - 2.0 * g;
    if (!(v > 0.0)) v = 0.0;
    const long long idx = (long long)i * n - (long long)i * (i + 1) / 2 + (j - i - 1);
    keys[idx] = (unsigned long long)__double_as_longlong(v);
  }
  D2[(size_t)i * n + j] = v;
  D2[(size_t)j * n + i] = v;
}

// Radix selection of up to two ranks of the multiset {n zeros} U {each upper
// D2 value twice}. sel: [0..1] prefix, [2] mask, [3..4] rank, [5..6] zero flag.
__global__ void median_init_kernel(int n, unsigned long long *sel, unsigned int *hist,
                                   unsigned int *done) {
  const long long N2 = (long long)n * n;
  long long kf[2];
  if (N2 % 2 == 0) { kf[0] = N2 / 2 - 1; kf[1] = N2 / 2; }
  else { kf[0] = kf[1] = (N2 - 1) / 2; }
  for (int r = 0; r < 2; ++r) {
    sel[r] = 0ull;
    const bool z = kf[r] < n;
    sel[5 + r] = z ? 1ull : 0ull;
    sel[3 + r] = z ? 0ull : (unsigned long long)((kf[r] - n) / 2);
  }
  sel[2] = 0ull;
  for (int q = 0; q < 512; ++q) hist[q] = 0u;
  *done = 0u;
}

// Digit selection of one radix pass, by one warp: lane l holds the counts of
// digits 8l .. 8l+7; a warp prefix sum over the lanes' totals finds the lane
// whose digits contain rank k, and that lane walks its eight. The histogram
// is cleared for the next pass by all lanes. The counts are read from L2,
// where the other blocks' atomics went.
__device__ void median_select_warp(int shift, unsigned long long *sel, unsigned int *hist) {
  const int l = threadIdx.x & 31;
  for (int r = 0; r < 2; ++r) {
    if (sel[5 + r]) continue;   // warp-uniform
    const unsigned long long k = sel[3 + r];
    unsigned int cnt[8];
    unsigned long long tot = 0ull;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      cnt[j] = __ldcg(&hist[r * 256 + 8 * l + j]);
      tot += cnt[j];
    }
    unsigned long long incl = tot;   // inclusive prefix over the lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
      if (l >= o) incl += v;
    }
    const unsigned long long excl = incl - tot;
    if (k >= excl && k < incl) {
      unsigned long long cum = excl;
      for (int j = 0; j < 8; ++j) {
        if (k < cum + cnt[j]) {
          sel[r] |= (unsigned long long)(8 * l + j) << shift;
          sel[3 + r] = k - cum;
          break;
        }
        cum += cnt[j];
      }
    }
    __syncwarp();
  }
  if (l == 0) sel[2] |= 255ull << shift;
  __syncwarp();
  for (int q = l; q < 512; q += 32) hist[q] = 0u;
}

// One radix pass: histogram of the 8-bit digit at shift of the keys that
// match the prefix selected so far, for both target ranks. The last block to
// finish (a counter taken after a memory fence) then selects the digits, so
// a pass is one launch.
__global__ void median_hist_kernel(const unsigned long long *__restrict__ keys, int M, int shift,
                                   unsigned long long *sel, unsigned int *hist,
                                   unsigned int *done) {
  __shared__ unsigned int h[512];
  __shared__ bool last;
  for (int q = threadIdx.x; q < 512; q += blockDim.x) h[q] = 0u;
  __syncthreads();
  const unsigned long long mask = sel[2], p0 = sel[0], p1 = sel[1];
  const bool z0 = sel[5] != 0ull, z1 = sel[6] != 0ull;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M; e += gridDim.x * blockDim.x) {
    const unsigned long long u = keys[e];
    const unsigned dg = (unsigned)((u >> shift) & 255ull);
    if (!z0 && (u & mask) == p0) atomicAdd(&h[dg], 1u);
    if (!z1 && (u & mask) == p1) atomicAdd(&h[256 + dg], 1u);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 512; q += blockDim.x)
    if (h[q]) atomicAdd(&hist[q], h[q]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < 32) median_select_warp(shift, sel, hist);
  if (threadIdx.x == 0) *done = 0u;
}

__global__ void bandwidth_kernel(int n, const unsigned long long *sel, float h2_user,
                                 const int *gram_err, double *h2, double *h2_out) {
  double v;
  if (gram_err && *gram_err) {
    v = __longlong_as_double(0x7ff8000000000000ll);   // NaN: the Gram did not complete
  } else if (h2_user > 0.f) {
    v = h2_user;
  } else {
    const double a = sel[5] ? 0.0 : __longlong_as_double((long long)sel[0]);
    const double b = sel[6] ? 0.0 : __longlong_as_double((long long)sel[1]);
    const double med = 0.5 * (a + b);
    v = med < 1e-30 ? 1.0 : med / (2.0 * log((double)n + 1.0));
  }
  h2[0] = v;
  h2[1] = (double)(float)(1.0 / v);   // 1/h^2 in FP32 for the update kernels
  if (h2_out) h2_out[0] = v;
}

__global__ void kbar_kernel(const double *__restrict__ D2, int n, const double *h2, float *K,
                            float *rs) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  const double inv = 1.0 / (2.0 * h2[0]);
  double s = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const float k = (float)exp(-D2[(size_t)i * n + j] * inv);
    K[(size_t)i * n + j] = k;
    s += (double)k;
  }
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) rs[i] = (float)t;
}

// ---------------------------------------------------------------------------
// Blocked right-looking Cholesky of A = Kbar + tau I (FP32), lower factor.
__global__ void chol_init_kernel(const float *K, int n, float tau, float *A, int *flag) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q == 0) *flag = 0;
  if (q >= (size_t)n * n) return;
  const int i = (int)(q / n), j = (int)(q % n);
  A[q] = K[q] + (i == j ? tau : 0.f);
}

constexpr int CB = 32;   // panel width

// Panel k0 of the blocked right-looking Cholesky, one warp per block: every
// block factors the nb x nb diagonal block A11 with lane r holding row r in
// registers (column c's entries of the other rows arrive by shuffle), in the
// operation order of a serial right-looking factorisation, then each lane
// solves one row below the panel, L21 = A21 L11^{-T}, with the row in
// registers and L11 in shared memory. Other blocks may still be reading A11,
// so L11 goes to the side buffer L11 (written by block 0), and the
// trailing-update launch that follows copies it into place; the last panel
// (no rows below, one block) writes it into A directly. A non-positive pivot
// is flagged (by block 0) and replaced by 1 so the factorisation ends.
__global__ void __launch_bounds__(32) chol_panel_kernel(float *A, int n, int k0, float *L11,
                                                        int *flag) {
  __shared__ float S[CB][CB + 1];
  const unsigned full = 0xffffffffu;
  const int nb = min(CB, n - k0);
  const int l = threadIdx.x;
  float a[CB];
#pragma unroll
  for (int c = 0; c < CB; ++c)
    a[c] = (l < nb && c < nb) ? A[(size_t)(k0 + l) * n + k0 + c] : 0.f;
#pragma unroll
  for (int c = 0; c < CB; ++c) {
    if (c < nb) {   // warp-uniform
      float d = __shfl_sync(full, a[c], c);
      if (!(d > 0.f)) {
        if (blockIdx.x == 0 && l == 0) atomicOr(flag, 1);
        d = 1.f;
      }
      const float piv = sqrtf(d);
      if (l == c) a[c] = piv;
      const float inv = 1.f / piv;
      if (l > c) a[c] *= inv;
#pragma unroll
      for (int cc = c + 1; cc < CB; ++cc) {
        const float scc = __shfl_sync(full, a[c], cc);   // scaled entry (cc, c)
        if (cc < nb && l >= cc) a[cc] = fmaf(-a[c], scc, a[cc]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < CB; ++c) S[l][c] = c <= l ? a[c] : 0.f;
  __syncwarp();
  const bool last = k0 + nb >= n;
  if (blockIdx.x == 0 && l < nb) {
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      if (c < nb) {
        if (last) A[(size_t)(k0 + l) * n + k0 + c] = S[l][c];
        else L11[l * nb + c] = S[l][c];
      }
    }
  }
  const int i = k0 + nb + blockIdx.x * 32 + l;
  if (i >= n) return;
  float x[CB];
#pragma unroll
  for (int c = 0; c < CB; ++c) x[c] = c < nb ? A[(size_t)i * n + k0 + c] : 0.f;
#pragma unroll
  for (int c = 0; c < CB; ++c) {
    if (c < nb) {
      float v = x[c];
#pragma unroll
      for (int t = 0; t < c; ++t) v = fmaf(-x[t], S[c][t], v);
      x[c] = v / S[c][c];
    }
  }
#pragma unroll
  for (int c = 0; c < CB; ++c)
    if (c < nb) A[(size_t)i * n + k0 + c] = x[c];
}

// Trailing update A22 -= L21 L21^T on the lower triangle; the first block
// also copies the panel's diagonal factor L11 into A (no block of this
// launch reads A11).
__global__ void chol_update_kernel(float *A, int n, int k0, const float *L11) {
  __shared__ float Ai[CB][65], Aj[CB][65];
  const int nb = min(CB, n - k0);
  const int k1 = k0 + nb;
  if (blockIdx.x == 0 && blockIdx.y == 0)
    for (int q = threadIdx.x; q < nb * nb; q += blockDim.x)
      A[(size_t)(k0 + q / nb) * n + k0 + q % nb] = L11[q];
  const int i0 = k1 + blockIdx.y * 64, j0 = k1 + blockIdx.x * 64;
  if (j0 > i0 + 63) return;
  for (int q = threadIdx.x; q < 64 * CB; q += 256) {
    const int r = q / CB, t = q % CB;
    Ai[t][r] = (i0 + r < n && t < nb) ? A[(size_t)(i0 + r) * n + k0 + t] : 0.f;
    Aj[t][r] = (j0 + r < n && t < nb) ? A[(size_t)(j0 + r) * n + k0 + t] : 0.f;
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  for (int t = 0; t < CB; ++t)
    for (int u = 0; u < 4; ++u)
      for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(Ai[t][ty * 4 + u], Aj[t][tx * 4 + v], acc[u][v]);
  for (int u = 0; u < 4; ++u)
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty * 4 + u, j = j0 + tx * 4 + v;
      if (i < n && j <= i) A[(size_t)i * n + j] -= acc[u][v];
    }
}

__global__ void chol_zero_upper_kernel(float *A, int n) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)n * n) return;
  if ((int)(q % n) > (int)(q / n)) A[q] = 0.f;
}

__global__ void philox_fill_kernel(float *out, int rows, int cols, uint64_t seed, uint64_t it) {
  const int nq = (cols + 3) / 4;
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)rows * nq) return;
  const int i = (int)(q / nq), c4 = (int)(q % nq);
  const float4 z = philox_normal4(seed, it, (uint32_t)i, (uint32_t)c4);
  const float zz[4] = {z.x, z.y, z.z, z.w};
  for (int u = 0; u < 4; ++u) {
    const int c = c4 * 4 + u;
    if (c < cols) out[(size_t)i * cols + c] = zz[u];
  }
}

// ---------------------------------------------------------------------------
// Three-piece BF16 split x ~ h + m + l (each remainder exact in FP32).
__device__ __forceinline__ void split3(float x, __nv_bfloat16 &h, __nv_bfloat16 &m,
                                       __nv_bfloat16 &l) {
  h = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// Operand A of the tensor-core update, [np][Kp]: row i = (Kbar_i, Lk_i) for
// sSVGD or Kbar_i for SVGD, zero-padded.
__global__ void split_a_kernel(const float *__restrict__ K, const float *__restrict__ Lk, int n,
                               int np, int Kp, __nv_bfloat16 *Ah, __nv_bfloat16 *Am,
                               __nv_bfloat16 *Al) {
  const size_t tot = (size_t)np * Kp;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot;
       q += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / Kp), k = (int)(q % Kp);
    float v = 0.f;
    if (i < n) {
      if (k < n) v = K[(size_t)i * n + k];
      else if (Lk && k < 2 * n) v = Lk[(size_t)i * n + (k - n)];
    }
    split3(v, Ah[q], Am[q], Al[q]);
  }
}

// Operand B, [dp][Kp] (coordinates x particles, a transpose through shared
// memory in 64 x 64 tiles, so that every warp reads 256 contiguous bytes of
// a particle row and writes 128 contiguous bytes of each piece's coordinate
// row): column k < n holds Y_kc = (eps/n) (gscale G_kc / q_c -
// Xc_kc / (sqrt(q_c) h^2)), columns n..2n-1 (sSVGD) Z = noise_scale Xi / sqrt(q_c).
constexpr int kSplitTile = 64;
__global__ void __launch_bounds__(256) split_b_kernel(
    const float *__restrict__ G, const float *__restrict__ Xc, const float *__restrict__ Xi,
    const double *h2p, const float *__restrict__ iqc, const float *__restrict__ isqc, int n,
    int d, int dp, int Kp, float en, float gscale, float ns, __nv_bfloat16 *Bh,
    __nv_bfloat16 *Bm, __nv_bfloat16 *Bl, int *nonfinite) {
  __shared__ float tile[kSplitTile][kSplitTile + 1];
  bool bad = false;
  const int c0 = blockIdx.x * kSplitTile, k0 = blockIdx.y * kSplitTile;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const float inv_h2 = (float)h2p[1];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int cc = tx + 32 * h, c = c0 + cc;
    // per-column factors of the matrix-valued kernel (1 without it)
    const float iq = (iqc && c < d) ? iqc[c] : 1.f, isq = (isqc && c < d) ? isqc[c] : 1.f;
    for (int kk = ty; kk < kSplitTile; kk += 8) {
      const int k = k0 + kk;
      float v = 0.f;
      if (c < d) {
        if (k < n) {
          const size_t g = (size_t)k * d + c;
          const float gv = G[g];
          bad |= !isfinite(gv);
          v = en * (gscale * iq * gv - isq * inv_h2 * Xc[g]);
        } else if (Xi && k < 2 * n) {
          v = ns * isq * Xi[(size_t)(k - n) * d + c];
        }
      }
      tile[kk][cc] = v;
    }
  }
  if (bad) atomicOr(nonfinite, 2);
  __syncthreads();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int kk = tx + 32 * h, k = k0 + kk;
    for (int cc = ty; cc < kSplitTile; cc += 8) {
      const int c = c0 + cc;
      if (c < dp && k < Kp) {
        const size_t o = (size_t)c * Kp + k;
        split3(tile[kk][cc], Bh[o], Bm[o], Bl[o]);
      }
    }
  }
}

__global__ void rcoef_kernel(const float *rs, const double *h2p, int n, float en, float *rc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rc[i] = en * rs[i] * (float)h2p[1];
}

// A bounded wait of the tensor-core update gave up: its tiles are unknown,
// so every particle is marked NaN rather than left half-updated.
__global__ void poison_kernel(const int *err, size_t nd, float *X) {
  if (!(*err & 1)) return;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < nd;
       q += (size_t)gridDim.x * blockDim.x)
    X[q] = __int_as_float(0x7fc00000);
}

// Fused update GEMM: per 64x64 tile of (particles x coordinates) accumulate
// Kbar G, Kbar Xc and (sSVGD) Lk Xi over all particles j, then apply Eq. (17)
// (and Eq. 22) with the bound reset.
template <bool NOISE>
__global__ void __launch_bounds__(256) update_kernel(
    const float *__restrict__ K, const float *__restrict__ G, const float *__restrict__ Xc,
    const float *__restrict__ Lk, const float *__restrict__ Xi, const float *__restrict__ rs,
    const double *h2p, int n, int d, float eps, float gscale, float noise_scale,
    const float *__restrict__ iqc, const float *__restrict__ isqc, const float *lo,
    const float *hi, float *X, int *nonfinite) {
  constexpr int BK = 16;
  bool bad = false;
  __shared__ float Ks[BK][64], Ls[NOISE ? BK : 1][64];
  __shared__ __align__(16) float Gs[BK][64], Xs[BK][64], Es[NOISE ? BK : 1][64];
  const int c0 = blockIdx.x * 64, i0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float a1[4][4] = {}, a2[4][4] = {}, a3[4][4] = {};
  for (int j0 = 0; j0 < n; j0 += BK) {
    for (int q = threadIdx.x; q < 64 * BK; q += 256) {
      const int m = q / BK, kk = q % BK;
      const bool ok = (i0 + m < n) && (j0 + kk < n);
      Ks[kk][m] = ok ? K[(size_t)(i0 + m) * n + j0 + kk] : 0.f;
      if (NOISE) Ls[kk][m] = ok ? Lk[(size_t)(i0 + m) * n + j0 + kk] : 0.f;
    }
    for (int q = threadIdx.x; q < 64 * BK; q += 256) {
      const int kk = q / 64, cc = q % 64;
      const bool ok = (j0 + kk < n) && (c0 + cc < d);
      const size_t g = (size_t)(j0 + kk) * d + c0 + cc;
      Gs[kk][cc] = ok ? G[g] : 0.f;
      bad |= !isfinite(Gs[kk][cc]);
      Xs[kk][cc] = ok ? Xc[g] : 0.f;
      if (NOISE) Es[kk][cc] = ok ? Xi[g] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float k4[4], g4[4], x4[4];
      for (int u = 0; u < 4; ++u) {
        k4[u] = Ks[kk][ty * 4 + u];
        g4[u] = Gs[kk][tx * 4 + u];
        x4[u] = Xs[kk][tx * 4 + u];
      }
      for (int u = 0; u < 4; ++u)
        for (int v = 0; v < 4; ++v) {
          a1[u][v] = fmaf(k4[u], g4[v], a1[u][v]);
          a2[u][v] = fmaf(k4[u], x4[v], a2[u][v]);
        }
      if (NOISE) {
        float l4[4], e4[4];
        for (int u = 0; u < 4; ++u) { l4[u] = Ls[kk][ty * 4 + u]; e4[u] = Es[kk][tx * 4 + u]; }
        for (int u = 0; u < 4; ++u)
          for (int v = 0; v < 4; ++v) a3[u][v] = fmaf(l4[u], e4[v], a3[u][v]);
      }
    }
    __syncthreads();
  }
  if (bad) atomicOr(nonfinite, 2);
  const float inv_h2 = (float)h2p[1];
  const float inv_n = 1.f / (float)n;
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + ty * 4 + u;
    if (i >= n) continue;
    const float ri = rs[i];
    for (int v = 0; v < 4; ++v) {
      const int c = c0 + tx * 4 + v;
      if (c >= d) continue;
      const size_t g = (size_t)i * d + c;
      float x;
      if (!iqc) {
        const float rep = (fmaf(ri, Xc[g], -a2[u][v])) * inv_h2;
        const float phi = fmaf(gscale, a1[u][v], rep) * inv_n;
        x = fmaf(eps, phi, X[g]);
        if (NOISE) x = fmaf(noise_scale, a3[u][v], x);
      } else {
        // matrix-valued kernel: Q^{-1} on the driving term, Q^{-1/2} on the
        // repulsion (built from sqrt(q)-scaled Xc) and on the noise
        const float iq = iqc[c], isq = isqc[c];
        const float rep = (fmaf(ri, Xc[g], -a2[u][v])) * inv_h2 * isq;
        const float phi = fmaf(gscale * iq, a1[u][v], rep) * inv_n;
        x = fmaf(eps, phi, X[g]);
        if (NOISE) x = fmaf(noise_scale * isq, a3[u][v], x);
      }
      if (lo) x = fmaxf(x, lo[c]);
      if (hi) x = fminf(x, hi[c]);
      X[g] = x;
    }
  }
}

// Steps 1-5: centring, Gram, FP64 distances and the bandwidth.
static int distances(const float *X, const float *q, int n, int d, float h2, int gp, SvgdWs &w,
                     double *h2_used, cudaStream_t st) {
  const bool tc = gp != VIP_GRAM_FP32;
  const bool x3 = gp == VIP_GRAM_BF16X3;
  VIP_TRY(cudaMemsetAsync(w.flag, 0, 4 * sizeof(int), st));
  centre_kernel<<<w.dp / 32, 32 * kCentreRows, 0, st>>>(X, q, n, d, w.dp, w.np, w.mean, w.Xc,
                                                        tc ? w.Xh : nullptr,
                                                        x3 ? w.Xm : nullptr,
                                                        x3 ? w.Xl : nullptr, w.qf, w.flag + 3);
  VIP_CHECK_LAUNCH();
  norms_kernel<<<n, 256, 0, st>>>(w.Xc, d, w.nrm);
  VIP_CHECK_LAUNCH();
  if (tc) {
    int rc = gram_tc_launch(w.Xh, x3 ? w.Xm : nullptr, x3 ? w.Xl : nullptr, n, w.dp, w.np,
                            w.splits, w.parts, w.flag + 1, st);
    if (rc) return rc;
  } else {
    const int T = idiv_up(n, 64);
    const int kchunk = idiv_up(idiv_up(d, w.splits), 32) * 32;
    gram_simt_kernel<<<dim3(T * (T + 1) / 2, w.splits), 256, 0, st>>>(w.Xc, n, d, w.np, kchunk,
                                                                       w.parts);
    VIP_CHECK_LAUNCH();
  }
  d2_finish_kernel<<<dim3(idiv_up(n, 128), n), 128, 0, st>>>(w.parts, w.splits, n, w.np, w.nrm,
                                                             w.D2, w.keys);
  VIP_CHECK_LAUNCH();
  if (!(h2 > 0.f)) {
    median_init_kernel<<<1, 1, 0, st>>>(n, w.sel, w.hist, w.done);
    VIP_CHECK_LAUNCH();
    if (w.M > 0) {
      const int blocks = std::min(1024, std::max(1, idiv_up(w.M, 256 * 8)));
      for (int shift = 56; shift >= 0; shift -= 8) {
        median_hist_kernel<<<blocks, 256, 0, st>>>(w.keys, w.M, shift, w.sel, w.hist, w.done);
        VIP_CHECK_LAUNCH();
      }
    }
  }
  bandwidth_kernel<<<1, 1, 0, st>>>(n, w.sel, h2, tc ? w.flag + 1 : nullptr, w.h2, h2_used);
  VIP_CHECK_LAUNCH();
  return VIP_OK;
}

static int check_args(const float *X, int n, int d, int gp, void *ws) {
  if (!X || n < 1 || d < 1 || !ws || ((uintptr_t)ws & 255) ||
      (gp != VIP_GRAM_BF16 && gp != VIP_GRAM_BF16X3 && gp != VIP_GRAM_FP32))
    return VIP_ERR_ARG;
  return VIP_OK;
}

// The update runs on the tensor cores (update_tc_launch) for the BF16 Gram
// precisions, or as the SIMT FP32 update_kernel for VIP_GRAM_FP32 (the
// reference path).
static int run_svgd(float *X, const float *G, float gscale, const float *q, int n, int d,
                    float eps, float h2, const float *lo, const float *hi, int gp, void *ws,
                    size_t ws_bytes, double *h2_used, bool stochastic, uint64_t seed,
                    uint64_t it, const float *xi, double *tau_used, cudaStream_t st) {
  if (check_args(X, n, d, gp, ws) || !G || !(eps >= 0.f)) return VIP_ERR_ARG;
  SvgdWs w;
  const size_t need = layout(n, d, gp, stochastic, gp != VIP_GRAM_FP32, ws, ws_bytes, w);
  if (need > ws_bytes) return VIP_ERR_NOMEM;
  int rc = distances(X, q, n, d, h2, gp, w, h2_used, st);
  if (rc) return rc;
  kbar_kernel<<<n, 256, 0, st>>>(w.D2, n, w.h2, w.K, w.rs);
  VIP_CHECK_LAUNCH();
  const dim3 ug(idiv_up(d, 64), idiv_up(n, 64));
  const float en = eps / (float)n;
  auto tc_update = [&](const float *Lk, const float *noise, float ns) -> int {
    split_a_kernel<<<1024, 256, 0, st>>>(w.K, Lk, n, w.unp, w.uKp, w.Ua[0], w.Ua[1], w.Ua[2]);
    VIP_CHECK_LAUNCH();
    split_b_kernel<<<dim3(w.udp / kSplitTile, w.uKp / kSplitTile), 256, 0, st>>>(
        G, w.Xc, noise, w.h2, q ? w.qf : nullptr, q ? w.qf + w.dp : nullptr, n, d, w.udp,
        w.uKp, en, gscale, ns, w.Ub[0], w.Ub[1], w.Ub[2], w.flag + 3);
    VIP_CHECK_LAUNCH();
    rcoef_kernel<<<idiv_up(n, 256), 256, 0, st>>>(w.rs, w.h2, n, en, w.rcoef);
    VIP_CHECK_LAUNCH();
    int rc2 = update_tc_launch(w.Ua, w.Ub, n, d, w.unp, w.udp, w.uKp, w.Xc, w.rcoef,
                               q ? w.qf + w.dp : nullptr, lo, hi, X, w.flag + 2, w.flag + 3, st);
    if (rc2) return rc2;
    poison_kernel<<<1024, 256, 0, st>>>(w.flag + 2, (size_t)n * d, X);
    VIP_CHECK_LAUNCH();
    return VIP_OK;
  };
  if (!stochastic && w.tcu) return tc_update(nullptr, nullptr, 0.f);
  if (!stochastic) {
    update_kernel<false><<<ug, 256, 0, st>>>(w.K, G, w.Xc, nullptr, nullptr, w.rs, w.h2, n, d,
                                             eps, gscale, 0.f, q ? w.qf : nullptr,
                                             q ? w.qf + w.dp : nullptr, lo, hi, X, w.flag + 3);
    VIP_CHECK_LAUNCH();
    return VIP_OK;
  }
  // sSVGD: jittered Cholesky with retries, then the noisy update
  double tau = 1e-6 * n;
  bool ok = false;
  const size_t nn = (size_t)n * n;
  for (int attempt = 0; attempt < 4 && !ok; ++attempt, tau *= 10.0) {
    chol_init_kernel<<<(unsigned)idiv_up((int)std::min(nn, (size_t)1 << 30), 256), 256, 0, st>>>(
        w.K, n, (float)tau, w.Lk, w.flag);
    VIP_CHECK_LAUNCH();
    for (int k0 = 0; k0 < n; k0 += CB) {
      const int rest = n - k0 - std::min(CB, n - k0);
      chol_panel_kernel<<<std::max(1, idiv_up(rest, 32)), 32, 0, st>>>(w.Lk, n, k0, w.L11,
                                                                      w.flag);
      VIP_CHECK_LAUNCH();
      if (rest > 0) {
        const int nb64 = idiv_up(rest, 64);
        chol_update_kernel<<<dim3(nb64, nb64), 256, 0, st>>>(w.Lk, n, k0, w.L11);
        VIP_CHECK_LAUNCH();
      }
    }
    int hflag = 0;
    VIP_TRY(cudaMemcpyAsync(&hflag, w.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    VIP_TRY(cudaStreamSynchronize(st));
    ok = hflag == 0;
    if (ok) break;
  }
  if (!ok) return VIP_ERR_NOTPD;
  if (tau_used) VIP_TRY(cudaMemcpyAsync(tau_used, &tau, sizeof(double), cudaMemcpyHostToDevice, st));
  chol_zero_upper_kernel<<<(unsigned)idiv_up((int)std::min(nn, (size_t)1 << 30), 256), 256, 0, st>>>(
      w.Lk, n);
  VIP_CHECK_LAUNCH();
  const float *noise = xi;
  if (!noise) {
    const size_t nq = (size_t)n * idiv_up(d, 4);
    philox_fill_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(w.Xi, n, d, seed, it);
    VIP_CHECK_LAUNCH();
    noise = w.Xi;
  }
  const float ns = (float)std::sqrt(2.0 * (double)eps / n);
  if (w.tcu) {
    rc = tc_update(w.Lk, noise, ns);
    if (rc) return rc;
    if (tau_used) VIP_TRY(cudaStreamSynchronize(st));
    return VIP_OK;
  }
  update_kernel<true><<<ug, 256, 0, st>>>(w.K, G, w.Xc, w.Lk, noise, w.rs, w.h2, n, d, eps, gscale,
                                          ns, q ? w.qf : nullptr, q ? w.qf + w.dp : nullptr, lo,
                                          hi, X, w.flag + 3);
  VIP_CHECK_LAUNCH();
  // tau is a host local: make the asynchronous copy complete before return
  if (tau_used) VIP_TRY(cudaStreamSynchronize(st));
  return VIP_OK;
}

// Scratch of svgd_step_noalloc: a fixed array in device memory that exists
// for as long as the library is loaded, on every GPU that loads it. Host code
// must not pass the symbol itself to a kernel (on the host it names a shadow
// variable, not device memory): its device address is looked up once per
// device with cudaGetSymbolAddress, with that device current.
constexpr size_t kNoallocScratchBytes = (size_t)VIP_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[128] = {};

static int noalloc_scratch(void **out) {
  int dev = -1;
  VIP_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return VIP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    VIP_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    if (!p || ((uintptr_t)p & 255)) return VIP_ERR_CUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return VIP_OK;
}

}  // namespace vip

using namespace vip;

extern "C" {

int svgd_step_noalloc(float *X, const float *G, float gscale, int n, int d, float eps, float h2,
                      const float *lo, const float *hi, int gram_precision, double *h2_used,
                      vip_stream_t stream) {
  if (!X || !G || n < 1 || d < 1 || !(eps >= 0.f) ||
      (gram_precision != VIP_GRAM_BF16 && gram_precision != VIP_GRAM_BF16X3 &&
       gram_precision != VIP_GRAM_FP32))
    return VIP_ERR_ARG;
  SvgdWs w;
  // size check before any device call: oversize problems never touch the GPU
  if (layout(n, d, gram_precision, 0, gram_precision != VIP_GRAM_FP32, nullptr, 0, w) + 256 >
      kNoallocScratchBytes)
    return VIP_ERR_NOMEM;
  void *ws = nullptr;
  int rc = noalloc_scratch(&ws);
  if (rc) return rc;
  return run_svgd(X, G, gscale, nullptr, n, d, eps, h2, lo, hi, gram_precision, ws,
                  kNoallocScratchBytes, h2_used, false, 0, 0, nullptr, nullptr, stream);
}

int svgd_status(const void *ws, vip_stream_t stream) {
  if (!ws || ((uintptr_t)ws & 255)) return VIP_ERR_ARG;
  int f[4] = {0, 0, 0, 0};
  VIP_TRY(cudaMemcpyAsync(f, ws, sizeof f, cudaMemcpyDeviceToHost, stream));
  VIP_TRY(cudaStreamSynchronize(stream));
  if ((f[1] | f[2]) & 1) return VIP_ERR_TIMEOUT;
  if (f[3]) return VIP_ERR_NONFINITE;
  return VIP_OK;
}

size_t svgd_workspace_size(int n, int d, int gram_precision, int stochastic) {
  if (n < 1 || d < 1) return 0;
  SvgdWs w;
  return layout(n, d, gram_precision, stochastic, gram_precision != VIP_GRAM_FP32, nullptr, 0,
                w) + 256;
}

int svgd_step(float *X, const float *G, float gscale, int n, int d, float eps, float h2,
              const float *lo, const float *hi, int gram_precision, void *ws, size_t ws_bytes,
              double *h2_used, vip_stream_t stream) {
  return run_svgd(X, G, gscale, nullptr, n, d, eps, h2, lo, hi, gram_precision, ws, ws_bytes,
                  h2_used, false, 0, 0, nullptr, nullptr, stream);
}

int ssvgd_step(float *X, const float *G, float gscale, int n, int d, float eps, float h2,
               const float *lo, const float *hi, int gram_precision, void *ws, size_t ws_bytes,
               double *h2_used, uint64_t seed, uint64_t iter, const float *xi,
               double *tau_used, vip_stream_t stream) {
  return run_svgd(X, G, gscale, nullptr, n, d, eps, h2, lo, hi, gram_precision, ws, ws_bytes,
                  h2_used, true, seed, iter, xi, tau_used, stream);
}

int svgd_step_q(float *X, const float *G, float gscale, const float *q, int n, int d, float eps,
                float h2, const float *lo, const float *hi, int gram_precision, void *ws,
                size_t ws_bytes, double *h2_used, vip_stream_t stream) {
  if (!q) return VIP_ERR_ARG;
  return run_svgd(X, G, gscale, q, n, d, eps, h2, lo, hi, gram_precision, ws, ws_bytes, h2_used,
                  false, 0, 0, nullptr, nullptr, stream);
}

int ssvgd_step_q(float *X, const float *G, float gscale, const float *q, int n, int d, float eps,
                 float h2, const float *lo, const float *hi, int gram_precision, void *ws,
                 size_t ws_bytes, double *h2_used, uint64_t seed, uint64_t iter, const float *xi,
                 double *tau_used, vip_stream_t stream) {
  if (!q) return VIP_ERR_ARG;
  return run_svgd(X, G, gscale, q, n, d, eps, h2, lo, hi, gram_precision, ws, ws_bytes, h2_used,
                  true, seed, iter, xi, tau_used, stream);
}

int svgd_inverse_variance(const float *X, int n, int d, float *q, vip_stream_t stream) {
  if (!X || !q || n < 1 || d < 1) return VIP_ERR_ARG;
  inverse_variance_kernel<<<idiv_up(d, 32), 32 * kCentreRows, 0, stream>>>(X, n, d, q);
  VIP_CHECK_LAUNCH();
  return VIP_OK;
}

int svgd_sqdist(const float *X, int n, int d, int gram_precision, double *D2,
                double *h2_used, void *ws, size_t ws_bytes, vip_stream_t stream) {
  if (check_args(X, n, d, gram_precision, ws) || !D2) return VIP_ERR_ARG;
  SvgdWs w;
  if (layout(n, d, gram_precision, 0, false, ws, ws_bytes, w) > ws_bytes) return VIP_ERR_NOMEM;
  int rc = distances(X, nullptr, n, d, 0.f, gram_precision, w, h2_used, stream);
  if (rc) return rc;
  const size_t nn = (size_t)n * n;
  copy_d2_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, stream>>>(w.D2, nn, D2);
  VIP_CHECK_LAUNCH();
  return VIP_OK;
}

int vip_philox_normal(float *out, int rows, int cols, uint64_t seed, uint64_t iter,
                      vip_stream_t stream) {
  if (!out || rows < 1 || cols < 1) return VIP_ERR_ARG;
  const size_t nq = (size_t)rows * idiv_up(cols, 4);
  philox_fill_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, stream>>>(out, rows, cols, seed, iter);
  VIP_CHECK_LAUNCH();
  return VIP_OK;
}

}  // extern "C"
