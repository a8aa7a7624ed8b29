// Wave-propagation kernels of the FWI hot path: forward modelling, exact
// discrete adjoint and imaging condition for the 2-D constant-density
// acoustic wave equation (paper Sec. 3 and Sec. 4.2).
//
// Scheme (one time step, padded grid of NZ x NX cells):
//   a^{n+1} = g [2 a^n + w' (Lh a^n + f_n delta_src)] - g^2 a^{n-1}
// with w' = (vpad dt / dx)^2, Lh the 8th-order 5-arm Laplacian without the
// 1/dx^2 factor (zero values outside the grid), g the Cerjan taper and f_n the
// Ricker wavelet at t = n dt. This is the recurrence
//   a^{n+1} = g [2 a^n + w (L a^n + s^n)] - g^2 a^{n-1},  w = vpad^2 dt^2,
// multiplied through by dx^2 inside the bracket.
//
// Adjoint. With lambda the exact discrete adjoint state,
//   lambda^k = (2I + L W) G lambda^{k+1} - G^2 lambda^{k+2} + rho^k,
// the scaled field mu = w g lambda obeys the same recurrence as the forward
// field, run backwards in time with the data residuals as sources:
//   mu^k = g [2 mu^{k+1} + w' (Lh mu^{k+1} + dx^2 rho^k)] - g^2 mu^{k+2},
// and the gradient of the misfit with respect to the padded velocity is
//   dJ/dvpad = 2 vpad dt^2 sum_n g lambda^{n+1} (L a^n + s^n)
//            = 2 / (vpad dx^2) sum_k mu^k D^k,
// D^k = Lh a^{k-1} + f_{k-1} delta_src being the bracketed Laplacian term the
// forward step already forms (the discrete counterpart of the -2/v^3 u_tt
// cross-correlation). The forward pass therefore stores D^k (FP32, BF16 or
// FP16 with a power-of-two scale per 128 cells) and the adjoint pass reads it
// back; with a restart-checkpoint interval K > 1 only the state every K steps
// is stored and each K-step segment is recomputed before its adjoint sweep.
//
// Batched kernel (FWI_MODE_BATCHED). One thread-block cluster of Q CTAs owns
// one (particle, source range) work item at a time. CTA b of the cluster
// keeps rows [b Hb, (b+1) Hb) of the padded grid in shared memory for all
// time steps: the two time levels of the propagated field (double-buffered,
// with 4 zero columns on either side), w' and the gradient accumulator.
// Each thread updates 4 adjacent cells (one float4) over V consecutive rows,
// holding the 9-row vertical stencil window in registers; the 4 rows above
// and below the band are read from the neighbouring CTAs' shared memory
// (distributed shared memory). One cluster barrier separates time steps.
// Global memory sees only the stored snapshots, the traces and the result.
//
// Plain kernels (FWI_MODE_PLAIN): one launch per time step for one
// (particle, source) pair, fields in global memory, one cell per thread.
// Both paths evaluate each cell update with the same explicitly rounded
// operation sequence, so their wavefields agree bit for bit.
#pragma once
#include "common.cuh"
#include <cooperative_groups.h>

namespace vip {
namespace cg = cooperative_groups;

enum WaveMode { WM_FORWARD = 0, WM_GRADIENT = 1, WM_ADJOINT = 2 };

struct WaveParams {
  // grid and time axis
  int nz, nx, nb, NZ, NX, N, S, R;
  float dtdx;            // dt / dx
  float dx2;             // dx^2
  float c1, c2, c3, c4;   // c1..c4 of the 8th-order stencil (c0 = -2 sum c_k)
  float w_cfl;           // largest stable w' = (v dt/dx)^2
  // band decomposition
  int Q, Hb, NXg, PX, ntask, ntask_pad, nwblk;
  // tables
  const float *gz;       // [Q*Hb] taper per padded row, 0 for dead rows
  const float *gx;       // [NXg*4] taper per padded column, 0 for dead columns
  const float *wavelet;  // [N] Ricker samples f(n dt)
  const int *src_z, *src_x;     // [S] padded source cell
  const uint32_t *rmask; // [Q*ntask_pad] receivers in each thread task
  const int *rbase;      // [Q*ntask_pad] first entry in rperm
  const int *rperm;      // [R] receiver numbers in task order
  // work decomposition
  int P, items, ipp, spi;
  int K, nseg;           // restart-checkpoint interval, segments
  // problem data
  const float *v;        // [P][nz][nx]
  const float *dobs;     // [S][R][N]
  const float *dseis;    // [P][S][R][N]
  float rho_scale;       // dx^2/sigma^2 (gradient) or dx^2 (adjoint)
  float *seis;           // [P][S][R][N]
  double *Jpart;         // [P*S][Q] sum of squared residuals per CTA
  float *grad;           // [P][nz][nx]
  int grad_atomic;       // 1 when several work items share a particle: each
                         // item then writes its partial gradient to GI
  float *GI;             // [items][nz][nx] partial gradients (split items)
  int *status;           // bit 0: CFL violation
  // per-cluster scratch slots
  void *Dbuf;   size_t Dslot;    // snapshot elements per slot
  float *Dscale; size_t DSslot;  // FP16 scales per slot
  float *rho;   size_t rhoslot;  // [R][N] adjoint sources per slot
  float *GP;    size_t GPslot;   // [NZ][NX] gradient gather per slot
  float *CK;    size_t CKslot;   // restart checkpoints per slot
  float *AS;    size_t ASslot;   // parked adjoint state per slot
};

// ---------------------------------------------------------------------------
// storage of the D snapshots
template <class DT> struct Snap;
template <> struct Snap<float> {
  static constexpr bool scaled = false;
  __device__ static void st(float *p, size_t i, float4 v, float) {
    *reinterpret_cast<float4 *>(p + i) = v;
  }
  __device__ static float4 ld(const float *p, size_t i, float) {
    return *reinterpret_cast<const float4 *>(p + i);
  }
};
template <> struct Snap<__nv_bfloat16> {
  static constexpr bool scaled = false;
  __device__ static void st(__nv_bfloat16 *p, size_t i, float4 v, float) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
    __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t *>(&a);
    u.y = *reinterpret_cast<uint32_t *>(&b);
    *reinterpret_cast<uint2 *>(p + i) = u;
  }
  __device__ static float4 ld(const __nv_bfloat16 *p, size_t i, float) {
    uint2 u = *reinterpret_cast<const uint2 *>(p + i);
    __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162 *>(&u.x);
    __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162 *>(&u.y);
    float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
  }
};
template <> struct Snap<__half> {
  static constexpr bool scaled = true;
  __device__ static void st(__half *p, size_t i, float4 v, float mul) {
    __half2 a = __floats2half2_rn(v.x * mul, v.y * mul);
    __half2 b = __floats2half2_rn(v.z * mul, v.w * mul);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t *>(&a);
    u.y = *reinterpret_cast<uint32_t *>(&b);
    *reinterpret_cast<uint2 *>(p + i) = u;
  }
  __device__ static float4 ld(const __half *p, size_t i, float inv) {
    uint2 u = *reinterpret_cast<const uint2 *>(p + i);
    __half2 a = *reinterpret_cast<__half2 *>(&u.x);
    __half2 b = *reinterpret_cast<__half2 *>(&u.y);
    float2 fa = __half22float2(a), fb = __half22float2(b);
    return make_float4(fa.x * inv, fa.y * inv, fb.x * inv, fb.y * inv);
  }
};

__device__ __forceinline__ float4 ld4(const float *p) {
  return *reinterpret_cast<const float4 *>(p);
}
__device__ __forceinline__ void st4(float *p, float4 v) {
  *reinterpret_cast<float4 *>(p) = v;
}
__device__ __forceinline__ float comp(const float4 &v, int j) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

// Laplacian bracket of one cell, 2 c0 u + sum_k c_k (h_k + v_k) with h_k, v_k
// the sums of the two neighbours at distance k along x and z. Because the
// coefficients sum to zero (c0 = -2 sum_k c_k) it equals
//   sum_k c_k [ ((h_k + v_k) - 4u) ],
// which is evaluated here, smallest coefficients first: the bracketed
// differences are small and nearly exact, so the FP32 rounding error of the
// bracket stays proportional to the bracket itself instead of to the 5.7 u
// that the first form cancels. Every operation is rounded explicitly so that
// all kernels agree bit for bit.
// h[0..7] = u at offsets -4,-3,-2,-1,+1,+2,+3,+4 along x; vv likewise along z.
__device__ __forceinline__ float lap_cell(const WaveParams &p, float u,
                                          const float h[8], const float vv[8]) {
  const float u4 = __fmul_rn(4.f, u);
  float s = __fmul_rn(p.c4, __fsub_rn(__fadd_rn(__fadd_rn(h[0], h[7]), __fadd_rn(vv[0], vv[7])), u4));
  s = __fmaf_rn(p.c3, __fsub_rn(__fadd_rn(__fadd_rn(h[1], h[6]), __fadd_rn(vv[1], vv[6])), u4), s);
  s = __fmaf_rn(p.c2, __fsub_rn(__fadd_rn(__fadd_rn(h[2], h[5]), __fadd_rn(vv[2], vv[5])), u4), s);
  s = __fmaf_rn(p.c1, __fsub_rn(__fadd_rn(__fadd_rn(h[3], h[4]), __fadd_rn(vv[3], vv[4])), u4), s);
  return s;
}

// New value of a cell from the bracket s, own value u, previous value ap.
__device__ __forceinline__ float update_cell(float g, float w, float s, float u,
                                             float ap) {
  float t = __fmaf_rn(w, s, __fadd_rn(u, u));
  return __fmul_rn(g, __fmaf_rn(-g, ap, t));
}

// ---------------------------------------------------------------------------
// Batched persistent cluster kernel.
struct Band {
  float *U[2];                 // local field buffers [Hb][PX]
  const float *up[2], *dn[2];  // neighbours' buffers (generic) or zero row
  const float *Zr;             // one row of zeros
  float *W;                    // [Hb][NXg*4] w'
  float *Gm;                   // [Hb][NXg*4] gradient accumulator
  float *gzs;                  // [Hb]
  float *gxs;                  // [NXg*4]
  int b;
};

// Row rr (band-local, -4 <= rr < Hb + 4) of the current level: own rows from
// shared memory, the 4 rows beyond either band edge from the neighbouring
// CTA (distributed shared memory) or zeros at the grid boundary.
__device__ __forceinline__ const float *band_row(const float *cur, const float *up,
                                                 const float *dn, const float *Zr,
                                                 int rr, int Hb, int PX) {
  if (rr < 0) return up == Zr ? Zr : up + (rr + Hb) * PX;
  if (rr >= Hb) return dn == Zr ? Zr : dn + (rr - Hb) * PX;
  return cur + rr * PX;
}

// Per-step context of the cell loop.
struct StepArgs {
  int ph;            // which local buffer holds the current level
  int t;             // forward: n (computes a^{n+1}); adjoint: k (computes mu^k)
  int slot;
  int pair;          // p*S + s
  int s;             // source number
  int src_task, src_bit;   // forward source position in this CTA (or -1)
  float src_val;
  bool record;       // forward: write traces / residuals
  size_t dofs;       // element offset of this step's snapshot slab
  size_t sofs;       // offset of this step's scale slab
  double *Jacc;      // per-thread squared-residual accumulator
};

template <int V, bool ADJ, bool SNAP, int MODE, class DT>
__device__ __forceinline__ void band_step(const WaveParams &p, const Band &B,
                                          const StepArgs &a, int tid, int T) {
  const int Hb = p.Hb, PX = p.PX, NXg = p.NXg, W4 = NXg * 4;
  const float *cur = a.ph ? B.U[1] : B.U[0];
  float *nxt = a.ph ? B.U[0] : B.U[1];
  const float *up = a.ph ? B.up[1] : B.up[0];
  const float *dn = a.ph ? B.dn[1] : B.dn[0];
  const float *Zr = B.Zr;
  DT *Dp = reinterpret_cast<DT *>(p.Dbuf) + a.slot * p.Dslot + a.dofs;
  float *Sp = Snap<DT>::scaled ? p.Dscale + a.slot * p.DSslot + a.sofs : nullptr;
  for (int task0 = tid; task0 < p.ntask_pad; task0 += T) {
    const bool valid = task0 < p.ntask;
    const int task = valid ? task0 : p.ntask - 1;
    const int sp = task / NXg;
    const int cgp = task - sp * NXg;
    const int r0 = sp * V;
    const int col = (cgp + 1) * 4;
    const int gcol = cgp * 4;
    const float4 gx4 = ld4(B.gxs + gcol);
    uint32_t rm = 0;
    int rb = 0;
    if ((!ADJ && a.record) || (ADJ && MODE != WM_FORWARD)) {
      rm = valid ? p.rmask[B.b * p.ntask_pad + task] : 0u;
      rb = p.rbase[B.b * p.ntask_pad + task];
    }
    float4 win[9];
#pragma unroll
    for (int i = 0; i < 8; ++i) win[i] = ld4(band_row(cur, up, dn, Zr, r0 - 4 + i, Hb, PX) + col);
#pragma unroll
    for (int i = 0; i < V; ++i) {
      const int r = r0 + i;
      win[8] = ld4(band_row(cur, up, dn, Zr, r + 4, Hb, PX) + col);
      const float *rp = cur + r * PX + col;
      const float4 Lf = ld4(rp - 4), Rf = ld4(rp + 4), C = win[4];
      const float hrow[12] = {Lf.x, Lf.y, Lf.z, Lf.w, C.x, C.y, C.z, C.w,
                              Rf.x, Rf.y, Rf.z, Rf.w};
      float s4[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float h[8], vv[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          h[k] = hrow[j + k];          // offsets -4..-1
          h[4 + k] = hrow[j + 5 + k];  // offsets +1..+4
          vv[k] = comp(win[k], j);
          vv[4 + k] = comp(win[5 + k], j);
        }
        s4[j] = lap_cell(p, hrow[4 + j], h, vv);
      }
      const uint32_t rbits = (rm >> (4 * i)) & 0xFu;
      if (!ADJ) {
        if (task == a.src_task && valid && (a.src_bit >> 2) == i)
          s4[a.src_bit & 3] = __fadd_rn(s4[a.src_bit & 3], a.src_val);
      } else if (MODE != WM_FORWARD && rbits) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (rbits & (1u << j)) {
            const int rr = p.rperm[rb + __popc(rm & ((1u << (4 * i + j)) - 1u))];
            float val;
            if (MODE == WM_GRADIENT)
              val = p.rho[a.slot * p.rhoslot + (size_t)rr * p.N + (a.t - 1)];
            else
              val = __fmul_rn(p.rho_scale,
                              p.dseis[((size_t)a.pair * p.R + rr) * p.N + (a.t - 1)]);
            s4[j] = __fadd_rn(s4[j], val);
          }
        }
      }
      const size_t cell = (size_t)r * W4 + gcol;
      const float4 Wv = ld4(B.W + cell);
      const float gzr = B.gzs[r];
      const float4 AP = ld4(nxt + r * PX + col);
      float4 an;
      an.x = update_cell(__fmul_rn(gzr, gx4.x), Wv.x, s4[0], C.x, AP.x);
      an.y = update_cell(__fmul_rn(gzr, gx4.y), Wv.y, s4[1], C.y, AP.y);
      an.z = update_cell(__fmul_rn(gzr, gx4.z), Wv.z, s4[2], C.z, AP.z);
      an.w = update_cell(__fmul_rn(gzr, gx4.w), Wv.w, s4[3], C.w, AP.w);
      if (valid) st4(nxt + r * PX + col, an);
      if (SNAP) {
        const float4 sv = make_float4(s4[0], s4[1], s4[2], s4[3]);
        if (!ADJ) {
          float mul = 1.f;
          if (Snap<DT>::scaled) {
            float m = valid ? fmaxf(fmaxf(fabsf(sv.x), fabsf(sv.y)),
                                    fmaxf(fabsf(sv.z), fabsf(sv.w)))
                            : 0.f;
            m = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(m)));
            int e = 0;
            if (m > 0.f) { frexpf(m, &e); e = 15 - e; }
            e = max(-120, min(120, e));
            mul = ldexpf(1.f, e);
            if ((tid & 31) == 0) Sp[(task0 / 32) * V + i] = ldexpf(1.f, -e);
          }
          if (valid) Snap<DT>::st(Dp, cell, sv, mul);
        } else {
          const float inv = Snap<DT>::scaled ? Sp[(task0 / 32) * V + i] : 1.f;
          const float4 dv = Snap<DT>::ld(Dp, cell, inv);
          if (valid) {
            float4 gm = ld4(B.Gm + cell);
            gm.x = __fmaf_rn(an.x, dv.x, gm.x);
            gm.y = __fmaf_rn(an.y, dv.y, gm.y);
            gm.z = __fmaf_rn(an.z, dv.z, gm.z);
            gm.w = __fmaf_rn(an.w, dv.w, gm.w);
            st4(B.Gm + cell, gm);
          }
        }
      }
      if (!ADJ && a.record && rbits) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (rbits & (1u << j)) {
            const int rr = p.rperm[rb + __popc(rm & ((1u << (4 * i + j)) - 1u))];
            const float d = comp(an, j);
            if (MODE == WM_FORWARD) {
              p.seis[((size_t)a.pair * p.R + rr) * p.N + a.t] = d;
            } else if (MODE == WM_GRADIENT) {
              const double res =
                  (double)d - (double)p.dobs[((size_t)a.s * p.R + rr) * p.N + a.t];
              *a.Jacc = __fma_rn(res, res, *a.Jacc);
              p.rho[a.slot * p.rhoslot + (size_t)rr * p.N + a.t] =
                  (float)(res * (double)p.rho_scale);
            }
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) win[k] = win[k + 1];
    }
  }
}

// Copy the own band of both levels between shared memory and a global slab.
__device__ __forceinline__ void band_copy(const WaveParams &p, const Band &B, int ph,
                                          float *g, bool to_global, int tid, int T) {
  const int W4 = p.NXg * 4;
  const int n4 = p.Hb * p.NXg;
  for (int lvl = 0; lvl < 2; ++lvl) {
    float *buf = (ph ^ lvl) ? B.U[1] : B.U[0];
    float *gg = g + (size_t)lvl * p.Hb * W4;
    for (int q = tid; q < n4; q += T) {
      const int r = q / p.NXg, c = q - r * p.NXg;
      float *sp = buf + r * p.PX + (c + 1) * 4;
      float *gp = gg + (size_t)r * W4 + c * 4;
      if (to_global) st4(gp, ld4(sp));
      else st4(sp, ld4(gp));
    }
  }
}

__device__ __forceinline__ void band_zero(const WaveParams &p, const Band &B, int tid, int T) {
  const int n = 2 * p.Hb * p.PX;
  for (int q = tid; q < n / 4; q += T) st4(B.U[0] + 4 * q, make_float4(0.f, 0.f, 0.f, 0.f));
}

template <int V, int MODE, class DT>
__global__ void __launch_bounds__(512, 1) wave_cluster_kernel(const __grid_constant__ WaveParams p) {
  cg::cluster_group cluster = cg::this_cluster();
  const int b = (int)cluster.block_rank();
  const int cid = blockIdx.x / p.Q;
  const int ncl = gridDim.x / p.Q;
  const int tid = threadIdx.x, T = blockDim.x;
  extern __shared__ __align__(16) float smem[];
  const int HP = p.Hb * p.PX;
  const int HW = p.Hb * p.NXg * 4;
  Band B;
  B.b = b;
  B.U[0] = smem;
  B.U[1] = smem + HP;
  float *Zr = smem + 2 * HP;
  B.Zr = Zr;
  B.W = Zr + p.PX;
  B.Gm = B.W + HW;
  B.gzs = B.Gm + (MODE != WM_FORWARD ? HW : 0);
  B.gxs = B.gzs + ((p.Hb + 3) & ~3);
  for (int ph = 0; ph < 2; ++ph) {
    B.up[ph] = b > 0 ? cluster.map_shared_rank(B.U[ph], b - 1) : Zr;
    B.dn[ph] = b < p.Q - 1 ? cluster.map_shared_rank(B.U[ph], b + 1) : Zr;
  }
  for (int q = tid; q < p.PX; q += T) Zr[q] = 0.f;
  for (int q = tid; q < p.Hb; q += T) B.gzs[q] = p.gz[b * p.Hb + q];
  for (int q = tid; q < p.NXg * 4; q += T) B.gxs[q] = p.gx[q];
  const int W4 = p.NXg * 4;
  const size_t slab = (size_t)p.Q * p.Hb * W4;   // elements of one snapshot

  for (int item = cid; item < p.items; item += ncl) {
    const int pp = item / p.ipp;
    const int s0 = (item - pp * p.ipp) * p.spi;
    const int s1 = min(p.S, s0 + p.spi);
    // model coefficients w' = (vpad dt/dx)^2 of this band; CFL check
    const float *vp = p.v + (size_t)pp * p.nz * p.nx;
    bool cfl_bad = false;
    for (int q = tid; q < HW; q += T) {
      const int r = q / W4, x = q - r * W4;
      const int z = b * p.Hb + r;
      float w = 0.f;
      if (z < p.NZ && x < p.NX) {
        const int iz = min(max(z - p.nb, 0), p.nz - 1);
        const int ix = min(max(x - p.nb, 0), p.nx - 1);
        const float c = __fmul_rn(vp[(size_t)iz * p.nx + ix], p.dtdx);
        w = __fmul_rn(c, c);
        cfl_bad |= !(w <= p.w_cfl);
      }
      B.W[q] = w;
      if (MODE != WM_FORWARD) B.Gm[q] = 0.f;
    }
    if (cfl_bad) atomicOr(p.status, 1);

    for (int s = s0; s < s1; ++s) {
      const int pair = pp * p.S + s;
      // source position in this band
      int src_task = -1, src_bit = 0;
      {
        const int z = p.src_z[s], x = p.src_x[s];
        const int rr = z - b * p.Hb;
        if (rr >= 0 && rr < p.Hb) {
          src_task = (rr / V) * p.NXg + x / 4;
          src_bit = (rr % V) * 4 + (x & 3);
        }
      }
      // ---------------- forward sweep
      band_zero(p, B, tid, T);
      cluster.sync();
      double jacc = 0.0;
      int ph = 0;
      for (int n = 0; n < p.N; ++n) {
        StepArgs a;
        a.ph = ph; a.t = n; a.slot = cid; a.pair = pair; a.s = s;
        a.src_task = src_task; a.src_bit = src_bit; a.src_val = p.wavelet[n];
        a.record = true; a.Jacc = &jacc;
        if (MODE == WM_FORWARD || p.K > 1) {
          if (MODE != WM_FORWARD && n % p.K == 0)
            band_copy(p, B, ph, p.CK + cid * p.CKslot + (size_t)(n / p.K) * 2 * slab +
                                    (size_t)b * 2 * p.Hb * W4, true, tid, T);
          __syncthreads();   // the copy and the step map cells to threads differently
          a.dofs = 0; a.sofs = 0;
          band_step<V, false, false, MODE, DT>(p, B, a, tid, T);
        } else {
          a.dofs = (size_t)n * slab + (size_t)b * p.Hb * W4;
          a.sofs = ((size_t)n * p.Q + b) * p.nwblk * V;
          band_step<V, false, true, MODE, DT>(p, B, a, tid, T);
        }
        cluster.sync();
        ph ^= 1;
      }
      if (MODE == WM_GRADIENT) {
        // CTA reduction of the squared residuals (deterministic order)
        __shared__ double red[32];
        double v = jacc;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[tid >> 5] = v;
        __syncthreads();
        if (tid == 0) {
          double t = 0.0;
          for (int w = 0; w < T / 32; ++w) t += red[w];
          p.Jpart[(size_t)pair * p.Q + b] = t;
        }
        __syncthreads();
      }
      if (MODE == WM_FORWARD) continue;

      // ---------------- adjoint sweep
      band_zero(p, B, tid, T);
      cluster.sync();
      ph = 0;
      if (p.K == 1) {
        for (int k = p.N; k >= 1; --k) {
          StepArgs a;
          a.ph = ph; a.t = k; a.slot = cid; a.pair = pair; a.s = s;
          a.src_task = -1; a.src_bit = 0; a.src_val = 0.f; a.record = false; a.Jacc = nullptr;
          a.dofs = (size_t)(k - 1) * slab + (size_t)b * p.Hb * W4;
          a.sofs = ((size_t)(k - 1) * p.Q + b) * p.nwblk * V;
          band_step<V, true, true, MODE, DT>(p, B, a, tid, T);
          cluster.sync();
          ph ^= 1;
        }
      } else {
        float *AS = p.AS + cid * p.ASslot + (size_t)b * 2 * p.Hb * W4;
        for (int j = p.nseg - 1; j >= 0; --j) {
          const int n0 = j * p.K, n1 = min(p.N, n0 + p.K);
          band_copy(p, B, ph, AS, true, tid, T);       // park mu^{k+1}, mu^{k+2}
          __syncthreads();
          band_copy(p, B, 0, p.CK + cid * p.CKslot + (size_t)j * 2 * slab +
                                 (size_t)b * 2 * p.Hb * W4, false, tid, T);
          cluster.sync();
          int fph = 0;
          for (int n = n0; n < n1; ++n) {              // recompute the segment
            StepArgs a;
            a.ph = fph; a.t = n; a.slot = cid; a.pair = pair; a.s = s;
            a.src_task = src_task; a.src_bit = src_bit; a.src_val = p.wavelet[n];
            a.record = false; a.Jacc = nullptr;
            a.dofs = (size_t)(n - n0) * slab + (size_t)b * p.Hb * W4;
            a.sofs = ((size_t)(n - n0) * p.Q + b) * p.nwblk * V;
            band_step<V, false, true, MODE, DT>(p, B, a, tid, T);
            cluster.sync();
            fph ^= 1;
          }
          band_copy(p, B, 0, AS, false, tid, T);       // restore the adjoint state
          ph = 0;
          cluster.sync();
          for (int k = n1; k > n0; --k) {
            StepArgs a;
            a.ph = ph; a.t = k; a.slot = cid; a.pair = pair; a.s = s;
            a.src_task = -1; a.src_bit = 0; a.src_val = 0.f; a.record = false; a.Jacc = nullptr;
            a.dofs = (size_t)(k - 1 - n0) * slab + (size_t)b * p.Hb * W4;
            a.sofs = ((size_t)(k - 1 - n0) * p.Q + b) * p.nwblk * V;
            band_step<V, true, true, MODE, DT>(p, B, a, tid, T);
            cluster.sync();
            ph ^= 1;
          }
        }
      }
    }
    if (MODE == WM_FORWARD) continue;
    // ---------------- gather the accumulator and fold onto the physical grid
    float *GP = p.GP + cid * p.GPslot;
    for (int q = tid; q < HW; q += T) {
      const int r = q / W4, x = q - r * W4;
      const int z = b * p.Hb + r;
      if (z < p.NZ && x < p.NX) GP[(size_t)z * p.NX + x] = B.Gm[q];
    }
    cluster.sync();
    const int rows = (p.nz + p.Q - 1) / p.Q;
    const int iz0 = b * rows, iz1 = min(p.nz, iz0 + rows);
    for (int q = tid; q < (iz1 - iz0) * p.nx; q += T) {
      const int iz = iz0 + q / p.nx, ix = q % p.nx;
      const int za = iz == 0 ? 0 : iz + p.nb;
      const int zb = iz == p.nz - 1 ? p.NZ - 1 : iz + p.nb;
      const int xa = ix == 0 ? 0 : ix + p.nb;
      const int xb = ix == p.nx - 1 ? p.NX - 1 : ix + p.nb;
      double acc = 0.0;
      for (int z = za; z <= zb; ++z)
        for (int x = xa; x <= xb; ++x) acc += (double)GP[(size_t)z * p.NX + x];
      const float vv = vp[(size_t)iz * p.nx + ix];
      const float val = (float)(acc * 2.0 / ((double)vv * (double)p.dx2));
      if (p.grad_atomic) p.GI[((size_t)item * p.nz + iz) * p.nx + ix] = val;
      else p.grad[((size_t)pp * p.nz + iz) * p.nx + ix] = val;
    }
    cluster.sync();
  }
  cluster.sync();
}

}  // namespace vip
