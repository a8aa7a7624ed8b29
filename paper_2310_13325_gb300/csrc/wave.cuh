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
// FP16 with a power-of-two scale per row of a task's 4 cells) and the adjoint pass reads it
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
  const unsigned long long *rmask; // [Q*ntask_pad] receivers in each thread task
  const int *rbase;      // [Q*ntask_pad] first entry in rperm
  const int *rperm;      // [R] receiver numbers in task order
  const int *rbstart;    // [Q+1] first rperm entry of each band
  const int *roff;       // [R] cell offset of each rperm entry within its band's level buffer
  int Rpad;              // receiver slots per band in shared memory
  // work decomposition
  int P, items, ipp, spi;
  int K, nseg;           // restart-checkpoint interval, segments
  // problem data
  const float *v;        // [P][nz][nx]
  const float *dobs;     // [S][R][N]
  const float *dseis;    // [P][S][R][N]
  float rho_scale;       // dx^2/sigma^2 (gradient) or dx^2 (adjoint)
  float *seis;           // [P][S][R][N]
  double *Jrec;          // [P*S][R] sum of squared residuals per receiver
  float *grad;           // [P][nz][nx]
  int grad_atomic;       // 1 when several work items share a particle: each
                         // item then writes its partial gradient to GI
  float *GI;             // [items][nz][nx] partial gradients (split items)
  int *status;           // bit 0: CFL violation; bit 1: non-finite velocity;
                         // bit 2: non-finite misfit
  int *work;             // next unclaimed work item, shared by every launch of a
                         // call (nullptr: cluster c takes items c, c + clusters, ...)
  // per-cluster scratch slots
  void *Dbuf;   size_t Dslot;    // snapshot elements per slot
  signed char *Dscale; size_t DSslot;  // FP16 scale exponents per slot (one per 4 cells)
  float *rho;   size_t rhoslot;  // [R][N] adjoint sources per slot
  float *GP;    size_t GPslot;   // [NZ][NX] gradient gather per slot
  float *CK;    size_t CKslot;   // restart checkpoints per slot
  float *AS;    size_t ASslot;   // parked adjoint state per slot
  // coefficients in global memory (kernels built with GW): w' and the
  // gradient accumulator per slot, [Q][Hb][NXg*4], so that the CTA's shared
  // memory holds only the two time levels and a taller band fits
  float *Wg;    size_t Wgslot;
  float *Gg;    size_t Ggslot;
};

// ---------------------------------------------------------------------------
// storage of the D snapshots
template <class DT> struct Snap;
template <> struct Snap<float> {
  static constexpr bool scaled = false;
  __device__ static void st(float *p, size_t i, float4 v, float) {
    __stcg(reinterpret_cast<float4 *>(p + i), v);
  }
  __device__ static float4 ld(const float *p, size_t i, float) {
    return __ldcg(reinterpret_cast<const float4 *>(p + i));
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
    uint2 u = __ldcg(reinterpret_cast<const uint2 *>(p + i));
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
    uint2 u = __ldcg(reinterpret_cast<const uint2 *>(p + i));
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

// Packed FP32 pairs (two cells per instruction, each lane rounded exactly as
// the scalar operation of the same name).
__device__ __forceinline__ unsigned long long pk(float2 a) {
  return *reinterpret_cast<unsigned long long *>(&a);
}
__device__ __forceinline__ float2 upk(unsigned long long r) {
  return *reinterpret_cast<float2 *>(&r);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
  return upk(r);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
  return upk(r);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
  return upk(r);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
  return upk(r);
}

// Laplacian bracket of the cell pair (j, j+1) from h[k], the sums of its
// left and right neighbours at distance k+1, and up[k], dn[k], its
// neighbours above and below; kN holds c_N in both lanes. Per lane the
// operations are those of lap_cell: 4u is exact, so fma(-4, u, x) rounds
// x - 4u exactly as the subtraction does.
__device__ __forceinline__ float2 lap_pair(float2 k1, float2 k2, float2 k3, float2 k4, float2 u,
                                           const float2 h[4], const float2 up[4],
                                           const float2 dn[4]) {
  const float2 m4 = make_float2(-4.f, -4.f);
  float2 s = mul2(k4, fma2(m4, u, add2(h[3], add2(up[3], dn[3]))));
  s = fma2(k3, fma2(m4, u, add2(h[2], add2(up[2], dn[2]))), s);
  s = fma2(k2, fma2(m4, u, add2(h[1], add2(up[1], dn[1]))), s);
  s = fma2(k1, fma2(m4, u, add2(h[0], add2(up[0], dn[0]))), s);
  return s;
}

// ---------------------------------------------------------------------------
// Batched persistent cluster kernel.
//
// Shared memory of a CTA (floats): the two time levels U[0], U[1] and the
// arrays W (w') and Gm (gradient accumulator) all use the row pitch PX, with
// the cells of a row at columns 4 .. 4+NXg*4-1, so one cell has the same
// offset in all four; a row of zeros; the row taper as (gz, gz) pairs; the
// column taper; the band's receiver numbers, cell offsets and two steps of
// receiver values.
struct Band {
  float *U[2];                 // local field buffers [Hb][PX]
  uint32_t sup[2], sdn[2];     // neighbours' buffers in the cluster window
  bool has_up, has_dn;         // whether the band has a neighbour above / below
  uint32_t szr;                // address of one row of zeros
  float *W;                    // [Hb][PX] w'
  float *Gm;                   // [Hb][PX] gradient accumulator
  float2 *gz2;                 // [Hb] (gz, gz) per row
  float *gxs;                  // [NXg*4]
  int *rid;                    // [Rpad] receiver numbers of this band (rperm order)
  int *roff;                   // [Rpad] their cell offsets in a level buffer
  float *val;                  // [2][Rpad] per-receiver values of two consecutive steps
  int rb0, nrb;                // first rperm entry and number of receivers of the band
  int b;
};

// 16-byte load from the cluster's shared-memory window (own CTA or a
// neighbour), 32-bit address.
__device__ __forceinline__ float4 ld_cluster4(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr));
  return v;
}

__device__ __forceinline__ uint32_t cluster_addr(uint32_t cta_addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(cta_addr), "r"(rank));
  return r;
}

// Split cluster barrier. A time step ends with step_fence(): the arrive
// publishes the step's shared-memory writes to the cluster, the CTA barrier
// makes them visible inside the CTA. The matching wait comes inside the next
// band_step, just before the first strip that reads a neighbouring band or
// overwrites rows a neighbour reads; the strips in between overlap the
// cluster barrier. A run of steps is closed with cluster_wait().
// A thread that wrote no row a neighbouring band reads (it updated inner
// strips only) arrives without release semantics: its writes are read
// inside the CTA only, which the CTA barrier orders.
__device__ __forceinline__ void cluster_arrive(bool release) {
  if (release) asm volatile("barrier.cluster.arrive.release;" ::: "memory");
  else asm volatile("barrier.cluster.arrive.relaxed;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ void step_fence(bool release = true) {
  cluster_arrive(release);
  __syncthreads();
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
  bool record;       // forward: record the current level at the receivers
  size_t dofs;       // element offset of this step's snapshot slab
  size_t sofs;       // offset of this step's scale slab (FP16: [Q][Hb][NXg] bytes)
  long long dnext;   // adjoint: element offset of the next step's slab (-1: none)
  int vnext_t;       // sample whose receiver values are fetched in this step (-1: none)
  int vnext_par;     // value slot they go to
  float *Jf;         // [4] squared residuals of the last few steps of the thread's
                     // receivers (FP32), one entry per receiver slot
};

// Receiver mask type of a task (4 bits per row).
template <int V> struct MaskT { using type = uint32_t; };
template <> struct MaskT<10> { using type = unsigned long long; };

// Per-task constants of one step.
struct TaskCtx {
  const float *cur;    // current level at (row r0, first cell of the task), own CTA
  const float2 *gz;    // (gz, gz) of row r0
  uint32_t top, tstr;  // cluster-window address of row r0-4 and row stride above the task
  uint32_t bot, bstr;  // same for row r0+V below the task
  bool tedge, bedge;   // rows above / below come from a neighbour or the zero row
  float2 gxa, gxb;     // column taper of the cell pairs (0,1) and (2,3)
  bool special;        // forward: holds the source; adjoint: holds receivers
  bool valid;
  int srow, slane;     // source row within the task (-1: none) and lane
  int rb;              // band-local index of the task's first receiver
};

// Add v to lane j of the cell quadruple held as the pairs (s01, s23).
__device__ __forceinline__ void add_lane(float2 &s01, float2 &s23, int j, float v) {
  if (j == 0) s01.x = __fadd_rn(s01.x, v);
  else if (j == 1) s01.y = __fadd_rn(s01.y, v);
  else if (j == 2) s23.x = __fadd_rn(s23.x, v);
  else s23.y = __fadd_rn(s23.y, v);
}

// The V rows of one task, 4 adjacent cells per row, top to bottom. Offsets
// (floats) from c.cur: dn to the next level, dW to w', dG to the gradient
// accumulator; PX is the row pitch of all four. With GW, w' and the
// accumulator are instead read from global memory at wg, gg (row r0 of the
// task, rows W4 apart), kAhead rows ahead of their use. The vertical stencil
// window of 9 rows lives in registers; each row loads one new window row, its
// left and right neighbour quadruples, w' and the previous value.
template <int V, bool ADJ, bool SNAP, int MODE, class DT, bool GW>
__device__ __forceinline__ void task_rows(const StepArgs &a, const TaskCtx &c,
                                          typename MaskT<V>::type rm, DT *Dtask,
                                          const DT *Dnext, const signed char *Stask,
                                          signed char *Sw,
                                          const float *vcur, int PX, int dn, int dW, int dG,
                                          const float *wg, float *gg, int W4, float2 k1,
                                          float2 k2, float2 k3, float2 k4, int tid) {
  using M = typename MaskT<V>::type;
  constexpr int kAhead = 3;      // rows between a global load and its use
  float4 wq[V], gq[V];
  if (GW) {
#pragma unroll
    for (int i = 0; i < kAhead && i < V; ++i) {
      wq[i] = ld4(wg + i * W4);
      if (ADJ && SNAP) gq[i] = __ldcg(reinterpret_cast<const float4 *>(gg + i * W4));
    }
  }
  // adjoint: snapshot rows are loaded kAhead rows ahead of their use
  float4 dq[V];
  float dinv[V];
  if (ADJ && SNAP) {
#pragma unroll
    for (int i = 0; i < kAhead && i < V; ++i) {
      dinv[i] = Snap<DT>::scaled ? __int_as_float((127 - Stask[i * (W4 >> 2)]) << 23) : 1.f;
      dq[i] = Snap<DT>::ld(Dtask, (size_t)i * W4, 1.f);
    }
  }
  float *cp = const_cast<float *>(c.cur);
  // window rows r0-4 .. r0+3; the four above the task come from the
  // neighbouring band (or the zero row) for the top strip
  float4 win[9];
#pragma unroll
  for (int j = 0; j < 4; ++j)
    win[j] = c.tedge ? ld_cluster4(c.top + (uint32_t)j * c.tstr) : ld4(cp + (j - 4) * PX);
#pragma unroll
  for (int j = 4; j < 8; ++j) win[j] = ld4(cp + (j - 4) * PX);
#pragma unroll
  for (int i = 0; i < V; ++i) {
    if (ADJ && SNAP && i + kAhead < V) {
      dinv[i + kAhead] =
          Snap<DT>::scaled ? __int_as_float((127 - Stask[(i + kAhead) * (W4 >> 2)]) << 23) : 1.f;
      dq[i + kAhead] = Snap<DT>::ld(Dtask, (size_t)(i + kAhead) * W4, 1.f);
    }
    if (GW && i + kAhead < V) {
      wq[i + kAhead] = ld4(wg + (i + kAhead) * W4);
      if (ADJ && SNAP) gq[i + kAhead] = __ldcg(reinterpret_cast<const float4 *>(gg + (i + kAhead) * W4));
    }
    float *rp = cp + i * PX;
    if (i + 4 < V)
      win[8] = ld4(rp + 4 * PX);
    else
      win[8] = c.bedge ? ld_cluster4(c.bot + (uint32_t)(i + 4 - V) * c.bstr) : ld4(rp + 4 * PX);
    const float4 Lf = ld4(rp - 4), Rf = ld4(rp + 4), C = win[4];
    // cell pairs (0,1) and (2,3). The horizontal neighbour sums at even
    // offsets pair aligned register pairs and take one packed add; those at odd
    // offsets are formed lane by lane (pairing them would need register moves)
    const float2 c01 = make_float2(C.x, C.y), c23 = make_float2(C.z, C.w);
    const float xs[12] = {Lf.x, Lf.y, Lf.z, Lf.w, C.x, C.y, C.z, C.w, Rf.x, Rf.y, Rf.z, Rf.w};
    float2 h01[4], h23[4], up01[4], dn01[4], up23[4], dn23[4];
#pragma unroll
    for (int d = 1; d <= 4; ++d) {
      if (d % 2 == 0) {
        h01[d - 1] = add2(make_float2(xs[4 - d], xs[5 - d]), make_float2(xs[4 + d], xs[5 + d]));
        h23[d - 1] = add2(make_float2(xs[6 - d], xs[7 - d]), make_float2(xs[6 + d], xs[7 + d]));
      } else {
        h01[d - 1] = make_float2(__fadd_rn(xs[4 - d], xs[4 + d]), __fadd_rn(xs[5 - d], xs[5 + d]));
        h23[d - 1] = make_float2(__fadd_rn(xs[6 - d], xs[6 + d]), __fadd_rn(xs[7 - d], xs[7 + d]));
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      up01[k] = make_float2(win[3 - k].x, win[3 - k].y);
      dn01[k] = make_float2(win[5 + k].x, win[5 + k].y);
      up23[k] = make_float2(win[3 - k].z, win[3 - k].w);
      dn23[k] = make_float2(win[5 + k].z, win[5 + k].w);
    }
    float2 s01 = lap_pair(k1, k2, k3, k4, c01, h01, up01, dn01);
    float2 s23 = lap_pair(k1, k2, k3, k4, c23, h23, up23, dn23);
    if (c.special) {
      if (!ADJ) {
        if (c.srow == i) add_lane(s01, s23, c.slane, a.src_val);
      } else if (MODE != WM_FORWARD) {
        const uint32_t rbits = (uint32_t)(rm >> (4 * i)) & 0xFu;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (rbits & (1u << j)) {
            const int lr = c.rb + __popcll((unsigned long long)(rm & (((M)1 << (4 * i + j)) - 1)));
            add_lane(s01, s23, j, vcur[lr]);
          }
        }
      }
    }
    const float4 Wv = GW ? wq[i] : ld4(rp + dW);
    const float4 AP = ld4(rp + dn);
    const float2 wa = make_float2(Wv.x, Wv.y), wb = make_float2(Wv.z, Wv.w);
    const float2 pa = make_float2(AP.x, AP.y), pb = make_float2(AP.z, AP.w);
    const float2 ta = fma2(wa, s01, add2(c01, c01));
    const float2 tb = fma2(wb, s23, add2(c23, c23));
    // g [2u + w s - g ap], as update_cell, on every cell: where the taper is
    // 1 this is exactly t - ap, and one code path without a per-row branch
    // runs faster than a separate taper-free path
    const float2 gz = c.gz[i];
    const float2 ga = mul2(gz, c.gxa), gb = mul2(gz, c.gxb);
    const float2 na = mul2(ga, fma2(make_float2(-ga.x, -ga.y), pa, ta));
    const float2 nb = mul2(gb, fma2(make_float2(-gb.x, -gb.y), pb, tb));
    if (c.valid) st4(rp + dn, make_float4(na.x, na.y, nb.x, nb.y));
    if (SNAP) {
      if (!ADJ) {
        const float4 sv = make_float4(s01.x, s01.y, s23.x, s23.y);
        float mul = 1.f;
        if (Snap<DT>::scaled) {
          // one power-of-two scale per row of the task's 4 cells: the largest
          // magnitude m and its binary exponent E (m = f 2^E, f in [0.5, 1):
          // E = exponent field - 126; non-negative floats order like their
          // bit patterns); the scale 2^(15 - E) brings the largest value just
          // below 2^15, clamped to 2^(+-120) (zero cells get scale 1, a
          // subnormal maximum the largest scale); its exponent is stored
          const float m = fmaxf(fmaxf(fabsf(sv.x), fabsf(sv.y)), fmaxf(fabsf(sv.z), fabsf(sv.w)));
          const unsigned mb = __float_as_uint(m);
          int e = mb ? 141 - (int)(mb >> 23) : 0;
          e = max(-120, min(120, e));
          mul = __int_as_float((e + 127) << 23);
          if (c.valid) Sw[i * (W4 >> 2)] = (signed char)e;
        }
        if (c.valid) Snap<DT>::st(Dtask, (size_t)i * W4, sv, mul);
      } else if (c.valid) {
        const float4 dv = dq[i];
        const float inv = dinv[i];
        float *gp = GW ? gg + i * W4 : rp + dG;
        const float4 gm = GW ? gq[i] : ld4(gp);
        float2 da = make_float2(dv.x, dv.y), db = make_float2(dv.z, dv.w);
        if (Snap<DT>::scaled) {
          da = mul2(da, make_float2(inv, inv));
          db = mul2(db, make_float2(inv, inv));
        }
        const float2 ga2 = fma2(na, da, make_float2(gm.x, gm.y));
        const float2 gb2 = fma2(nb, db, make_float2(gm.z, gm.w));
        if (GW) __stcg(reinterpret_cast<float4 *>(gp), make_float4(ga2.x, ga2.y, gb2.x, gb2.y));
        else st4(gp, make_float4(ga2.x, ga2.y, gb2.x, gb2.y));
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) win[k] = win[k + 1];
  }
}

// Forward sweep: the level a^t held in lev is trace sample t-1. Traces
// (forward modelling) or residuals against the observed sample, parked in
// value slot (t-1)&1 by the thread that reads it here (gradient). The
// residual r = d - d_obs and the adjoint source r dx^2/sigma^2 are rounded
// to FP32 once each; r^2 is summed per receiver in FP32 over a few steps
// (Jf[u] for the thread's u-th receiver) and then added to that receiver's
// FP64 accumulator by the caller. Each receiver belongs to one band and one
// thread of it, so its sum does not depend on the launch shape. The
// adjoint-only mode records nothing.
template <int MODE>
__device__ __forceinline__ void record_receivers(const WaveParams &p, const Band &B,
                                                 const float *lev, int t, int pair, int slot,
                                                 float *Jf, int tid, int T) {
  const float *vrec = B.val + ((t - 1) & 1) * p.Rpad;
#pragma unroll
  for (int u = 0; u < 4; ++u) {        // at most 4 receivers per thread (R <= 4 T)
    const int q = tid + u * T;
    if (q >= B.nrb) break;
    const int rr = B.rid[q];
    const float d = lev[B.roff[q]];
    if (MODE == WM_FORWARD) {
      p.seis[((size_t)pair * p.R + rr) * p.N + (t - 1)] = d;
    } else if (MODE == WM_GRADIENT) {
      const float res = __fsub_rn(d, vrec[q]);
      Jf[u] = __fmaf_rn(res, res, Jf[u]);
      p.rho[slot * p.rhoslot + (size_t)rr * p.N + (t - 1)] = __fmul_rn(res, p.rho_scale);
    }
  }
}

// Pull a contiguous range of snapshot elements towards L2 (bulk prefetch in
// 4 KB pieces, one per thread; only the 16-byte aligned interior).
template <class DT>
__device__ __forceinline__ void prefetch_slab_l2(const DT *p, size_t n, int tid, int T) {
  uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15;
  const uintptr_t e = (reinterpret_cast<uintptr_t>(p + n)) & ~(uintptr_t)15;
  if (e <= a) return;
  const size_t bytes = e - a;
  const size_t piece = 4096;
  for (size_t o = (size_t)tid * piece; o < bytes; o += (size_t)T * piece) {
    const uint32_t sz = (uint32_t)min(piece, bytes - o);
    asm volatile("{\n\t.reg .u64 g;\n\tcvta.to.global.u64 g, %0;\n\t"
                 "cp.async.bulk.prefetch.L2.global [g], %1;\n\t}" ::"l"(a + o), "r"(sz)
                 : "memory");
  }
}

// One time step of the band: every thread updates its tasks (4 adjacent
// cells x V rows). Tasks are numbered so that the strips away from the band
// edges come first: they touch no row a neighbouring band reads, so they run
// before the wait on the previous step's cluster barrier. The strips at the
// band edges follow the wait; their window rows beyond the band come from
// the neighbouring bands' shared memory (or the zero row at the grid edge).
// Returns whether the thread's warp reached the edge strips (its writes may
// be read by a neighbouring band).
template <int V, bool ADJ, bool SNAP, int MODE, class DT, bool GW>
__device__ __forceinline__ bool band_step(const WaveParams &p, const Band &B,
                                          const StepArgs &a, int tid, int T) {
  using M = typename MaskT<V>::type;
  const int Hb = p.Hb, PX = p.PX, NXg = p.NXg, W4 = NXg * 4;
  float *cur = a.ph ? B.U[1] : B.U[0];
  float *nxt = a.ph ? B.U[0] : B.U[1];
  const int dn = (int)(nxt - cur);
  const int dW = GW ? 0 : (int)(B.W - cur), dG = GW ? 0 : (int)(B.Gm - cur);
  // GW: this band's w' and accumulator in the cluster's slot
  const float *Wgb = GW ? p.Wg + a.slot * p.Wgslot + (size_t)B.b * Hb * W4 : nullptr;
  float *Ggb = GW ? p.Gg + a.slot * p.Ggslot + (size_t)B.b * Hb * W4 : nullptr;
  const uint32_t up_s = a.ph ? B.sup[1] : B.sup[0];
  const uint32_t dn_s = a.ph ? B.sdn[1] : B.sdn[0];
  const uint32_t rowb = (uint32_t)PX * 4u;
  DT *Dp = reinterpret_cast<DT *>(p.Dbuf) + a.slot * p.Dslot + a.dofs;
  const DT *Dn = a.dnext >= 0 ? reinterpret_cast<const DT *>(p.Dbuf) + a.slot * p.Dslot + a.dnext
                              : nullptr;
  signed char *Sp = Snap<DT>::scaled ? p.Dscale + a.slot * p.DSslot + a.sofs : nullptr;
  const float *vcur = B.val + (a.t & 1) * p.Rpad;
  if (!ADJ && a.record && a.t >= 1)
    record_receivers<MODE>(p, B, cur, a.t, a.pair, a.slot, a.Jf, tid, T);
  // receiver values of a later step are fetched now and parked in shared
  // memory at the end of this step, so no dependent global load sits on the
  // critical path of the receiver rows
  float vnext[4];
  const bool fetch = a.vnext_t >= 0;
  if (fetch) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = tid + u * T;
      if (q < B.nrb) {
        const int rr = B.rid[q];
        if (!ADJ)
          vnext[u] = __ldg(&p.dobs[((size_t)a.s * p.R + rr) * p.N + a.vnext_t]);
        else if (MODE == WM_GRADIENT)
          vnext[u] = p.rho[a.slot * p.rhoslot + (size_t)rr * p.N + a.vnext_t];
        else
          vnext[u] = __fmul_rn(p.rho_scale,
                               __ldg(&p.dseis[((size_t)a.pair * p.R + rr) * p.N + a.vnext_t]));
      }
    }
  }
  // adjoint: pull the band's snapshot slab of the next step towards L2
  if (ADJ && SNAP && Dn) prefetch_slab_l2(Dn, (size_t)Hb * W4, tid, T);
  const float2 k1 = make_float2(p.c1, p.c1), k2 = make_float2(p.c2, p.c2);
  const float2 k3 = make_float2(p.c3, p.c3), k4 = make_float2(p.c4, p.c4);
  const int nstrip = Hb / V;
  const int nin = (nstrip > 2 ? nstrip - 2 : 0) * NXg;   // tasks of the inner strips
  bool waited = false;
  for (int task0 = tid; task0 < p.ntask_pad; task0 += T) {
    // warp-uniform: the warp's 32 consecutive tasks reach the edge strips
    if (!waited && (task0 | 31) >= nin) {
      cluster_wait();
      waited = true;
    }
    TaskCtx c;
    c.valid = task0 < p.ntask;
    if (!c.valid) break;
    const int t = c.valid ? task0 : p.ntask - 1;
    int sp, cgp;
    if (t < nin) {
      sp = 1 + t / NXg;
      cgp = t - (sp - 1) * NXg;
    } else {
      const int e = t - nin;
      sp = e < NXg ? 0 : nstrip - 1;
      cgp = e < NXg ? e : e - NXg;
    }
    const int task = sp * NXg + cgp;   // row-major task number of the tables
    const int r0 = sp * V, gcol = cgp * 4;
    c.cur = cur + r0 * PX + gcol + 4;
    c.gz = B.gz2 + r0;
    const uint32_t colb = (uint32_t)(gcol + 4) * 4u;
    c.tedge = sp == 0;
    c.bedge = sp == nstrip - 1;
    c.top = B.has_up ? up_s + (uint32_t)(Hb - 4) * rowb + colb : B.szr + colb;
    c.tstr = B.has_up ? rowb : 0u;
    c.bot = B.has_dn ? dn_s + colb : B.szr + colb;
    c.bstr = B.has_dn ? rowb : 0u;
    const float4 gx4 = ld4(B.gxs + gcol);
    c.gxa = make_float2(gx4.x, gx4.y);
    c.gxb = make_float2(gx4.z, gx4.w);
    M rm = 0;
    c.rb = 0;
    c.srow = -1;
    c.slane = 0;
    c.special = false;
    if (!ADJ) {
      if (c.valid && task == a.src_task) {
        c.srow = a.src_bit >> 2;
        c.slane = a.src_bit & 3;
        c.special = true;
      }
    } else if (MODE != WM_FORWARD) {
      rm = c.valid ? (M)__ldg(&p.rmask[B.b * p.ntask_pad + task]) : (M)0;
      c.special = rm != 0;
      if (c.special) c.rb = __ldg(&p.rbase[B.b * p.ntask_pad + task]) - B.rb0;   // band-local
    }
    const size_t toff = (size_t)r0 * W4 + gcol;
    DT *Dt = Dp + toff;
    const DT *Dnt = Dn ? Dn + toff : nullptr;
    // FP16 scale exponents of the task's rows: one byte per row of its 4 cells
    const signed char *St = Sp ? Sp + (size_t)r0 * NXg + cgp : nullptr;
    signed char *Sw = Sp ? Sp + (size_t)r0 * NXg + cgp : nullptr;
    task_rows<V, ADJ, SNAP, MODE, DT, GW>(a, c, rm, Dt, Dnt, St, Sw, vcur, PX, dn, dW, dG,
                                          GW ? Wgb + toff : nullptr,
                                          (GW && ADJ) ? Ggb + toff : nullptr, W4, k1, k2, k3,
                                          k4, tid);
  }
  const bool edge = waited;
  if (!waited) cluster_wait();
  if (fetch) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (tid + u * T < B.nrb) B.val[a.vnext_par * p.Rpad + tid + u * T] = vnext[u];
  }
  return edge;
}

// Value used at the receivers in the first step of an adjoint sweep (before
// the per-step fetch takes over): the adjoint source at sample t, into slot
// par.
template <int MODE>
__device__ __forceinline__ void receiver_values(const WaveParams &p, const Band &B, int tid,
                                                int slot, int pair, int t, int par) {
  for (int q = tid; q < B.nrb; q += blockDim.x) {
    const int rr = B.rid[q];
    float v;
    if (MODE == WM_GRADIENT)
      v = p.rho[slot * p.rhoslot + (size_t)rr * p.N + t];
    else
      v = __fmul_rn(p.rho_scale, p.dseis[((size_t)pair * p.R + rr) * p.N + t]);
    B.val[par * p.Rpad + q] = v;
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

// Threads per CTA allowed for V rows per thread. The register file of an SM
// is split over its 4 schedulers (16384 registers each), so 16, 14 and 12
// warps leave 128, 128 and 168 registers per thread. The global-coefficient
// kernels keep two rows of w' and of the accumulator in flight and take 12.
template <int V, bool GW = false> struct WaveMaxThreads {
  static constexpr int value = (V >= 10 || GW) ? 384 : (V >= 8 ? 448 : 512);
};

template <int V, int MODE, class DT, bool GW>
__global__ void __launch_bounds__(WaveMaxThreads<V, GW>::value, 1)
    wave_cluster_kernel(const __grid_constant__ WaveParams p) {
  cg::cluster_group cluster = cg::this_cluster();
  const int b = (int)cluster.block_rank();
  const int cid = blockIdx.x / p.Q;
  const int ncl = gridDim.x / p.Q;
  const int tid = threadIdx.x, T = blockDim.x;
  extern __shared__ __align__(16) float smem[];
  const int HP = p.Hb * p.PX;
  const int W4 = p.NXg * 4;
  const int HW = p.Hb * W4;
  Band B;
  B.b = b;
  B.U[0] = smem;
  B.U[1] = smem + HP;
  float *Zr = smem + 2 * HP;
  B.W = GW ? nullptr : Zr + p.PX;
  B.Gm = GW ? nullptr : B.W + HP;
  B.gz2 = reinterpret_cast<float2 *>(GW ? Zr + p.PX : B.Gm + (MODE != WM_FORWARD ? HP : 0));
  B.gxs = reinterpret_cast<float *>(B.gz2) + ((2 * p.Hb + 3) & ~3);
  B.rid = reinterpret_cast<int *>(B.gxs + W4);
  B.roff = B.rid + p.Rpad;
  B.val = reinterpret_cast<float *>(B.roff + p.Rpad);
  B.rb0 = p.rbstart[b];
  B.nrb = p.rbstart[b + 1] - B.rb0;
  for (int q = tid; q < B.nrb; q += T) {
    B.rid[q] = p.rperm[B.rb0 + q];
    B.roff[q] = p.roff[B.rb0 + q];
  }
  B.szr = (uint32_t)__cvta_generic_to_shared(Zr);
  B.has_up = b > 0;
  B.has_dn = b < p.Q - 1;
  for (int ph = 0; ph < 2; ++ph) {
    const uint32_t su = (uint32_t)__cvta_generic_to_shared(B.U[ph]);
    B.sup[ph] = B.has_up ? cluster_addr(su, (uint32_t)(b - 1)) : 0u;
    B.sdn[ph] = B.has_dn ? cluster_addr(su, (uint32_t)(b + 1)) : 0u;
  }
  for (int q = tid; q < p.PX; q += T) Zr[q] = 0.f;
  for (int q = tid; q < p.Hb; q += T) {
    const float g = p.gz[b * p.Hb + q];
    B.gz2[q] = make_float2(g, g);
  }
  for (int q = tid; q < W4; q += T) B.gxs[q] = p.gx[q];
  const size_t slab = (size_t)p.Q * HW;   // elements of one snapshot

  // Work items: with a shared counter (several launches of one call draw from
  // it) the cluster's first thread claims the next item and the other CTAs
  // read it from that CTA's shared memory after a cluster barrier; every item
  // ends with a cluster barrier, so the next claim cannot overwrite a value a
  // CTA has not read yet.
  __shared__ int claimed;
  auto next_item = [&](int prev) -> int {
    if (!p.work) return prev < 0 ? cid : prev + ncl;
    if (b == 0 && tid == 0) claimed = atomicAdd(p.work, 1);
    cluster.sync();
    return *cluster.map_shared_rank(&claimed, 0);
  };
  for (int item = next_item(-1); item < p.items; item = next_item(item)) {
    const int pp = item / p.ipp;
    const int s0 = (item - pp * p.ipp) * p.spi;
    const int s1 = min(p.S, s0 + p.spi);
    // model coefficients w' = (vpad dt/dx)^2 of this band; CFL check
    const float *vp = p.v + (size_t)pp * p.nz * p.nx;
    bool cfl_bad = false, nonfinite = false;
    for (int q = tid; q < HW; q += T) {
      const int r = q / W4, x = q - r * W4;
      const int z = b * p.Hb + r;
      float w = 0.f;
      if (z < p.NZ && x < p.NX) {
        const int iz = min(max(z - p.nb, 0), p.nz - 1);
        const int ix = min(max(x - p.nb, 0), p.nx - 1);
        const float vv = vp[(size_t)iz * p.nx + ix];
        const float c = __fmul_rn(vv, p.dtdx);
        w = __fmul_rn(c, c);
        cfl_bad |= !(w <= p.w_cfl);
        nonfinite |= !isfinite(vv);
      }
      if (GW) {
        p.Wg[(size_t)cid * p.Wgslot + (size_t)b * HW + q] = w;
        if (MODE != WM_FORWARD) p.Gg[(size_t)cid * p.Ggslot + (size_t)b * HW + q] = 0.f;
      } else {
        B.W[r * p.PX + 4 + x] = w;
        if (MODE != WM_FORWARD) B.Gm[r * p.PX + 4 + x] = 0.f;
      }
    }
    if (cfl_bad) atomicOr(p.status, 1);
    if (nonfinite) atomicOr(p.status, 2);

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
      step_fence();
      double jacc[4] = {0.0, 0.0, 0.0, 0.0};
      float jf[4] = {0.f, 0.f, 0.f, 0.f};
      int ph = 0;
      bool edge;
      for (int n = 0; n < p.N; ++n) {
        StepArgs a;
        a.ph = ph; a.t = n; a.slot = cid; a.pair = pair; a.s = s;
        a.src_task = src_task; a.src_bit = src_bit; a.src_val = __ldg(&p.wavelet[n]);
        a.record = MODE != WM_ADJOINT; a.Jf = jf; a.dnext = -1;
        a.vnext_t = MODE == WM_GRADIENT ? n : -1;
        a.vnext_par = n & 1;
        if (MODE == WM_FORWARD || p.K > 1) {
          if (MODE != WM_FORWARD && n % p.K == 0) {
            band_copy(p, B, ph, p.CK + cid * p.CKslot + (size_t)(n / p.K) * 2 * slab +
                                    (size_t)b * 2 * HW, true, tid, T);
            __syncthreads();   // the copy and the step map cells to threads differently
          }
          a.dofs = 0; a.sofs = 0;
          edge = band_step<V, false, false, MODE, DT, GW>(p, B, a, tid, T);
        } else {
          a.dofs = (size_t)n * slab + (size_t)b * HW;
          a.sofs = ((size_t)n * p.Q + b) * p.Hb * p.NXg;
          edge = band_step<V, false, true, MODE, DT, GW>(p, B, a, tid, T);
        }
        step_fence(edge);
        ph ^= 1;
        if ((n & 15) == 15) {
#pragma unroll
          for (int u = 0; u < 4; ++u) { jacc[u] += (double)jf[u]; jf[u] = 0.f; }
        }
      }
      // the last level a^N is trace sample N-1
      if (MODE != WM_ADJOINT)
        record_receivers<MODE>(p, B, ph ? B.U[1] : B.U[0], p.N, pair, cid, jf, tid, T);
      cluster_wait();
      if (MODE == WM_GRADIENT) {
        // per-receiver sums of squared residuals (FP64)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = tid + u * T;
          if (q < B.nrb) p.Jrec[(size_t)pair * p.R + B.rid[q]] = jacc[u] + (double)jf[u];
        }
      }
      // every thread has read the last level before the next sweep zeroes it
      __syncthreads();
      if (MODE == WM_FORWARD) continue;

      // ---------------- adjoint sweep
      band_zero(p, B, tid, T);
      ph = 0;
      if (p.K == 1) {
        receiver_values<MODE>(p, B, tid, cid, pair, p.N - 1, p.N & 1);
        step_fence();
        for (int k = p.N; k >= 1; --k) {
          StepArgs a;
          a.ph = ph; a.t = k; a.slot = cid; a.pair = pair; a.s = s;
          a.src_task = -1; a.src_bit = 0; a.src_val = 0.f; a.record = false; a.Jf = nullptr;
          a.dofs = (size_t)(k - 1) * slab + (size_t)b * HW;
          a.sofs = ((size_t)(k - 1) * p.Q + b) * p.Hb * p.NXg;
          a.dnext = k >= 2 ? (long long)((size_t)(k - 2) * slab + (size_t)b * HW) : -1;
          a.vnext_t = k >= 2 ? k - 2 : -1;
          a.vnext_par = (k - 1) & 1;
          step_fence(band_step<V, true, true, MODE, DT, GW>(p, B, a, tid, T));
          ph ^= 1;
        }
        cluster_wait();
      } else {
        float *AS = p.AS + cid * p.ASslot + (size_t)b * 2 * HW;
        step_fence();
        cluster_wait();
        for (int j = p.nseg - 1; j >= 0; --j) {
          const int n0 = j * p.K, n1 = min(p.N, n0 + p.K);
          band_copy(p, B, ph, AS, true, tid, T);       // park mu^{k+1}, mu^{k+2}
          __syncthreads();
          band_copy(p, B, 0, p.CK + cid * p.CKslot + (size_t)j * 2 * slab + (size_t)b * 2 * HW,
                    false, tid, T);
          step_fence();
          int fph = 0;
          for (int n = n0; n < n1; ++n) {              // recompute the segment
            StepArgs a;
            a.ph = fph; a.t = n; a.slot = cid; a.pair = pair; a.s = s;
            a.src_task = src_task; a.src_bit = src_bit; a.src_val = __ldg(&p.wavelet[n]);
            a.record = false; a.Jf = nullptr; a.dnext = -1; a.vnext_t = -1; a.vnext_par = 0;
            a.dofs = (size_t)(n - n0) * slab + (size_t)b * HW;
            a.sofs = ((size_t)(n - n0) * p.Q + b) * p.Hb * p.NXg;
            step_fence(band_step<V, false, true, MODE, DT, GW>(p, B, a, tid, T));
            fph ^= 1;
          }
          cluster_wait();
          band_copy(p, B, 0, AS, false, tid, T);       // restore the adjoint state
          receiver_values<MODE>(p, B, tid, cid, pair, n1 - 1, n1 & 1);
          ph = 0;
          step_fence();
          for (int k = n1; k > n0; --k) {
            StepArgs a;
            a.ph = ph; a.t = k; a.slot = cid; a.pair = pair; a.s = s;
            a.src_task = -1; a.src_bit = 0; a.src_val = 0.f; a.record = false; a.Jf = nullptr;
            a.dofs = (size_t)(k - 1 - n0) * slab + (size_t)b * HW;
            a.sofs = ((size_t)(k - 1 - n0) * p.Q + b) * p.Hb * p.NXg;
            a.dnext = k - 2 >= n0 ? (long long)((size_t)(k - 2 - n0) * slab + (size_t)b * HW)
                                  : -1;
            a.vnext_t = k - 1 > n0 ? k - 2 : -1;
            a.vnext_par = (k - 1) & 1;
            step_fence(band_step<V, true, true, MODE, DT, GW>(p, B, a, tid, T));
            ph ^= 1;
          }
          cluster_wait();
        }
      }
    }
    if (MODE == WM_FORWARD) continue;
    // ---------------- gather the accumulator and fold onto the physical grid
    // (GW: the accumulator already sits in global memory, rows W4 apart)
    float *GP = GW ? p.Gg + cid * p.Ggslot : p.GP + cid * p.GPslot;
    const int gpitch = GW ? W4 : p.NX;
    if (!GW) {
      for (int q = tid; q < HW; q += T) {
        const int r = q / W4, x = q - r * W4;
        const int z = b * p.Hb + r;
        if (z < p.NZ && x < p.NX) GP[(size_t)z * p.NX + x] = B.Gm[r * p.PX + 4 + x];
      }
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
        for (int x = xa; x <= xb; ++x) acc += (double)GP[(size_t)z * gpitch + x];
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
