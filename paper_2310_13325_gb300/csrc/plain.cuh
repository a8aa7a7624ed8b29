// Plain per-step kernels (FWI_MODE_PLAIN), used only by fwi.cu.
#pragma once
#include "wave.cuh"

namespace vip {

// ---------------------------------------------------------------------------
// Plain per-step kernels: one cell per thread, fields in global memory.
struct PlainParams {
  int NZ, NX, N, R;
  float c1, c2, c3, c4;
  const float *gz, *gx;     // [NZ], [NX]
  const float *W;           // [NZ][NX] w'
  const int *recmap;        // [NZ][NX] receiver number or -1
};

__device__ __forceinline__ float gld(const float *a, int z, int x, int NZ, int NX) {
  return (z >= 0 && z < NZ && x >= 0 && x < NX) ? a[(size_t)z * NX + x] : 0.f;
}

// Forward step n: nxt <- a^{n+1} from cur = a^n and nxt = a^{n-1}; optional
// snapshot D^{n+1}; records traces (seis) or residuals (rho, J).
__global__ void plain_fwd_step(PlainParams q, const float *__restrict__ cur, float *nxt,
                               int n, int sz, int sx, float fval, float *D,
                               float *seis, const float *dobs_s, float *rho,
                               float rho_scale, double *J) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= q.NZ * q.NX) return;
  const int z = idx / q.NX, x = idx - z * q.NX;
  float h[8], vv[8];
  for (int k = 0; k < 4; ++k) {
    h[k] = gld(cur, z, x - 4 + k, q.NZ, q.NX);
    h[4 + k] = gld(cur, z, x + 1 + k, q.NZ, q.NX);
    vv[k] = gld(cur, z - 4 + k, x, q.NZ, q.NX);
    vv[4 + k] = gld(cur, z + 1 + k, x, q.NZ, q.NX);
  }
  const float u = cur[idx];
  WaveParams wp;
  wp.c1 = q.c1; wp.c2 = q.c2; wp.c3 = q.c3; wp.c4 = q.c4;
  float s = lap_cell(wp, u, h, vv);
  if (z == sz && x == sx) s = __fadd_rn(s, fval);
  if (D) D[idx] = s;
  const float an = update_cell(__fmul_rn(q.gz[z], q.gx[x]), q.W[idx], s, u, nxt[idx]);
  nxt[idx] = an;
  const int r = q.recmap[idx];
  if (r >= 0) {
    if (seis) seis[(size_t)r * q.N + n] = an;
    if (rho) {
      const float res = __fsub_rn(an, dobs_s[(size_t)r * q.N + n]);
      rho[(size_t)r * q.N + n] = __fmul_rn(res, rho_scale);
      atomicAdd(J, (double)res * (double)res);
    }
  }
}

// Adjoint step k: nxt <- mu^k from cur = mu^{k+1} and nxt = mu^{k+2};
// injects the residual sources and accumulates Gm += mu^k D^k.
__global__ void plain_adj_step(PlainParams q, const float *__restrict__ cur, float *nxt,
                               int k, const float *rho, float rho_mul,
                               const float *D, float *Gm) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= q.NZ * q.NX) return;
  const int z = idx / q.NX, x = idx - z * q.NX;
  float h[8], vv[8];
  for (int kk = 0; kk < 4; ++kk) {
    h[kk] = gld(cur, z, x - 4 + kk, q.NZ, q.NX);
    h[4 + kk] = gld(cur, z, x + 1 + kk, q.NZ, q.NX);
    vv[kk] = gld(cur, z - 4 + kk, x, q.NZ, q.NX);
    vv[4 + kk] = gld(cur, z + 1 + kk, x, q.NZ, q.NX);
  }
  const float u = cur[idx];
  WaveParams wp;
  wp.c1 = q.c1; wp.c2 = q.c2; wp.c3 = q.c3; wp.c4 = q.c4;
  float s = lap_cell(wp, u, h, vv);
  const int r = q.recmap[idx];
  if (r >= 0) {
    float val = rho[(size_t)r * q.N + (k - 1)];
    if (rho_mul != 1.f) val = __fmul_rn(rho_mul, val);
    s = __fadd_rn(s, val);
  }
  const float an = update_cell(__fmul_rn(q.gz[z], q.gx[x]), q.W[idx], s, u, nxt[idx]);
  nxt[idx] = an;
  Gm[idx] = __fmaf_rn(an, D[idx], Gm[idx]);
}

}  // namespace vip
