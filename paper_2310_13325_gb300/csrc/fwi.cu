// Host side of the FWI entry points: context, launch planning, autotuning,
// CUDA-graph replay of the batched path and the plain per-step path.
#include "wave_inst.cuh"
#include "plain.cuh"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <tuple>
#include <vector>

namespace vip {

static thread_local char g_last_error[512] = "";

void note_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
  if (g_last_error[0] == 0)
    snprintf(g_last_error, sizeof g_last_error, "%s: %s (%s:%d)", what,
             cudaGetErrorString(e), file, line);
}

static const double kC8[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0,
                              -1.0 / 560.0};
// Largest stable Courant number of the 2-D 8th-order leapfrog scheme:
// (v dt/dx)^2 * 2 * |c0 + 2 sum_k c_k (-1)^k| <= 4.
static double cfl_w_limit() {
  double s = kC8[0];
  for (int k = 1; k <= 4; ++k) s += 2.0 * kC8[k] * ((k & 1) ? -1.0 : 1.0);
  return 4.0 / (2.0 * std::fabs(s));
}

struct Plan {
  int Q = 0, V = 0, T = 0, Hb = 0, NXg = 0, PX = 0, ntask = 0, ntask_pad = 0, nwblk = 0;
  size_t smem = 0;
  int maxcl = 0, ncl = 0;
  int K = 1, nseg = 1;
  int items = 0, ipp = 1, spi = 1;
  size_t Dslot = 0, DSslot = 0, rhoslot = 0, GPslot = 0, CKslot = 0, ASslot = 0;
  size_t Wgslot = 0, Ggslot = 0;
  bool gw = false;   // w' and the accumulator in global memory
  size_t slot_bytes = 0, total_bytes = 0;
  int mode = 0, dtype = 0;
  double est = 0;
};

struct Tables {
  int Q, V, Hb, NXg, ntask_pad;
  float *gz = nullptr, *gx = nullptr;
  unsigned long long *rmask = nullptr;
  int *rbase = nullptr, *rperm = nullptr, *rbstart = nullptr, *roff = nullptr;
  int rmax = 0;   // largest number of receivers in one band
};

constexpr int kGraphKeyLen = 18;
struct GraphEntry {
  std::array<uintptr_t, kGraphKeyLen> key;
  cudaGraphExec_t exec;
};

}  // namespace vip

using namespace vip;

struct fwi_ctx {
  int nz, nx, nb, NZ, NX, N, S, R;
  float dx, dt, alpha, f0, t0;
  std::vector<int> src_z, src_x, rec_z, rec_x;   // padded indices
  size_t ws_limit = 0;
  int mode = FWI_MODE_BATCHED, ckpt = 1, autotune = 0;
  int device = 0, sm_count = 0;
  size_t smem_optin = 0;
  float *d_wavelet = nullptr;
  int *d_src_z = nullptr, *d_src_x = nullptr, *d_status = nullptr;
  std::vector<Tables> tables;
  void *scratch = nullptr;
  size_t scratch_bytes = 0;
  std::vector<GraphEntry> graphs;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t last_stream = nullptr;
  std::map<std::tuple<int, int, int>, std::array<int, 4>> tuned;   // (P, mode*16+dtype, S) -> Q,V,T,gw
  std::set<std::tuple<int, int, int>> untunable;   // keys whose trials all exceeded the budget
  int force_Q = 0, force_V = 0, force_T = 0, force_spi = 0;          // launch override
  int force_coeff = 0;   // 0 any, 1 coefficients in shared memory, 2 in global memory
  int use_graphs = 1;   // VIPGB_GRAPHS=0 in the environment: eager launches
  int fill = 1;         // second launch on the SMs the main launch leaves idle
  cudaStream_t fill_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int prio_hi = 0, prio_lo = 0;
  size_t need_bytes = 0;   // device bytes the last planned call needs (or lacked)
  // plain-mode buffers
  float *pl_W = nullptr, *pl_a = nullptr, *pl_Gm = nullptr, *pl_gz = nullptr, *pl_gx = nullptr;
  int *pl_recmap = nullptr;
  bool pl_ready = false;   // every plain-mode buffer allocated and filled
  // source minibatches (fwi_gradient_sources): the chosen sources' positions
  // and observed traces, gathered in front of a call, sized for all sources
  int *d_sub_z = nullptr, *d_sub_x = nullptr;
  float *d_sub_dobs = nullptr;
  double *pl_J = nullptr;
};

namespace vip {

static const void *kernel_ptr(int V, int mode, int dtype, bool gw) {
  if (mode == WM_FORWARD) return wave_kernel_f32(V, mode, gw);
  if (dtype == FWI_FP32) return wave_kernel_f32(V, mode, gw);
  if (dtype == FWI_CKPT_BF16) return wave_kernel_bf16(V, mode, gw);
  if (dtype == FWI_CKPT_FP16) return wave_kernel_f16(V, mode, gw);
  return nullptr;
}

static size_t dtype_size(int dtype) { return dtype == FWI_FP32 ? 4 : 2; }

static int band_height(int NZ, int Q, int V) {
  const int h = idiv_up(NZ, Q);
  return idiv_up(h, V) * V;
}

static int receiver_pad(int R) { return (R + 3) & ~3; }

// Shared memory of the batched kernel (floats): two levels, the zero row, w'
// and (gradient) the accumulator, all [Hb][PX] (w' and the accumulator are
// left out when they live in global memory, gw); (gz, gz) per row; the
// column taper; receiver numbers, cell offsets and two value slots.
static size_t wave_smem(int Hb, int V, int PX, int NXg, bool grad, int R, bool gw) {
  const size_t HP = (size_t)Hb * PX;
  size_t f = (gw ? 2 : (grad ? 4 : 3)) * HP + PX + ((2 * Hb + 3) & ~3) + (size_t)NXg * 4 +
             4 * (size_t)receiver_pad(R);
  return f * 4;
}

static int get_tables(fwi_ctx *c, int Q, int V, Tables **out) {
  for (auto &t : c->tables)
    if (t.Q == Q && t.V == V) { *out = &t; return VIP_OK; }
  Tables t;
  t.Q = Q; t.V = V;
  t.Hb = band_height(c->NZ, Q, V);
  t.NXg = idiv_up(c->NX, 4);
  const int ntask = (t.Hb / V) * t.NXg;
  t.ntask_pad = idiv_up(ntask, 32) * 32;
  std::vector<float> gz((size_t)Q * t.Hb, 0.f), gx((size_t)t.NXg * 4, 0.f);
  auto prof = [&](int i, int n) {
    const int into = std::max(std::max(c->nb - i, i - (n - 1 - c->nb)), 0);
    const double a = c->alpha * into;
    return (float)std::exp(-a * a);
  };
  for (int z = 0; z < c->NZ; ++z) gz[z] = prof(z, c->NZ);
  for (int x = 0; x < c->NX; ++x) gx[x] = prof(x, c->NX);
  std::vector<unsigned long long> mask((size_t)Q * t.ntask_pad, 0ull);
  std::vector<int> base((size_t)Q * t.ntask_pad, 0), perm(std::max(c->R, 1), 0);
  std::vector<std::array<long, 2>> order(c->R);
  for (int r = 0; r < c->R; ++r) {
    const int z = c->rec_z[r], x = c->rec_x[r];
    const int b = z / t.Hb, rr = z - b * t.Hb;
    const int task = (rr / V) * t.NXg + x / 4;
    const int bit = (rr % V) * 4 + (x & 3);
    order[r] = {((long)b * t.ntask_pad + task) * 64 + bit, r};
  }
  std::sort(order.begin(), order.end());
  // cell offset of each receiver in its band's level buffer (row pitch PX,
  // cells from column 4)
  const int PX = 4 * (t.NXg + 2);
  std::vector<int> roff(std::max(c->R, 1), 0);
  for (int i = 0; i < c->R; ++i) {
    const long key = order[i][0];
    const long bt = key / 64;
    const int bit = (int)(key % 64);
    if (mask[bt] == 0) base[bt] = i;
    mask[bt] |= 1ull << bit;
    const int r = (int)order[i][1];
    perm[i] = r;
    roff[i] = (c->rec_z[r] % t.Hb) * PX + 4 + c->rec_x[r];
  }
  std::vector<int> bstart(Q + 1, 0);
  for (int i = 0; i < c->R; ++i) bstart[order[i][0] / 64 / t.ntask_pad + 1]++;
  for (int b = 0; b < Q; ++b) {
    t.rmax = std::max(t.rmax, bstart[b + 1]);
    bstart[b + 1] += bstart[b];
  }
  // device copies, all or none (a failure part way frees what was made)
  auto upload = [&]() -> int {
    VIP_TRY(cudaMalloc(&t.gz, gz.size() * 4));
    VIP_TRY(cudaMalloc(&t.gx, gx.size() * 4));
    VIP_TRY(cudaMalloc(&t.rmask, mask.size() * 8));
    VIP_TRY(cudaMalloc(&t.rbase, base.size() * 4));
    VIP_TRY(cudaMalloc(&t.rperm, perm.size() * 4));
    VIP_TRY(cudaMalloc(&t.roff, roff.size() * 4));
    VIP_TRY(cudaMalloc(&t.rbstart, bstart.size() * 4));
    VIP_TRY(cudaMemcpy(t.rbstart, bstart.data(), bstart.size() * 4, cudaMemcpyHostToDevice));
    VIP_TRY(cudaMemcpy(t.gz, gz.data(), gz.size() * 4, cudaMemcpyHostToDevice));
    VIP_TRY(cudaMemcpy(t.gx, gx.data(), gx.size() * 4, cudaMemcpyHostToDevice));
    VIP_TRY(cudaMemcpy(t.rmask, mask.data(), mask.size() * 8, cudaMemcpyHostToDevice));
    VIP_TRY(cudaMemcpy(t.rbase, base.data(), base.size() * 4, cudaMemcpyHostToDevice));
    VIP_TRY(cudaMemcpy(t.rperm, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice));
    VIP_TRY(cudaMemcpy(t.roff, roff.data(), roff.size() * 4, cudaMemcpyHostToDevice));
    return VIP_OK;
  };
  if (const int rc = upload()) {
    cudaFree(t.gz); cudaFree(t.gx); cudaFree(t.rmask); cudaFree(t.rbase); cudaFree(t.rperm);
    cudaFree(t.roff); cudaFree(t.rbstart);
    return rc;
  }
  c->tables.push_back(t);
  *out = &c->tables.back();
  return VIP_OK;
}

static size_t free_budget(fwi_ctx *c) {
  if (c->ws_limit) return c->ws_limit;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return 0;
  return (size_t)(0.85 * (double)(fr + c->scratch_bytes));
}

// Fill the memory fields of a plan for its (ncl, K); returns total bytes.
static void plan_memory(const fwi_ctx *c, Plan &pl, int P) {
  const size_t W4 = (size_t)pl.NXg * 4;
  const size_t slab = (size_t)pl.Q * pl.Hb * W4;
  const bool grad = pl.mode != WM_FORWARD;
  pl.Dslot = pl.DSslot = pl.rhoslot = pl.GPslot = pl.CKslot = pl.ASslot = 0;
  pl.Wgslot = pl.gw ? slab : 0;
  pl.Ggslot = (pl.gw && grad) ? slab : 0;
  if (grad) {
    const int steps = pl.K == 1 ? c->N : pl.K;
    pl.Dslot = (size_t)steps * slab;
    // FP16: one scale exponent (a byte) per row of 4 cells
    if (pl.dtype == FWI_CKPT_FP16) pl.DSslot = (size_t)steps * pl.Q * pl.Hb * pl.NXg;
    pl.GPslot = pl.gw ? 0 : (size_t)c->NZ * c->NX;   // gw: the fold reads the accumulator
    if (pl.mode == WM_GRADIENT) pl.rhoslot = (size_t)c->R * c->N;
    if (pl.K > 1) {
      pl.nseg = idiv_up(c->N, pl.K);
      pl.CKslot = (size_t)pl.nseg * 2 * slab;
      pl.ASslot = 2 * slab;
    } else {
      pl.nseg = 1;
    }
  }
  // keep every slot 256-byte aligned
  auto a = [](size_t n, size_t es) { return align_up(n * es, 256); };
  pl.slot_bytes = a(pl.Dslot, dtype_size(pl.dtype)) + a(pl.DSslot, 1) + a(pl.rhoslot, 4) +
                  a(pl.GPslot, 4) + a(pl.CKslot, 4) + a(pl.ASslot, 4) + a(pl.Wgslot, 4) +
                  a(pl.Ggslot, 4);
  const size_t gi = (pl.mode != WM_FORWARD && pl.ipp > 1)
                        ? align_up((size_t)P * pl.ipp * c->nz * c->nx * 4, 256) : 0;
  pl.total_bytes = 256 + align_up((size_t)P * c->S * c->R * 8, 256) + gi +
                   (size_t)pl.ncl * pl.slot_bytes;
}

// Launch attributes of a wave kernel: the dynamic shared-memory cap is set to
// the most the device allows (less the kernel's static shared memory) and
// clusters beyond 8 CTAs are allowed, once and to the same values whatever the
// plan. A launch then carries its own dynamic size, and nothing a later plan
// or candidate enumeration does can change what a captured graph's kernel node
// was instantiated with.
static int set_wave_attrs(fwi_ctx *c, const void *fn) {
  cudaFuncAttributes fa;
  VIP_TRY(cudaFuncGetAttributes(&fa, fn));
  const int cap = (int)(c->smem_optin - fa.sharedSizeBytes);
  if (fa.maxDynamicSharedSizeBytes != cap)
    VIP_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
  VIP_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  return VIP_OK;
}

static int make_candidates(fwi_ctx *c, int P, int mode, int dtype, std::vector<Plan> &out) {
  const bool grad = mode != WM_FORWARD;
  const int Vs[4] = {4, 5, 8, 10};
  for (int gwi = 0; gwi < 2; ++gwi)
  for (int V : Vs) {
    const bool gw = gwi == 1;
    if (c->force_coeff && c->force_coeff != (gw ? 2 : 1)) continue;
    const void *fn = kernel_ptr(V, mode, dtype, gw);
    if (!fn) continue;
    cudaFuncAttributes fa;
    VIP_TRY(cudaFuncGetAttributes(&fa, fn));
    if (int rc = set_wave_attrs(c, fn)) return rc;
    for (int Q = 1; Q <= 16; ++Q) {
      const int Hb = band_height(c->NZ, Q, V);
      if ((Q - 1) * Hb >= c->NZ) continue;
      if (Hb < 4) continue;
      const int NXg = idiv_up(c->NX, 4);
      const int PX = 4 * (NXg + 2);
      const size_t smem = wave_smem(Hb, V, PX, NXg, grad, c->R, gw);
      if (smem + fa.sharedSizeBytes > c->smem_optin) continue;
      const int ntask = (Hb / V) * NXg;
      const int ntask_pad = idiv_up(ntask, 32) * 32;
      // threads per CTA: whole numbers of tasks per thread (1, 2, 3) where
      // possible, rounded up to warps, within the kernel's register budget
      const int Tmax = wave_max_threads(V, gw);
      int Ts[4] = {ntask_pad, idiv_up(idiv_up(ntask_pad, 2), 32) * 32,
                   idiv_up(idiv_up(ntask_pad, 3), 32) * 32, c->force_T};
      for (int ti = 0; ti < 4; ++ti) {
        if (Ts[ti] <= 0 || Ts[ti] > Tmax) continue;
        const int T = std::max(64, Ts[ti]);
        bool dup = false;
        for (int tj = 0; tj < ti; ++tj) dup |= std::max(64, Ts[tj]) == T;
        if (dup) continue;
        if (c->R > 4 * T) continue;   // receiver staging: at most 4 slots per thread
        Plan pl;
        pl.Q = Q; pl.V = V; pl.T = T; pl.Hb = Hb; pl.NXg = NXg; pl.PX = PX;
        pl.ntask = ntask; pl.ntask_pad = ntask_pad; pl.nwblk = ntask_pad / 32;
        pl.smem = smem; pl.mode = mode; pl.dtype = dtype; pl.gw = gw;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(Q, 1, 1);
        cfg.blockDim = dim3(T, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = Q; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
        cfg.attrs = at; cfg.numAttrs = 1;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, fn, &cfg) != cudaSuccess) {
          cudaGetLastError();
          continue;
        }
        if (ncl < 1) continue;
        pl.maxcl = ncl;
        // work items: split the sources of a particle over several clusters
        // only when the particles alone leave clusters idle
        double best = 1e300;
        for (int ipp = 1; ipp <= c->S; ++ipp) {
          const int spi = idiv_up(c->S, ipp);
          if (c->force_spi && spi != std::min(c->force_spi, c->S)) continue;
          const int ipp2 = idiv_up(c->S, spi);
          const int items = P * ipp2;
          const int waves = idiv_up(items, std::min(items, ncl));
          const double cost = (double)waves * spi;
          if (cost < best - 1e-9) { best = cost; pl.ipp = ipp2; pl.spi = spi; pl.items = items; }
        }
        pl.ncl = std::min(pl.items, ncl);
        // per step: tasks per thread x (rows + ~3 rows of window warm-up)
        // plus a fixed barrier cost
        const double tpt = (double)idiv_up(ntask_pad, T);
        const double per_step = tpt * (V + 3.0) + 6.0;
        // coefficients in global memory: every row also loads w' (and in the
        // adjoint reads and writes the accumulator) through L1/L2
        pl.est = best * per_step * (grad ? 2.0 : 1.0) * (gw ? 1.25 : 1.0);
        out.push_back(pl);
      }
    }
  }
  // the global-coefficient layout is for grids whose shared-memory bands
  // leave SMs idle; when a shared-memory plan already occupies 80 % of the
  // SMs it only adds L2 traffic, so it is not offered (unless forced)
  if (c->force_coeff != 2) {
    bool full = false;
    for (auto &p : out) full |= !p.gw && (double)p.maxcl * p.Q >= 0.8 * c->sm_count;
    if (full) {
      std::vector<Plan> keep;
      for (auto &p : out)
        if (!p.gw) keep.push_back(p);
      out.swap(keep);
    }
  }
  return out.empty() ? VIP_ERR_UNSUPPORTED : VIP_OK;
}

// Choose K and ncl under the memory budget.
static int fit_memory(fwi_ctx *c, Plan &pl, int P) {
  const size_t budget = free_budget(c);
  size_t least = (size_t)-1;   // smallest footprint tried
  std::vector<int> Ks;
  if (pl.mode == WM_FORWARD) Ks = {1};
  else if (c->ckpt >= 1) Ks = {std::min(c->ckpt, c->N)};
  else Ks = {1, 8, 16, 25, 32, 50, 64, 100, 128, 200, 256};
  for (int K : Ks) {
    pl.K = K;
    for (int ncl = pl.ncl; ncl >= 1; ncl = (ncl > 8 ? ncl * 3 / 4 : ncl - 1)) {
      Plan t = pl;
      t.ncl = ncl;
      plan_memory(c, t, P);
      least = std::min(least, t.total_bytes);
      if (t.total_bytes <= budget) { c->need_bytes = t.total_bytes; pl = t; return VIP_OK; }
      if (c->ckpt == 0 && ncl < pl.ncl / 2) break;   // prefer a larger K over idling SMs
    }
  }
  // the smallest footprint among the plans tried (one cluster for the
  // interval(s) allowed): what the caller would have to grant
  c->need_bytes = least;
  return VIP_ERR_NOMEM;
}

static int choose_plan(fwi_ctx *c, int P, int mode, int dtype, Plan &out) {
  std::vector<Plan> cand;
  int rc = make_candidates(c, P, mode, dtype, cand);
  if (rc) return rc;
  auto key = std::make_tuple(P, mode * 16 + dtype, c->S);
  auto it = c->tuned.find(key);
  const Plan *pick = nullptr;
  if (c->force_Q || c->force_spi) {
    for (auto &p : cand)
      if ((!c->force_Q || p.Q == c->force_Q) && (!c->force_V || p.V == c->force_V) &&
          (!c->force_T || p.T == c->force_T) && (!pick || p.est < pick->est))
        pick = &p;
    if (!pick) return VIP_ERR_UNSUPPORTED;
  } else if (it != c->tuned.end()) {
    for (auto &p : cand)
      if (p.Q == it->second[0] && p.V == it->second[1] && p.T == it->second[2] &&
          (int)p.gw == it->second[3])
        pick = &p;
  }
  if (!pick) {
    pick = &cand[0];
    for (auto &p : cand)
      if (p.est < pick->est - 1e-9 ||
          (std::fabs(p.est - pick->est) < 1e-9 && p.Q < pick->Q))
        pick = &p;
  }
  out = *pick;
  return fit_memory(c, out, P);
}

// Drop every cached graph (their launches may no longer be what a call with
// the current settings would enqueue).
static void drop_graphs(fwi_ctx *c) {
  for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

// A second launch for the SMs the main launch leaves idle (clusters of the
// main shape cannot be placed on every SM: on the GB300 36 four-CTA clusters
// take 144 of its 152 SMs). Its clusters are smaller, use the
// global-coefficient layout so that their taller band fits shared memory, and
// draw work items from the counter the main launch uses. Only for automatic
// plans, when the main launch has more items than clusters; the plan that
// puts the most idle SMs to work wins, then the cheaper one.
static bool choose_fill(fwi_ctx *c, const Plan &mn, int P, Plan &fp) {
  if (!c->fill || c->force_Q || c->force_V || c->force_T || c->force_coeff || c->force_spi)
    return false;
  if (mn.items <= mn.ncl) return false;
  const int idle = c->sm_count - mn.Q * mn.ncl;
  if (idle < 2) return false;
  std::vector<Plan> cand;
  c->force_coeff = 2;
  const int rc = make_candidates(c, P, mn.mode, mn.dtype, cand);
  c->force_coeff = 0;
  if (rc) {
    cudaGetLastError();
    return false;
  }
  const Plan *best = nullptr;
  auto used = [&](const Plan &q) { return std::min(q.maxcl, idle / q.Q) * q.Q; };
  for (auto &q : cand) {
    if (q.Q >= mn.Q || used(q) < 2) continue;
    if (!best || used(q) > used(*best) || (used(q) == used(*best) && q.est < best->est))
      best = &q;
  }
  if (!best) return false;
  fp = *best;
  fp.ipp = mn.ipp; fp.spi = mn.spi; fp.items = mn.items; fp.K = mn.K;
  fp.ncl = used(fp) / fp.Q;
  plan_memory(c, fp, P);
  return true;
}

static int ensure_scratch(fwi_ctx *c, size_t bytes) {
  if (bytes <= c->scratch_bytes) return VIP_OK;
  drop_graphs(c);
  if (c->scratch) {
    VIP_TRY(cudaDeviceSynchronize());
    VIP_TRY(cudaFree(c->scratch));
  }
  c->scratch = nullptr;
  c->scratch_bytes = 0;
  if (cudaMalloc(&c->scratch, bytes) != cudaSuccess) {
    cudaGetLastError();
    c->scratch = nullptr;
    return VIP_ERR_NOMEM;
  }
  c->scratch_bytes = bytes;
  return VIP_OK;
}

// Ordered sum of the partial gradients of the work items of each particle.
__global__ void grad_merge_kernel(const float *GI, int P, int ipp, int d, float *grad) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)P * d) return;
  const size_t p = q / d, i = q - p * d;
  float acc = 0.f;
  for (int k = 0; k < ipp; ++k) acc += GI[(p * ipp + k) * d + i];
  grad[q] = acc;
}

// Misfit of each particle from its per-receiver sums Jrec [P][S*R] (FP64): one
// block per particle, a fixed strided split over the threads and a fixed
// reduction tree, so the result does not depend on how the wave kernel split
// the grid or the work.
constexpr int kJThreads = 256;
__global__ void __launch_bounds__(kJThreads) j_reduce_kernel(const double *Jrec, int SR,
                                                             double scale, double *misfit,
                                                             int *status) {
  __shared__ double red[kJThreads];
  const int p = blockIdx.x;
  double t = 0.0;
  for (int k = threadIdx.x; k < SR; k += kJThreads) t += Jrec[(size_t)p * SR + k];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int h = kJThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    misfit[p] = red[0] * scale;
    // a non-finite misfit (non-finite observed data or wavefield) is reported
    if (!isfinite(red[0])) atomicOr(status, 4);
  }
}

// Misfit of the plain path: one accumulator per (particle, source).
__global__ void j_pairs_kernel(const double *Jpair, int P, int S, double scale, double *misfit,
                               int *status) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double t = 0.0;
  for (int s = 0; s < S; ++s) t += Jpair[(size_t)p * S + s];
  misfit[p] = t * scale;
  if (!isfinite(t)) atomicOr(status, 4);
}

// Kernel parameters of one launch. Scratch layout: the work counter, the
// per-receiver misfit sums, the per-item gradients, the main launch's slots,
// then (fill launch) its own slots. main_of_fill: the main plan when pl is the
// fill launch's; use_work: draw items from the shared counter.
static int fill_params(fwi_ctx *c, const Plan &pl, Tables *tb, int P, WaveParams &wp,
                       const Plan *main_of_fill = nullptr, bool use_work = false) {
  memset(&wp, 0, sizeof wp);
  wp.nz = c->nz; wp.nx = c->nx; wp.nb = c->nb; wp.NZ = c->NZ; wp.NX = c->NX;
  wp.N = c->N; wp.S = c->S; wp.R = c->R;
  wp.dtdx = (float)((double)c->dt / (double)c->dx);
  wp.dx2 = c->dx * c->dx;
  wp.c1 = (float)kC8[1]; wp.c2 = (float)kC8[2]; wp.c3 = (float)kC8[3]; wp.c4 = (float)kC8[4];
  wp.w_cfl = (float)cfl_w_limit();
  wp.Q = pl.Q; wp.Hb = pl.Hb; wp.NXg = pl.NXg; wp.PX = pl.PX;
  wp.ntask = pl.ntask; wp.ntask_pad = pl.ntask_pad; wp.nwblk = pl.nwblk;
  wp.gz = tb->gz; wp.gx = tb->gx; wp.wavelet = c->d_wavelet;
  wp.src_z = c->d_src_z; wp.src_x = c->d_src_x;
  wp.rmask = tb->rmask; wp.rbase = tb->rbase; wp.rperm = tb->rperm;
  wp.rbstart = tb->rbstart; wp.roff = tb->roff; wp.Rpad = receiver_pad(c->R);
  wp.items = pl.items; wp.ipp = pl.ipp; wp.spi = pl.spi;
  wp.K = pl.K; wp.nseg = pl.nseg;
  wp.status = c->d_status;
  wp.grad_atomic = pl.ipp > 1;
  // scratch carve
  Carve cv(c->scratch, c->scratch_bytes);
  int *work = cv.take<int>(64);
  wp.work = use_work ? work : nullptr;
  wp.Jrec = cv.take<double>((size_t)P * c->S * c->R);
  wp.GI = cv.take<float>((pl.mode != WM_FORWARD && pl.ipp > 1)
                             ? (size_t)P * pl.ipp * c->nz * c->nx : 0);
  const Plan &first = main_of_fill ? *main_of_fill : pl;
  char *slots = cv.take<char>((size_t)first.ncl * first.slot_bytes);
  if (main_of_fill) slots = cv.take<char>((size_t)pl.ncl * pl.slot_bytes);
  size_t off = 0;
  auto sub = [&](size_t n, size_t es) {
    char *r = slots + off;
    off += align_up(n * es, 256);
    return r;
  };
  // slot s occupies [s*slot_bytes, (s+1)*slot_bytes); fields are strided by
  // slot_bytes so that per-slot offsets below are in elements of each field
  wp.Dbuf = sub(pl.Dslot, dtype_size(pl.dtype));
  wp.Dscale = (signed char *)sub(pl.DSslot, 1);
  wp.rho = (float *)sub(pl.rhoslot, 4);
  wp.GP = (float *)sub(pl.GPslot, 4);
  wp.CK = (float *)sub(pl.CKslot, 4);
  wp.AS = (float *)sub(pl.ASslot, 4);
  wp.Wg = (float *)sub(pl.Wgslot, 4);
  wp.Gg = (float *)sub(pl.Ggslot, 4);
  const size_t sb = pl.slot_bytes;
  wp.Dslot = sb / dtype_size(pl.dtype);
  wp.DSslot = sb; wp.rhoslot = sb / 4; wp.GPslot = sb / 4; wp.CKslot = sb / 4;
  wp.ASslot = sb / 4; wp.Wgslot = sb / 4; wp.Ggslot = sb / 4;
  return cv.ok() ? VIP_OK : VIP_ERR_NOMEM;
}

static int prepare_wave(fwi_ctx *c, const Plan &pl) {
  const void *fn = kernel_ptr(pl.V, pl.mode, pl.dtype, pl.gw);
  if (!fn) return VIP_ERR_UNSUPPORTED;
  return set_wave_attrs(c, fn);
}

// One launch of the wave kernel; prio (a stream-priority value, 0 = the
// default) orders the placement of its clusters against a concurrent launch.
static int launch_wave(const Plan &pl, const WaveParams &wp, int ncl, cudaStream_t st,
                       int prio = 0) {
  const void *fn = kernel_ptr(pl.V, pl.mode, pl.dtype, pl.gw);
  if (!fn) return VIP_ERR_UNSUPPORTED;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ncl * pl.Q, 1, 1);
  cfg.blockDim = dim3(pl.T, 1, 1);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = pl.Q; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributePriority;
  at[1].val.priority = prio;
  cfg.attrs = at; cfg.numAttrs = prio ? 2 : 1;
  WaveParams local = wp;
  void *args[1] = {&local};
  VIP_TRY(cudaLaunchKernelExC(&cfg, fn, args));
  return VIP_OK;
}

// Enqueue one batched call (no graph): status reset, optional grad zeroing,
// the persistent kernel, the misfit reduction.
static int enqueue_batched(fwi_ctx *c, const Plan &pl, WaveParams &wp, int P, double sigma,
                           double *misfit, cudaStream_t st, const Plan *fp = nullptr,
                           const WaveParams *wpf = nullptr) {
  VIP_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int), st));
  int rc;
  if (fp) {
    // the fill launch runs on its own stream, joined before the reductions;
    // the main launch has the higher priority, so its clusters are placed
    // first and the fill's take the SMs left over
    VIP_TRY(cudaMemsetAsync(wp.work, 0, sizeof(int), st));
    VIP_TRY(cudaEventRecord(c->ev_fork, st));
    VIP_TRY(cudaStreamWaitEvent(c->fill_stream, c->ev_fork, 0));
    if ((rc = launch_wave(pl, wp, pl.ncl, st, c->prio_hi))) return rc;
    if ((rc = launch_wave(*fp, *wpf, fp->ncl, c->fill_stream, c->prio_lo))) return rc;
    VIP_TRY(cudaEventRecord(c->ev_join, c->fill_stream));
    VIP_TRY(cudaStreamWaitEvent(st, c->ev_join, 0));
  } else if ((rc = launch_wave(pl, wp, pl.ncl, st))) {
    return rc;
  }
  if (pl.mode != WM_FORWARD && wp.grad_atomic) {
    const size_t tot = (size_t)P * c->nz * c->nx;
    grad_merge_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(wp.GI, P, pl.ipp,
                                                                     c->nz * c->nx, wp.grad);
    VIP_CHECK_LAUNCH();
  }
  if (pl.mode == WM_GRADIENT && misfit) {
    const double scale = 0.5 / (sigma * sigma);
    j_reduce_kernel<<<P, kJThreads, 0, st>>>(wp.Jrec, c->S * c->R, scale, misfit, c->d_status);
    VIP_CHECK_LAUNCH();
  }
  return VIP_OK;
}

static int autotune_plan(fwi_ctx *c, int P, int mode, int dtype, const float *v,
                         const float *dobs, const float *dseis, double sigma, cudaStream_t st);

static int run_batched(fwi_ctx *c, int mode, const float *v, int P, const float *dobs,
                       const float *dseis, double sigma, double *misfit, float *grad,
                       float *seis, int dtype, cudaStream_t st) {
  const auto tkey = std::make_tuple(P, mode * 16 + dtype, c->S);
  if (c->autotune && !c->tuned.count(tkey) && !c->untunable.count(tkey)) {
    int rc = autotune_plan(c, P, mode, dtype, v, dobs, dseis, sigma, st);
    if (rc) return rc;
    if (!c->tuned.count(tkey)) c->untunable.insert(tkey);
  }
  Plan pl, fp;
  int rc = choose_plan(c, P, mode, dtype, pl);
  if (rc) return rc;
  bool fill = choose_fill(c, pl, P, fp);
  const size_t need = pl.total_bytes + (fill ? (size_t)fp.ncl * fp.slot_bytes : 0);
  if (fill && need > free_budget(c)) fill = false;
  Tables *tb = nullptr, *tbf = nullptr;
  rc = get_tables(c, pl.Q, pl.V, &tb);
  if (rc) return rc;
  if (fill && (rc = get_tables(c, fp.Q, fp.V, &tbf))) return rc;
  // (get_tables may grow the table list: look the main table up again)
  if (fill && (rc = get_tables(c, pl.Q, pl.V, &tb))) return rc;
  rc = ensure_scratch(c, fill ? need : pl.total_bytes);
  if (rc) return rc;
  WaveParams wp, wpf;
  rc = fill_params(c, pl, tb, P, wp, nullptr, fill);
  if (rc) return rc;
  wp.P = P; wp.v = v; wp.dobs = dobs; wp.dseis = dseis; wp.seis = seis; wp.grad = grad;
  wp.rho_scale = mode == WM_GRADIENT ? (float)((double)wp.dx2 / (sigma * sigma)) : wp.dx2;
  if (fill) {
    if ((rc = fill_params(c, fp, tbf, P, wpf, &pl, true))) return rc;
    wpf.P = P; wpf.v = v; wpf.dobs = dobs; wpf.dseis = dseis; wpf.seis = seis; wpf.grad = grad;
    wpf.rho_scale = wp.rho_scale;
  }
  // graph replay keyed by everything the launch depends on
  uint64_t sigma_bits;
  memcpy(&sigma_bits, &sigma, 8);
  std::array<uintptr_t, kGraphKeyLen> key = {
      (uintptr_t)mode | ((uintptr_t)c->S << 8), (uintptr_t)c->d_src_z,
      (uintptr_t)P, (uintptr_t)dtype, (uintptr_t)v, (uintptr_t)dobs,
      (uintptr_t)dseis, (uintptr_t)seis, (uintptr_t)misfit, (uintptr_t)grad,
      (uintptr_t)sigma_bits,
      ((uintptr_t)pl.Q << 32) | ((uintptr_t)pl.V << 16) | (uintptr_t)pl.T,
      ((uintptr_t)pl.ncl << 32) | (uintptr_t)pl.K,
      ((uintptr_t)pl.gw << 32) | (uintptr_t)pl.Hb,
      ((uintptr_t)pl.spi << 32) | (uintptr_t)pl.ipp,
      ((uintptr_t)pl.items << 32) | (uintptr_t)pl.nseg,
      (uintptr_t)pl.smem,
      fill ? (((uintptr_t)fp.Q << 48) | ((uintptr_t)fp.V << 32) | ((uintptr_t)fp.T << 16) |
              (uintptr_t)fp.ncl)
           : 0};
  const Plan *fpp = fill ? &fp : nullptr;
  const WaveParams *wpfp = fill ? &wpf : nullptr;
  if (!c->use_graphs) {
    if ((rc = prepare_wave(c, pl))) return rc;
    if (fill && (rc = prepare_wave(c, fp))) return rc;
    rc = enqueue_batched(c, pl, wp, P, sigma, misfit, st, fpp, wpfp);
    c->last_stream = st;
    return rc;
  }
  for (auto &g : c->graphs) {
    if (g.key == key) {
      VIP_TRY(cudaGraphLaunch(g.exec, st));
      c->last_stream = st;
      return VIP_OK;
    }
  }
  if ((rc = prepare_wave(c, pl))) return rc;
  if (fill && (rc = prepare_wave(c, fp))) return rc;
  cudaGraph_t graph;
  VIP_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  rc = enqueue_batched(c, pl, wp, P, sigma, misfit, c->cap_stream, fpp, wpfp);
  cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &graph);
  if (rc) { if (ce == cudaSuccess) cudaGraphDestroy(graph); return rc; }
  VIP_TRY(ce);
  GraphEntry ge;
  ge.key = key;
  cudaError_t ie = cudaGraphInstantiate(&ge.exec, graph, 0);
  cudaGraphDestroy(graph);
  VIP_TRY(ie);
  if (c->graphs.size() >= 16) {
    cudaGraphExecDestroy(c->graphs.front().exec);
    c->graphs.erase(c->graphs.begin());
  }
  c->graphs.push_back(ge);
  VIP_TRY(cudaGraphLaunch(ge.exec, st));
  c->last_stream = st;
  return VIP_OK;
}

// Autotuning: time the candidate launches on a one-wave, short-run problem
// built from the caller's own inputs, keep the fastest.
static int autotune_plan(fwi_ctx *c, int P, int mode, int dtype, const float *v,
                         const float *dobs, const float *dseis, double sigma, cudaStream_t st) {
  std::vector<Plan> cand;
  int rc = make_candidates(c, P, mode, dtype, cand);
  if (rc) return rc;
  std::sort(cand.begin(), cand.end(), [](const Plan &a, const Plan &b) { return a.est < b.est; });
  if (cand.size() > 6) cand.resize(6);
  const size_t outn = mode == WM_FORWARD ? (size_t)P * c->S * c->R * c->N
                                         : (size_t)P * c->nz * c->nx;
  // every resource below is released on every return path
  struct Held {
    fwi_ctx *c;
    int Nsave;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Held() {
      c->N = Nsave;
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      if (out) cudaFree(out);
    }
  } h{c, c->N};
  VIP_TRY(cudaMalloc(&h.out, outn * 4));
  VIP_TRY(cudaEventCreate(&h.e0));
  VIP_TRY(cudaEventCreate(&h.e1));
  float best = 1e30f;
  bool timed = false;
  std::array<int, 4> pick = {0, 0, 0, 0};
  c->N = std::min(c->N, 48);
  for (auto &pl0 : cand) {
    Plan pl = pl0;
    pl.K = 1;
    pl.items = std::min(pl.items, pl.maxcl);
    pl.ncl = pl.items;
    plan_memory(c, pl, P);
    if (pl.total_bytes > free_budget(c)) continue;
    Tables *tb = nullptr;
    if ((rc = get_tables(c, pl.Q, pl.V, &tb))) return rc;
    if ((rc = ensure_scratch(c, pl.total_bytes))) return rc;
    WaveParams wp;
    if ((rc = fill_params(c, pl, tb, P, wp))) return rc;
    wp.P = P; wp.v = v; wp.dobs = dobs; wp.dseis = dseis;
    wp.seis = h.out; wp.grad = h.out; wp.grad_atomic = 0;
    wp.rho_scale = 1.f;
    wp.items = pl.items;
    if ((rc = prepare_wave(c, pl))) return rc;
    for (int rep = 0; rep < 3; ++rep) {
      if (rep == 2) VIP_TRY(cudaEventRecord(h.e0, st));
      if ((rc = launch_wave(pl, wp, pl.ncl, st))) return rc;
      if (rep == 2) VIP_TRY(cudaEventRecord(h.e1, st));
    }
    VIP_TRY(cudaEventSynchronize(h.e1));
    float ms = 0.f;
    VIP_TRY(cudaEventElapsedTime(&ms, h.e0, h.e1));
    // normalise by the full problem's number of waves
    const float score = (float)(ms * idiv_up(pl0.items, pl0.ncl));
    if (score < best) { best = score; pick = {pl.Q, pl.V, pl.T, (int)pl.gw}; }
    timed = true;
  }
  // nothing fitted the memory budget: leave the choice to the cost model
  if (timed) c->tuned[std::make_tuple(P, mode * 16 + dtype, c->S)] = pick;
  (void)sigma;
  return VIP_OK;
}

// ---------------------------------------------------------------------------
// Plain per-step path.
__global__ void plain_set_w(const float *v, int nz, int nx, int nb, int NZ, int NX, float dtdx,
                            float wcfl, float *W, int *status) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= NZ * NX) return;
  const int z = idx / NX, x = idx - z * NX;
  const int iz = min(max(z - nb, 0), nz - 1), ix = min(max(x - nb, 0), nx - 1);
  const float vv = v[(size_t)iz * nx + ix];
  const float cc = __fmul_rn(vv, dtdx);
  const float w = __fmul_rn(cc, cc);
  if (!(w <= wcfl)) atomicOr(status, 1);
  if (!isfinite(vv)) atomicOr(status, 2);
  W[idx] = w;
}

__global__ void plain_fold(const float *Gm, const float *v, int nz, int nx, int nb, int NZ,
                           int NX, float dx2, float *grad) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nz * nx) return;
  const int iz = q / nx, ix = q - iz * nx;
  const int za = iz == 0 ? 0 : iz + nb, zb = iz == nz - 1 ? NZ - 1 : iz + nb;
  const int xa = ix == 0 ? 0 : ix + nb, xb = ix == nx - 1 ? NX - 1 : ix + nb;
  double acc = 0.0;
  for (int z = za; z <= zb; ++z)
    for (int x = xa; x <= xb; ++x) acc += (double)Gm[(size_t)z * NX + x];
  grad[q] = (float)(acc * 2.0 / ((double)v[q] * (double)dx2));
}

static void free_plain(fwi_ctx *c) {
  cudaFree(c->pl_W); cudaFree(c->pl_a); cudaFree(c->pl_Gm); cudaFree(c->pl_gz);
  cudaFree(c->pl_gx); cudaFree(c->pl_recmap); cudaFree(c->pl_J);
  c->pl_W = c->pl_a = c->pl_Gm = c->pl_gz = c->pl_gx = nullptr;
  c->pl_recmap = nullptr;
  c->pl_J = nullptr;
  c->pl_ready = false;
}

static int alloc_plain(fwi_ctx *c) {
  const size_t C = (size_t)c->NZ * c->NX;
  VIP_TRY(cudaMalloc(&c->pl_W, C * 4));
  VIP_TRY(cudaMalloc(&c->pl_a, 2 * C * 4));
  VIP_TRY(cudaMalloc(&c->pl_Gm, C * 4));
  VIP_TRY(cudaMalloc(&c->pl_gz, c->NZ * 4));
  VIP_TRY(cudaMalloc(&c->pl_gx, c->NX * 4));
  VIP_TRY(cudaMalloc(&c->pl_recmap, C * 4));
  VIP_TRY(cudaMalloc(&c->pl_J, sizeof(double) * 4096));
  std::vector<float> gz(c->NZ), gx(c->NX);
  auto prof = [&](int i, int n) {
    const int into = std::max(std::max(c->nb - i, i - (n - 1 - c->nb)), 0);
    const double a = c->alpha * into;
    return (float)std::exp(-a * a);
  };
  for (int z = 0; z < c->NZ; ++z) gz[z] = prof(z, c->NZ);
  for (int x = 0; x < c->NX; ++x) gx[x] = prof(x, c->NX);
  std::vector<int> rm(C, -1);
  for (int r = 0; r < c->R; ++r) rm[(size_t)c->rec_z[r] * c->NX + c->rec_x[r]] = r;
  VIP_TRY(cudaMemcpy(c->pl_gz, gz.data(), c->NZ * 4, cudaMemcpyHostToDevice));
  VIP_TRY(cudaMemcpy(c->pl_gx, gx.data(), c->NX * 4, cudaMemcpyHostToDevice));
  VIP_TRY(cudaMemcpy(c->pl_recmap, rm.data(), C * 4, cudaMemcpyHostToDevice));
  return VIP_OK;
}

// The plain-mode buffers are made on first use, all or none: a failure part
// way releases what was allocated, so a later call retries instead of
// launching on a missing buffer.
static int ensure_plain(fwi_ctx *c) {
  if (c->pl_ready) return VIP_OK;
  const int rc = alloc_plain(c);
  if (rc) {
    free_plain(c);
    return rc;
  }
  c->pl_ready = true;
  return VIP_OK;
}

static int run_plain(fwi_ctx *c, int mode, const float *v, int P, const float *dobs,
                     const float *dseis, double sigma, double *misfit, float *grad, float *seis,
                     cudaStream_t st) {
  int rc = ensure_plain(c);
  if (rc) return rc;
  const size_t C = (size_t)c->NZ * c->NX;
  const int N = c->N;
  const int K = mode == WM_FORWARD ? 1 : std::max(1, std::min(c->ckpt == 0 ? 1 : c->ckpt, N));
  const int nseg = idiv_up(N, K);
  // scratch: D slabs (N or K), checkpoints, parked adjoint state, rho
  const size_t Dn = mode == WM_FORWARD ? 0 : (size_t)(K == 1 ? N : K) * C;
  const size_t CKn = K > 1 ? (size_t)nseg * 2 * C : 0;
  const size_t ASn = K > 1 ? 2 * C : 0;
  const size_t rhon = (size_t)c->R * N;
  const size_t need = align_up(Dn * 4, 256) + align_up(CKn * 4, 256) + align_up(ASn * 4, 256) +
                      align_up(rhon * 4, 256);
  c->need_bytes = need;
  if (need > free_budget(c)) return VIP_ERR_NOMEM;
  if ((rc = ensure_scratch(c, need))) return rc;
  Carve cv(c->scratch, c->scratch_bytes);
  float *D = cv.take<float>(Dn);
  float *CK = cv.take<float>(CKn);
  float *AS = cv.take<float>(ASn);
  float *rho = cv.take<float>(rhon);
  PlainParams q;
  q.NZ = c->NZ; q.NX = c->NX; q.N = N; q.R = c->R;
  q.c1 = (float)kC8[1]; q.c2 = (float)kC8[2];
  q.c3 = (float)kC8[3]; q.c4 = (float)kC8[4];
  q.gz = c->pl_gz; q.gx = c->pl_gx; q.W = c->pl_W; q.recmap = c->pl_recmap;
  const float dtdx = (float)((double)c->dt / (double)c->dx);
  const float dx2 = c->dx * c->dx;
  const float rho_scale = (float)((double)dx2 / (sigma * sigma));
  std::vector<float> wav(N);
  for (int n = 0; n < N; ++n) {
    const double tau = n * (double)c->dt - c->t0;
    const double a = M_PI * M_PI * (double)c->f0 * c->f0 * tau * tau;
    wav[n] = (float)((1.0 - 2.0 * a) * std::exp(-a));
  }
  const int TB = 256, GB = idiv_up((int)C, TB);
  VIP_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int), st));
  if (mode == WM_GRADIENT) VIP_TRY(cudaMemsetAsync(c->pl_J, 0, sizeof(double) * (size_t)P * c->S, st));
  float *a0 = c->pl_a, *a1 = c->pl_a + C;
  for (int p = 0; p < P; ++p) {
    const float *vp = v + (size_t)p * c->nz * c->nx;
    plain_set_w<<<GB, TB, 0, st>>>(vp, c->nz, c->nx, c->nb, c->NZ, c->NX, dtdx,
                                   (float)cfl_w_limit(), c->pl_W, c->d_status);
    VIP_CHECK_LAUNCH();
    if (mode != WM_FORWARD) VIP_TRY(cudaMemsetAsync(c->pl_Gm, 0, C * 4, st));
    for (int s = 0; s < c->S; ++s) {
      const int pair = p * c->S + s;
      const int sz = c->src_z[s], sx = c->src_x[s];
      VIP_TRY(cudaMemsetAsync(c->pl_a, 0, 2 * C * 4, st));
      float *cur = a0, *nxt = a1;
      for (int n = 0; n < N; ++n) {
        if (K > 1 && n % K == 0) {
          VIP_TRY(cudaMemcpyAsync(CK + (size_t)(n / K) * 2 * C, cur, C * 4, cudaMemcpyDeviceToDevice, st));
          VIP_TRY(cudaMemcpyAsync(CK + (size_t)(n / K) * 2 * C + C, nxt, C * 4, cudaMemcpyDeviceToDevice, st));
        }
        float *Dn_ = (mode != WM_FORWARD && K == 1) ? D + (size_t)n * C : nullptr;
        plain_fwd_step<<<GB, TB, 0, st>>>(
            q, cur, nxt, n, sz, sx, wav[n], Dn_,
            mode == WM_FORWARD ? seis + (size_t)pair * c->R * N : nullptr,
            mode == WM_GRADIENT ? dobs + (size_t)s * c->R * N : nullptr,
            mode == WM_GRADIENT ? rho : nullptr, rho_scale,
            mode == WM_GRADIENT ? c->pl_J + pair : nullptr);
        VIP_CHECK_LAUNCH();
        std::swap(cur, nxt);
      }
      if (mode == WM_FORWARD) continue;
      const float *rsrc = mode == WM_GRADIENT ? rho : dseis + (size_t)pair * c->R * N;
      const float rmul = mode == WM_GRADIENT ? 1.f : dx2;
      VIP_TRY(cudaMemsetAsync(c->pl_a, 0, 2 * C * 4, st));
      cur = a0; nxt = a1;
      if (K == 1) {
        for (int k = N; k >= 1; --k) {
          plain_adj_step<<<GB, TB, 0, st>>>(q, cur, nxt, k, rsrc, rmul, D + (size_t)(k - 1) * C,
                                            c->pl_Gm);
          VIP_CHECK_LAUNCH();
          std::swap(cur, nxt);
        }
      } else {
        for (int j = nseg - 1; j >= 0; --j) {
          const int n0 = j * K, n1 = std::min(N, n0 + K);
          VIP_TRY(cudaMemcpyAsync(AS, cur, C * 4, cudaMemcpyDeviceToDevice, st));
          VIP_TRY(cudaMemcpyAsync(AS + C, nxt, C * 4, cudaMemcpyDeviceToDevice, st));
          float *fc = a0, *fn = a1;
          VIP_TRY(cudaMemcpyAsync(fc, CK + (size_t)j * 2 * C, C * 4, cudaMemcpyDeviceToDevice, st));
          VIP_TRY(cudaMemcpyAsync(fn, CK + (size_t)j * 2 * C + C, C * 4, cudaMemcpyDeviceToDevice, st));
          for (int n = n0; n < n1; ++n) {
            plain_fwd_step<<<GB, TB, 0, st>>>(q, fc, fn, n, sz, sx, wav[n], D + (size_t)(n - n0) * C,
                                              nullptr, nullptr, nullptr, 0.f, nullptr);
            VIP_CHECK_LAUNCH();
            std::swap(fc, fn);
          }
          cur = a0; nxt = a1;
          VIP_TRY(cudaMemcpyAsync(cur, AS, C * 4, cudaMemcpyDeviceToDevice, st));
          VIP_TRY(cudaMemcpyAsync(nxt, AS + C, C * 4, cudaMemcpyDeviceToDevice, st));
          for (int k = n1; k > n0; --k) {
            plain_adj_step<<<GB, TB, 0, st>>>(q, cur, nxt, k, rsrc, rmul,
                                              D + (size_t)(k - 1 - n0) * C, c->pl_Gm);
            VIP_CHECK_LAUNCH();
            std::swap(cur, nxt);
          }
        }
      }
    }
    if (mode != WM_FORWARD) {
      plain_fold<<<idiv_up(c->nz * c->nx, TB), TB, 0, st>>>(
          c->pl_Gm, vp, c->nz, c->nx, c->nb, c->NZ, c->NX, dx2, grad + (size_t)p * c->nz * c->nx);
      VIP_CHECK_LAUNCH();
    }
  }
  if (mode == WM_GRADIENT && misfit) {
    j_pairs_kernel<<<idiv_up(P, 128), 128, 0, st>>>(c->pl_J, P, c->S, 0.5 / (sigma * sigma),
                                                    misfit, c->d_status);
    VIP_CHECK_LAUNCH();
  }
  c->last_stream = st;
  return VIP_OK;
}

// P = 0 is an empty batch: the entry points check their other arguments and
// return VIP_OK without touching the device (pointers may then be NULL).
static int check_call(fwi_ctx *c, const float *v, int P) {
  if (!c || P < 0 || (P > 0 && !v)) return VIP_ERR_ARG;
  return VIP_OK;
}

}  // namespace vip

// ===========================================================================
extern "C" {

const char *vip_strerror(int code) {
  switch (code) {
    case VIP_OK: return "ok";
    case VIP_ERR_ARG: return "invalid argument";
    case VIP_ERR_CFL: return "stability bound violated: max(v) dt/dx > 0.5547";
    case VIP_ERR_NOMEM: return "workspace too small or device allocation failed";
    case VIP_ERR_CUDA: return "CUDA runtime error";
    case VIP_ERR_TIMEOUT: return "bounded device wait expired";
    case VIP_ERR_NOTPD: return "kernel matrix not positive definite";
    case VIP_ERR_UNSUPPORTED: return "no feasible launch plan on this device";
    case VIP_ERR_NONFINITE: return "non-finite input (NaN or infinity)";
  }
  return "unknown status";
}

const char *vip_last_error(void) { return g_last_error; }

void vip_clear_error(void) { g_last_error[0] = 0; }

int fwi_create(const fwi_geom *g, size_t workspace_limit_bytes, fwi_ctx **out) {
  if (!g || !out) return VIP_ERR_ARG;
  *out = nullptr;
  if (g->nz < 1 || g->nx < 1 || g->nt < 1 || g->nsrc < 1 || g->nrec < 1 || g->nsponge < 0 ||
      !(g->dx > 0) || !(g->dt > 0) || !(g->f0 > 0) || !g->src_iz || !g->src_ix ||
      !g->rec_iz || !g->rec_ix || g->nrec > (1 << 24))
    return VIP_ERR_ARG;
  fwi_ctx *c = new fwi_ctx();
  c->nz = g->nz; c->nx = g->nx; c->nb = g->nsponge;
  c->NZ = g->nz + 2 * g->nsponge; c->NX = g->nx + 2 * g->nsponge;
  c->N = g->nt; c->S = g->nsrc; c->R = g->nrec;
  c->dx = g->dx; c->dt = g->dt; c->alpha = g->sponge_alpha; c->f0 = g->f0;
  c->t0 = g->t0 > 0 ? g->t0 : 1.0f / g->f0;
  c->ws_limit = workspace_limit_bytes;
  std::vector<long> seen;
  for (int s = 0; s < c->S; ++s) {
    if (g->src_iz[s] < 0 || g->src_iz[s] >= c->nz || g->src_ix[s] < 0 || g->src_ix[s] >= c->nx) {
      delete c; return VIP_ERR_ARG;
    }
    c->src_z.push_back(g->src_iz[s] + c->nb);
    c->src_x.push_back(g->src_ix[s] + c->nb);
  }
  for (int r = 0; r < c->R; ++r) {
    if (g->rec_iz[r] < 0 || g->rec_iz[r] >= c->nz || g->rec_ix[r] < 0 || g->rec_ix[r] >= c->nx) {
      delete c; return VIP_ERR_ARG;
    }
    c->rec_z.push_back(g->rec_iz[r] + c->nb);
    c->rec_x.push_back(g->rec_ix[r] + c->nb);
    seen.push_back((long)c->rec_z.back() * c->NX + c->rec_x.back());
  }
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) { delete c; return VIP_ERR_ARG; }
  auto fail = [&](int rc) { fwi_destroy(c); return rc; };
  if (cudaGetDevice(&c->device) != cudaSuccess) return fail(VIP_ERR_CUDA);
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
    return fail(VIP_ERR_CUDA);
  c->sm_count = v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device) != cudaSuccess)
    return fail(VIP_ERR_CUDA);
  c->smem_optin = (size_t)v;
  std::vector<float> wav(c->N);
  for (int n = 0; n < c->N; ++n) {
    const double tau = n * (double)c->dt - c->t0;
    const double a = M_PI * M_PI * (double)c->f0 * c->f0 * tau * tau;
    wav[n] = (float)((1.0 - 2.0 * a) * std::exp(-a));
  }
  if (cudaMalloc(&c->d_wavelet, c->N * 4) != cudaSuccess ||
      cudaMalloc(&c->d_src_z, c->S * 4) != cudaSuccess ||
      cudaMalloc(&c->d_src_x, c->S * 4) != cudaSuccess ||
      cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess)
    return fail(VIP_ERR_CUDA);
  if (cudaMemcpy(c->d_wavelet, wav.data(), c->N * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_src_z, c->src_z.data(), c->S * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_src_x, c->src_x.data(), c->S * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess)
    return fail(VIP_ERR_CUDA);
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(VIP_ERR_CUDA);
  if (cudaDeviceGetStreamPriorityRange(&c->prio_lo, &c->prio_hi) != cudaSuccess ||
      cudaStreamCreateWithPriority(&c->fill_stream, cudaStreamNonBlocking, c->prio_lo) !=
          cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return fail(VIP_ERR_CUDA);
  if (const char *e = getenv("VIPGB_GRAPHS")) c->use_graphs = atoi(e) != 0;
  *out = c;
  return VIP_OK;
}

void fwi_destroy(fwi_ctx *c) {
  if (!c) return;
  cudaDeviceSynchronize();
  for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
  for (auto &t : c->tables) {
    cudaFree(t.gz); cudaFree(t.gx); cudaFree(t.rmask); cudaFree(t.rbase); cudaFree(t.rperm);
    cudaFree(t.rbstart); cudaFree(t.roff);
  }
  cudaFree(c->scratch);
  cudaFree(c->d_wavelet); cudaFree(c->d_src_z); cudaFree(c->d_src_x); cudaFree(c->d_status);
  vip::free_plain(c);
  cudaFree(c->d_sub_z); cudaFree(c->d_sub_x); cudaFree(c->d_sub_dobs);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->fill_stream) cudaStreamDestroy(c->fill_stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  delete c;
}

int fwi_set_mode(fwi_ctx *c, int mode, int ckpt_every) {
  if (!c || (mode != FWI_MODE_BATCHED && mode != FWI_MODE_PLAIN) || ckpt_every < 0)
    return VIP_ERR_ARG;
  c->mode = mode;
  c->ckpt = ckpt_every;
  vip::drop_graphs(c);
  return VIP_OK;
}

int fwi_set_plan(fwi_ctx *c, int Q, int V, int T, int sources_per_item, int coeff) {
  if (!c || Q < 0 || Q > 16 || (V != 0 && V != 4 && V != 5 && V != 8 && V != 10) || T < 0 ||
      T > 512 || (T % 32) || sources_per_item < 0 || coeff < 0 || coeff > 2)
    return VIP_ERR_ARG;
  c->force_Q = Q; c->force_V = V; c->force_T = T; c->force_spi = sources_per_item;
  c->force_coeff = coeff;
  vip::drop_graphs(c);
  return VIP_OK;
}

int fwi_set_fill(fwi_ctx *c, int enable) {
  if (!c) return VIP_ERR_ARG;
  c->fill = enable ? 1 : 0;
  vip::drop_graphs(c);
  return VIP_OK;
}

int fwi_query_fill(fwi_ctx *c, int P, int precision, int *fill_out) {
  if (!c || P < 1 || !fill_out || precision < FWI_FP32 || precision > FWI_CKPT_FP16)
    return VIP_ERR_ARG;
  Plan pl, fp;
  int rc = choose_plan(c, P, WM_GRADIENT, precision, pl);
  if (rc) return rc;
  const bool fill = choose_fill(c, pl, P, fp) &&
                    pl.total_bytes + (size_t)fp.ncl * fp.slot_bytes <= free_budget(c);
  fill_out[0] = fill ? fp.Q : 0;
  fill_out[1] = fill ? fp.V : 0;
  fill_out[2] = fill ? fp.T : 0;
  fill_out[3] = fill ? fp.ncl : 0;
  return VIP_OK;
}

int fwi_set_autotune(fwi_ctx *c, int enable) {
  if (!c) return VIP_ERR_ARG;
  c->autotune = enable ? 1 : 0;
  vip::drop_graphs(c);
  return VIP_OK;
}

int fwi_autotune(fwi_ctx *c, int P, int precision) {
  (void)c; (void)P; (void)precision;
  // Tuning needs inputs; the tuner runs inside the first call with autotuning
  // enabled. This entry point only enables it for subsequent calls.
  return fwi_set_autotune(c, 1);
}

int fwi_query_plan(fwi_ctx *c, int P, int precision, int *plan_out, size_t *bytes_out) {
  if (!c || P < 1 || !plan_out) return VIP_ERR_ARG;
  Plan pl;
  int rc = choose_plan(c, P, WM_GRADIENT, precision, pl);
  if (rc == VIP_ERR_NOMEM && bytes_out) *bytes_out = c->need_bytes;
  if (rc) return rc;
  plan_out[0] = pl.Q; plan_out[1] = pl.V; plan_out[2] = pl.T; plan_out[3] = pl.Hb;
  plan_out[4] = pl.ncl; plan_out[5] = pl.K; plan_out[6] = pl.items; plan_out[7] = pl.spi;
  plan_out[8] = pl.gw ? 2 : 1; plan_out[9] = (int)pl.smem;
  if (bytes_out) *bytes_out = pl.total_bytes;
  return VIP_OK;
}

int fwi_forward(fwi_ctx *c, const float *v, int P, float *seis, vip_stream_t stream) {
  int rc = check_call(c, v, P);
  if (rc || (P > 0 && !seis)) return rc ? rc : VIP_ERR_ARG;
  if (P == 0) return VIP_OK;
  if (c->mode == FWI_MODE_PLAIN)
    return run_plain(c, WM_FORWARD, v, P, nullptr, nullptr, 1.f, nullptr, nullptr, seis, stream);
  return run_batched(c, WM_FORWARD, v, P, nullptr, nullptr, 1.f, nullptr, nullptr, seis,
                     FWI_FP32, stream);
}

int fwi_gradient(fwi_ctx *c, const float *v, int P, const float *dobs, double sigma,
                 double *misfit, float *grad, int precision, vip_stream_t stream) {
  int rc = check_call(c, v, P);
  if (rc) return rc;
  if ((P > 0 && (!dobs || !grad)) || !(sigma > 0) || precision < FWI_FP32 ||
      precision > FWI_CKPT_FP16)
    return VIP_ERR_ARG;
  if (c->mode == FWI_MODE_PLAIN && precision != FWI_FP32) return VIP_ERR_ARG;
  if (P == 0) return VIP_OK;
  if (c->mode == FWI_MODE_PLAIN) {
    if (P * c->S > 4096) return VIP_ERR_ARG;
    return run_plain(c, WM_GRADIENT, v, P, dobs, nullptr, sigma, misfit, grad, nullptr, stream);
  }
  return run_batched(c, WM_GRADIENT, v, P, dobs, nullptr, sigma, misfit, grad, nullptr,
                     precision, stream);
}

int fwi_gradient_sources(fwi_ctx *c, const float *v, int P, const float *dobs, double sigma,
                         const int *sources, int nb, double *misfit, float *grad,
                         int precision, vip_stream_t stream) {
  int rc = check_call(c, v, P);
  if (rc) return rc;
  if ((P > 0 && (!dobs || !grad)) || !sources || nb < 1 || nb > c->S || !(sigma > 0) ||
      precision < FWI_FP32 || precision > FWI_CKPT_FP16)
    return VIP_ERR_ARG;
  for (int k = 0; k < nb; ++k)
    if (sources[k] < 0 || sources[k] >= c->S) return VIP_ERR_ARG;
  if (c->mode == FWI_MODE_PLAIN) return VIP_ERR_UNSUPPORTED;
  if (P == 0) return VIP_OK;
  const size_t trace = (size_t)c->R * c->N;
  if (!c->d_sub_z) {
    // all three buffers or none: a partial allocation is released, so a later
    // call retries instead of using a null table
    int *sz_d = nullptr, *sx_d = nullptr;
    float *do_d = nullptr;
    if (cudaMalloc(&sz_d, sizeof(int) * c->S) != cudaSuccess ||
        cudaMalloc(&sx_d, sizeof(int) * c->S) != cudaSuccess ||
        cudaMalloc(&do_d, sizeof(float) * trace * c->S) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(sz_d); cudaFree(sx_d); cudaFree(do_d);
      return VIP_ERR_NOMEM;
    }
    c->d_sub_z = sz_d; c->d_sub_x = sx_d; c->d_sub_dobs = do_d;
  }
  // gather the minibatch in front of the launch, in stream order (a copy from
  // pageable host memory returns once the source has been staged, so sz, sx
  // may go out of scope)
  std::vector<int> sz(nb), sx(nb);
  for (int k = 0; k < nb; ++k) { sz[k] = c->src_z[sources[k]]; sx[k] = c->src_x[sources[k]]; }
  VIP_TRY(cudaMemcpyAsync(c->d_sub_z, sz.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, stream));
  VIP_TRY(cudaMemcpyAsync(c->d_sub_x, sx.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, stream));
  for (int k = 0; k < nb; ++k)
    VIP_TRY(cudaMemcpyAsync(c->d_sub_dobs + k * trace, dobs + (size_t)sources[k] * trace,
                            sizeof(float) * trace, cudaMemcpyDeviceToDevice, stream));
  // the batched path sees a problem with nb sources
  const int S0 = c->S;
  int *z0 = c->d_src_z, *x0 = c->d_src_x;
  c->S = nb; c->d_src_z = c->d_sub_z; c->d_src_x = c->d_sub_x;
  rc = run_batched(c, WM_GRADIENT, v, P, c->d_sub_dobs, nullptr, sigma, misfit, grad, nullptr,
                   precision, stream);
  c->S = S0; c->d_src_z = z0; c->d_src_x = x0;
  return rc;
}

int fwi_adjoint(fwi_ctx *c, const float *v, int P, const float *dseis, float *grad,
                int precision, vip_stream_t stream) {
  int rc = check_call(c, v, P);
  if (rc) return rc;
  if ((P > 0 && (!dseis || !grad)) || precision < FWI_FP32 || precision > FWI_CKPT_FP16)
    return VIP_ERR_ARG;
  if (c->mode == FWI_MODE_PLAIN && precision != FWI_FP32) return VIP_ERR_ARG;
  if (P == 0) return VIP_OK;
  if (c->mode == FWI_MODE_PLAIN) {
    return run_plain(c, WM_ADJOINT, v, P, nullptr, dseis, 1.f, nullptr, grad, nullptr, stream);
  }
  return run_batched(c, WM_ADJOINT, v, P, nullptr, dseis, 1.f, nullptr, grad, nullptr, precision,
                     stream);
}

size_t fwi_bytes_needed(fwi_ctx *c) { return c ? c->need_bytes : 0; }

int fwi_last_status(fwi_ctx *c) {
  if (!c) return VIP_ERR_ARG;
  if (cudaStreamSynchronize(c->last_stream) != cudaSuccess) return VIP_ERR_CUDA;
  int h = 0;
  if (cudaMemcpy(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return VIP_ERR_CUDA;
  if (h & 6) return VIP_ERR_NONFINITE;
  return (h & 1) ? VIP_ERR_CFL : VIP_OK;
}

}  // extern "C"
