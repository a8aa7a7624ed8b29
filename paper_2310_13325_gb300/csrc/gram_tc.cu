// tcgen05 Gram kernel for sm_103a.
//
// One CTA of 4 warps computes one 128x128 FP32 tile of Xc Xc^T over a range
// of 64-wide coordinate blocks:
//   - thread 0 issues TMA tile loads (128 rows x 64 BF16 = 128 B per row,
//     128-byte swizzle) of the row block i and the row block j into a
//     shared-memory ring, signalling a "full" mbarrier per stage. With the
//     three-piece split a stage holds all three pieces of both row blocks
//     (96 KB) and all six products of the split are issued from it, so each
//     piece is read from L2 once per coordinate block; the ring is then one
//     stage, and the two CTAs that share an SM overlap one's copies and
//     epilogue with the other's products. One-piece BF16 stages (32 KB) form
//     a 3-stage ring;
//   - thread 32 issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M=128,
//     N=128, K=16, both operands K-major) into a 128-column TMEM accumulator
//     and releases each stage with tcgen05.commit on its "empty" mbarrier;
//   - after the last block all four warps read the accumulator back with
//     tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = tile rows) and store
//     the partial tile.
// Every mbarrier wait is bounded (about one second of clock cycles by
// default); on expiry the kernel records bit 0 in *err, skips its remaining
// work, waits for the copies it has issued with the same bound, frees TMEM
// and returns. A test hook (vip_test_set_wait) shortens the bound and can
// stop the copy producer from issuing anything, so that the consumer's wait
// expires on purpose without any fault.
#include "gram.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

namespace vip {

constexpr int GT_TILE_BYTES = 128 * 64 * 2;           // one operand tile
constexpr int GT_MAX_STAGES = 3;
constexpr long long GT_WAIT_CYCLES = 2000000000ll;    // ~1 s at 2 GHz

// Ring shape for P operand pieces: stages of 2P tiles (A pieces, then B
// pieces); one 96 KB stage for P = 3, three 32 KB stages for P = 1.
template <int P> struct Ring {
  static constexpr int kStages = P == 3 ? 1 : 3;
  static constexpr int kStageBytes = 2 * P * GT_TILE_BYTES;
  static constexpr int kBytes = kStages * kStageBytes;
};

// Test hook state (host): the wait bound passed to the next launches and
// whether their producers issue no copies.
static long long g_wait_cycles = GT_WAIT_CYCLES;
static int g_stall_producer = 0;

__device__ __forceinline__ uint32_t su32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; returns false (and flags *err) when the bound expires.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, int *err,
                                          long long limit) {
  if (mbar_try(b, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(b, parity)) {
    if (clock64() - t0 > limit) {
      atomicOr(err, 1);
      return false;
    }
  }
  return true;
}

// After an abort: wait (bounded) until every stage's last issued copy has
// landed, so no bulk copy into this CTA's shared memory is left in flight.
// Stage s was last filled by load number s + NST * floor((issued-1-s)/NST).
template <int NST>
__device__ __forceinline__ void drain_issued(uint64_t *full_bar, int issued, int *err,
                                             long long limit) {
  for (int s = 0; s < NST && s < issued; ++s) {
    const int use = (issued - 1 - s) / NST;   // last use of stage s issued
    mbar_wait(&full_bar[s], (uint32_t)(use & 1), err, limit);
  }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4}], [%2];" ::"r"(su32(dst)),
      "l"((uint64_t)map), "r"(su32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile stored with the
// 128-byte swizzle: rows of 128 B, 8-row (1024 B) swizzle atoms stacked along
// M/N (stride byte offset 1024), leading byte offset unused for this layout,
// descriptor version 1, layout type 2 (SWIZZLE_128B).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N>>3 at bits
// 17-22, M>>4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) |
                            ((128u >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t dt, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
      "[%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Product p of the split uses pieces (A, B) = (pass_a(p), pass_b(p)) with
// 0 = h, 1 = m, 2 = l: hh, hm, mh, hl, lh, mm (the dropped ml, lm, ll are
// below FP32 resolution).
__host__ __device__ constexpr int pass_a(int p) { return p == 2 ? 1 : (p == 4 ? 2 : (p == 5 ? 1 : 0)); }
__host__ __device__ constexpr int pass_b(int p) { return p == 1 ? 1 : (p == 3 ? 2 : (p == 5 ? 1 : 0)); }
static_assert(pass_a(0) == 0 && pass_a(1) == 0 && pass_a(2) == 1 && pass_a(3) == 0 &&
                  pass_a(4) == 2 && pass_a(5) == 1 && pass_b(0) == 0 && pass_b(1) == 1 &&
                  pass_b(2) == 0 && pass_b(3) == 2 && pass_b(4) == 0 && pass_b(5) == 1,
              "products hh, hm, mh, hl, lh, mm");

// Copy producer (thread 0) and MMA issuer (thread 32) of one CTA over the
// coordinate blocks kb0 .. kb1-1: per block one stage with the P pieces of
// row block ya of A and of row block yb of B, and the P == 3 ? 6 : 1 products
// accumulated into tacc. On an expired wait the thread sets *abort_flag and
// stops; the producer counts its issued loads in *n_issued.
template <int P>
__device__ __forceinline__ void tc_mainloop(const CUtensorMap *const ma[3],
                                            const CUtensorMap *const mb[3], int ya, int yb,
                                            int kb0, int kb1, uint8_t *ring, uint64_t *full_bar,
                                            uint64_t *empty_bar, uint64_t *done_bar,
                                            uint32_t tacc, int *abort_flag, int *n_issued,
                                            int *err, long long wait, int stall) {
  using R = Ring<P>;
  const int n_iter = kb1 - kb0;
  if (threadIdx.x == 0) {
    // producer (with the test hook's stall it issues nothing)
    for (int i = 0; i < (stall ? 0 : n_iter); ++i) {
      const int s = i % R::kStages;
      const uint32_t use = (uint32_t)(i / R::kStages);
      if (!mbar_wait(&empty_bar[s], (use & 1u) ^ 1u, err, wait)) { *abort_flag = 1; break; }
      if (*(volatile int *)abort_flag) break;
      const int kb = kb0 + i;
      uint8_t *st = ring + s * R::kStageBytes;
      mbar_expect_tx(&full_bar[s], R::kStageBytes);
#pragma unroll
      for (int k = 0; k < P; ++k) {
        tma_load_2d(st + k * GT_TILE_BYTES, ma[k], &full_bar[s], kb * 64, ya * 128);
        tma_load_2d(st + (P + k) * GT_TILE_BYTES, mb[k], &full_bar[s], kb * 64, yb * 128);
      }
      *n_issued = i + 1;
    }
  } else if (threadIdx.x == 32) {
    // MMA issuer
    for (int i = 0; i < n_iter; ++i) {
      const int s = i % R::kStages;
      const uint32_t use = (uint32_t)(i / R::kStages);
      if (!mbar_wait(&full_bar[s], use & 1u, err, wait)) { *abort_flag = 1; break; }
      tc_fence_after();
      const uint32_t st = su32(ring + s * R::kStageBytes);
#pragma unroll
      for (int pr = 0; pr < (P == 3 ? 6 : 1); ++pr) {
        const uint32_t sa = st + pass_a(pr) * GT_TILE_BYTES;
        const uint32_t sb = st + (P + pass_b(pr)) * GT_TILE_BYTES;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          umma(tacc, sdesc(sa + k * 32), sdesc(sb + k * 32),
               (i > 0 || pr > 0 || k > 0) ? 1u : 0u);
      }
      umma_commit(&empty_bar[s]);
    }
    umma_commit(done_bar);
  }
}

template <int P>
__global__ void __launch_bounds__(128, 1) gram_tc_kernel(const __grid_constant__ CUtensorMap mh,
                                                         const __grid_constant__ CUtensorMap mm,
                                                         const __grid_constant__ CUtensorMap ml,
                                                         int KB, int kper, int np, float *parts,
                                                         int *err, long long wait, int stall) {
  extern __shared__ __align__(1024) uint8_t gsm_raw[];
  // 1024-byte aligned stage ring (required by the 128-byte swizzle atoms)
  uint8_t *ring = (uint8_t *)(((uintptr_t)gsm_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full_bar[GT_MAX_STAGES], empty_bar[GT_MAX_STAGES], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, n_issued;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int t = blockIdx.x, ti = 0;
  const int T = np / 128;
  while (t >= T - ti) { t -= T - ti; ++ti; }
  const int tj = ti + t;
  const int kb0 = blockIdx.y * kper, kb1 = min(KB, kb0 + kper);
  float *Pt = parts + (size_t)blockIdx.y * np * np;
  const int row = ti * 128 + warp * 32 + lane;

  if (kb0 >= kb1) {   // empty coordinate range: the partial tile is zero
    float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 *dst = reinterpret_cast<float4 *>(Pt + (size_t)row * np + tj * 128);
    for (int c = 0; c < 32; ++c) dst[c] = z;
    return;
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < Ring<P>::kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    n_issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
                     su32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tacc = tmem_base;

  const CUtensorMap *const maps[3] = {&mh, &mm, &ml};
  tc_mainloop<P>(maps, maps, ti, tj, kb0, kb1, ring, full_bar, empty_bar, &done_bar, tacc,
                 &abort_flag, &n_issued, err, wait, stall);
  __syncwarp();
  // epilogue: wait for the accumulator
  const bool done = __all_sync(0xffffffffu, mbar_wait(&done_bar, 0u, err, wait));
  tc_fence_after();
  if (done && !*(volatile int *)&abort_flag) {
    const uint32_t lane_base = tacc + ((uint32_t)(warp * 32) << 16);
    float *dst = Pt + (size_t)row * np + tj * 128;
    for (int c = 0; c < 4; ++c) {
      uint32_t r[32];
      tmem_ld32(lane_base + c * 32, r);
      float4 *d4 = reinterpret_cast<float4 *>(dst + c * 32);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        d4[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                            __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
    }
  }
  // drain: every stage's copies must have landed before the CTA retires
  if (threadIdx.x == 0 && abort_flag) drain_issued<Ring<P>::kStages>(full_bar, n_issued, err, wait);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tacc) : "memory");
  }
}

// ---------------------------------------------------------------------------
// SVGD / sSVGD update on the tensor cores: one CTA computes a 128 x 128 tile
// of D = A B^T with A [np][Kp] (rows: particles; columns: the kernel matrix
// and, for sSVGD, the Cholesky factor) and B [dp][Kp] (rows: coordinates;
// columns: the matching right-hand sides), both as three BF16 pieces and the
// six-product split, the same pipeline as gram_tc_kernel (one 96 KB stage of
// all six tiles per block of K) over all KB blocks, then applies the update
// in the epilogue:
//   X[i][c] = clip(X[i][c] + D[i][c] + rcoef[i] Xc[i][c] isq[c], lo, hi)
// with isq[c] = 1/sqrt(q_c) of the matrix-valued kernel (isq NULL: 1). Tiles
// are ordered with the particle tiles of one coordinate tile adjacent, so its
// B rows are read once into L2.
__global__ void __launch_bounds__(128, 1) update_tc_kernel(
    const __grid_constant__ CUtensorMap ah, const __grid_constant__ CUtensorMap am,
    const __grid_constant__ CUtensorMap al, const __grid_constant__ CUtensorMap bh,
    const __grid_constant__ CUtensorMap bm, const __grid_constant__ CUtensorMap bl, int KB,
    int MT, int n, int d, const float *__restrict__ Xc, const float *__restrict__ rcoef,
    const float *__restrict__ isq, const float *__restrict__ lo, const float *__restrict__ hi,
    float *X, int *err, const int *skip, long long wait, int stall) {
  extern __shared__ __align__(1024) uint8_t usm_raw[];
  uint8_t *ring = (uint8_t *)(((uintptr_t)usm_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full_bar[GT_MAX_STAGES], empty_bar[GT_MAX_STAGES], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, n_issued;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ti = blockIdx.x % MT, tj = blockIdx.x / MT;

  if (threadIdx.x == 0) {
    for (int s = 0; s < Ring<3>::kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    n_issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
                     su32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tacc = tmem_base;

  const CUtensorMap *const mas[3] = {&ah, &am, &al};
  const CUtensorMap *const mbs[3] = {&bh, &bm, &bl};
  tc_mainloop<3>(mas, mbs, ti, tj, 0, KB, ring, full_bar, empty_bar, &done_bar, tacc,
                 &abort_flag, &n_issued, err, wait, stall);
  __syncwarp();
  const bool done = __all_sync(0xffffffffu, mbar_wait(&done_bar, 0u, err, wait));
  tc_fence_after();
  // a non-finite input reported by an earlier kernel of the step (*skip):
  // the particles are left as they were. The decision is taken for the whole
  // CTA, since the epilogue below synchronises it.
  const bool write = __syncthreads_and(done && !*(volatile int *)&abort_flag && !(skip && *skip));
  if (write) {
    // the accumulator tile goes through shared memory (the operand ring is
    // idle once every MMA has completed), [128][129] floats so that both the
    // row-wise writes from TMEM and the column-wise reads are free of bank
    // conflicts; the update then walks each row with consecutive lanes on
    // consecutive coordinates, so X, Xc, q, lo and hi are read and X written
    // in whole cache lines
    constexpr int TP = 129;
    float *tile = reinterpret_cast<float *>(ring);
    const uint32_t lane_base = tacc + ((uint32_t)(warp * 32) << 16);
    const int trow = warp * 32 + lane;
    for (int ch = 0; ch < 4; ++ch) {
      uint32_t r[32];
      tmem_ld32(lane_base + ch * 32, r);   // all lanes take part
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) tile[trow * TP + ch * 32 + jj] = __uint_as_float(r[jj]);
    }
    __syncthreads();
    // Each lane owns the tile columns lane + 32 k (k < 4) of the rows its warp
    // walks (warp, warp + 4, ...): their column terms are read once, and the
    // rows go in groups of kRows so that a thread has 2 kRows x 4 loads of X
    // and Xc in flight at a time instead of one pair per DRAM round trip.
    constexpr int kRows = 4;
    int cidx[4];
    float cs[4], clo[4], chi[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int c = tj * 128 + lane + 32 * k;
      cidx[k] = c < d ? c : -1;
      cs[k] = (isq && c < d) ? isq[c] : 1.f;
      clo[k] = (lo && c < d) ? lo[c] : 0.f;
      chi[k] = (hi && c < d) ? hi[c] : 0.f;
    }
    for (int m0 = 0; m0 < 32; m0 += kRows) {
      float xv[kRows][4], xcv[kRows][4], rc[kRows];
#pragma unroll
      for (int t = 0; t < kRows; ++t) {
        const int i = ti * 128 + warp + 4 * (m0 + t);
        rc[t] = i < n ? rcoef[i] : 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const bool ok = i < n && cidx[k] >= 0;
          const size_t g = (size_t)i * d + cidx[k];
          xv[t][k] = ok ? X[g] : 0.f;
          xcv[t][k] = ok ? Xc[g] : 0.f;
        }
      }
#pragma unroll
      for (int t = 0; t < kRows; ++t) {
        const int rr = warp + 4 * (m0 + t);
        const int i = ti * 128 + rr;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (i >= n || cidx[k] < 0) continue;
          const float xs = isq ? xcv[t][k] * cs[k] : xcv[t][k];
          // the move first (its two parts cancel in part), then one rounding
          // at the particle's own magnitude
          float x = xv[t][k] + fmaf(rc[t], xs, tile[rr * TP + lane + 32 * k]);
          if (lo) x = fmaxf(x, clo[k]);
          if (hi) x = fminf(x, chi[k]);
          X[(size_t)i * d + cidx[k]] = x;
        }
      }
    }
  }
  if (threadIdx.x == 0 && abort_flag) drain_issued<Ring<3>::kStages>(full_bar, n_issued, err, wait);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tacc) : "memory");
  }
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

static int make_map(CUtensorMap *m, const __nv_bfloat16 *base, int dp, int np) {
  auto fn = encode_fn();
  if (!fn) return VIP_ERR_CUDA;
  const cuuint64_t dims[2] = {(cuuint64_t)dp, (cuuint64_t)np};
  const cuuint64_t strides[1] = {(cuuint64_t)dp * 2};
  const cuuint32_t box[2] = {64, 128};
  const cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? VIP_OK : VIP_ERR_CUDA;
}

int gram_tc_launch(const __nv_bfloat16 *Xh, const __nv_bfloat16 *Xm, const __nv_bfloat16 *Xl,
                   int n, int dp, int np, int splits, float *parts, int *err, cudaStream_t st) {
  if (np % 128 || dp % 64 || ((uintptr_t)Xh & 15) || (!Xm) != (!Xl) ||
      (Xm && (((uintptr_t)Xm & 15) || ((uintptr_t)Xl & 15))) || n > np)
    return VIP_ERR_ARG;
  CUtensorMap mh, mm, ml;
  int rc = make_map(&mh, Xh, dp, np);
  if (rc) return rc;
  rc = make_map(&mm, Xm ? Xm : Xh, dp, np);
  if (rc) return rc;
  rc = make_map(&ml, Xl ? Xl : Xh, dp, np);
  if (rc) return rc;
  const int T = np / 128;
  const int tiles = T * (T + 1) / 2;
  const int KB = dp / 64;
  const int kper = (KB + splits - 1) / splits;
  VIP_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  if (Xm) {
    const size_t smem = (size_t)Ring<3>::kBytes + 1024;
    VIP_TRY(cudaFuncSetAttribute(gram_tc_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    gram_tc_kernel<3><<<dim3(tiles, splits), 128, smem, st>>>(mh, mm, ml, KB, kper, np, parts,
                                                              err, g_wait_cycles,
                                                              g_stall_producer);
  } else {
    const size_t smem = (size_t)Ring<1>::kBytes + 1024;
    VIP_TRY(cudaFuncSetAttribute(gram_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    gram_tc_kernel<1><<<dim3(tiles, splits), 128, smem, st>>>(mh, mm, ml, KB, kper, np, parts,
                                                              err, g_wait_cycles,
                                                              g_stall_producer);
  }
  VIP_CHECK_LAUNCH();
  return VIP_OK;
}

int update_tc_launch(const __nv_bfloat16 *const A[3], const __nv_bfloat16 *const Bm[3], int n,
                     int d, int np, int dp, int Kp, const float *Xc, const float *rcoef,
                     const float *isq, const float *lo, const float *hi, float *X, int *err,
                     const int *skip, cudaStream_t st) {
  if (np % 128 || dp % 128 || Kp % 64 || n > np || d > dp) return VIP_ERR_ARG;
  for (int k = 0; k < 3; ++k)
    if (((uintptr_t)A[k] & 15) || ((uintptr_t)Bm[k] & 15)) return VIP_ERR_ARG;
  CUtensorMap ma[3], mb[3];
  for (int k = 0; k < 3; ++k) {
    int rc = make_map(&ma[k], A[k], Kp, np);
    if (rc) return rc;
    rc = make_map(&mb[k], Bm[k], Kp, dp);
    if (rc) return rc;
  }
  const int MT = np / 128, NT = dp / 128;
  const size_t smem = (size_t)Ring<3>::kBytes + 1024;
  VIP_TRY(cudaFuncSetAttribute(update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
  VIP_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  update_tc_kernel<<<MT * NT, 128, smem, st>>>(ma[0], ma[1], ma[2], mb[0], mb[1], mb[2], Kp / 64,
                                               MT, n, d, Xc, rcoef, isq, lo, hi, X, err, skip,
                                               g_wait_cycles, g_stall_producer);
  VIP_CHECK_LAUNCH();
  return VIP_OK;
}

}  // namespace vip

extern "C" int vip_test_set_wait(long long cycles, int stall_producer) {
  if (cycles < 0 || stall_producer < 0 || stall_producer > 1) return VIP_ERR_ARG;
  vip::g_wait_cycles = cycles == 0 ? vip::GT_WAIT_CYCLES : cycles;
  vip::g_stall_producer = stall_producer;
  return VIP_OK;
}
