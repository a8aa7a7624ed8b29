// Shared host/device helpers of libvipgb (error plumbing, small math).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stddef.h>
#include "vipgb.h"

namespace vip {

// Records the first failing CUDA call of this thread for diagnostics.
void note_cuda_error(cudaError_t e, const char *what, const char *file, int line);

}  // namespace vip

#define VIP_TRY(expr)                                                       \
  do {                                                                      \
    cudaError_t e_ = (expr);                                                \
    if (e_ != cudaSuccess) {                                                \
      vip::note_cuda_error(e_, #expr, __FILE__, __LINE__);                  \
      return VIP_ERR_CUDA;                                                  \
    }                                                                       \
  } while (0)

#define VIP_CHECK_LAUNCH()                                                  \
  do {                                                                      \
    cudaError_t e_ = cudaGetLastError();                                    \
    if (e_ != cudaSuccess) {                                                \
      vip::note_cuda_error(e_, "kernel launch", __FILE__, __LINE__);        \
      return VIP_ERR_CUDA;                                                  \
    }                                                                       \
  } while (0)

namespace vip {

static inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
static inline int idiv_up(int a, int b) { return (a + b - 1) / b; }

// Bump allocator over a caller-provided workspace (256-byte aligned slices).
struct Carve {
  char *base;
  size_t off, cap;
  Carve(void *p, size_t c) : base((char *)p), off(0), cap(c) {}
  template <class T> T *take(size_t n) {
    off = align_up(off, 256);
    T *r = (T *)(base ? base + off : nullptr);
    off += n * sizeof(T);
    return r;
  }
  bool ok() const { return off <= cap; }
};

}  // namespace vip
