// Particle Gram matrix Xc Xc^T on the tensor cores (the only dense
// contraction of the SVGD update: the squared distances of the RBF kernel,
// Eq. 16, are |xc_i|^2 + |xc_j|^2 - 2 (Xc Xc^T)_ij).
#pragma once
#include "common.cuh"

namespace vip {

// Partial Gram sums of the upper-triangle 128x128 tiles, split along the
// coordinate axis: parts[split][i][j] (np x np per split, np a multiple of
// 128). Xh [np][dp] is the BF16 image of the centred particles (rows >= n and
// columns >= d zero). With Xm, Xl (the BF16 pieces of the successive
// remainders, x ~ h + m + l) the product is accumulated from the six terms
// hh + hm + mh + hl + lh + mm, whose dropped terms are below 2^-24 |x||y|;
// with Xm = Xl = NULL it is the single product hh. dp is a multiple of 64.
// err: device word, bit 0 set when a bounded wait inside the kernel expired.
int gram_tc_launch(const __nv_bfloat16 *Xh, const __nv_bfloat16 *Xm, const __nv_bfloat16 *Xl,
                   int n, int dp, int np, int splits, float *parts, int *err, cudaStream_t st);

// SVGD / sSVGD update on the tensor cores: X[i][c] <- clip(X[i][c] +
// sum_k A[i][k] B[c][k] + rcoef[i] Xc[i][c] isq[c], lo, hi) for i < n, c < d,
// with A [np][Kp] and B [dp][Kp] each given as three BF16 pieces (h, m, l)
// multiplied with the six-product split (FP32-class accuracy), and isq[c] =
// 1/sqrt(q_c) of the matrix-valued kernel (FP32). np, dp multiples of 128,
// Kp of 64; isq, lo, hi may be NULL (no scaling, no bound). err as for
// gram_tc_launch. skip (device word, may be NULL): when nonzero at the time
// the kernel runs, X is left unchanged (an earlier kernel of the step saw a
// non-finite input).
int update_tc_launch(const __nv_bfloat16 *const A[3], const __nv_bfloat16 *const B[3], int n,
                     int d, int np, int dp, int Kp, const float *Xc, const float *rcoef,
                     const float *isq, const float *lo, const float *hi, float *X, int *err,
                     const int *skip, cudaStream_t st);

}  // namespace vip
