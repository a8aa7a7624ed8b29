"""Plain FP64 CPU oracle for the variational Bayesian FWI hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
execute this package: only the test suite, the smoke check and the
benchmark's CPU-baseline leg use it. It shares no code with the CUDA library
(no kernels, headers, helpers, tables or constant generators); the only module
both sides use is the seeded input generator ``synth``.

Contents, each following the paper (Zhang & Curtis, "VIP - Variational
Inversion Package", arXiv 2310.13325):

  fwi     forward wave simulation, Gaussian misfit (Eq. 26), exact discrete
          adjoint and velocity gradient (Sec. 3, Sec. 4.2)
  svgd    RBF kernel (Eq. 16), median bandwidth, SVGD update (Eq. 17),
          stochastic SVGD with Cholesky-correlated noise (Eq. 21-25)
  advi    logit transform (Eq. 12), mean-field ADVI gradients (Eq. 10-11)
          and Adam ascent (Sec. 2.2)
  tomo    travel-time tomography (Sec. 4.1): first-order upwind eikonal
          travel times by fast marching, misfit (Eq. 26) and its ray-traced
          velocity gradient
  philox  the Philox-4x32-10 counter-based generator (Salmon et al. 2011)
          with Box-Muller, to reproduce the device noise stream

Everything is float64 numpy, written for readability, not speed.
"""
