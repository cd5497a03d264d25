"""CPU oracle for the textured 2D-Gaussian-splat renderer (TEST INFRASTRUCTURE).

This package is the slow, plain reference the CUDA path is checked against.
It is test infrastructure only: the tests, the smoke check and the benchmark's
CPU-baseline leg may import it; the rendering library never does, and it
imports nothing from the rendering library (only ``scenegen`` for inputs).

Modules
  keys.py    FP32 specification of culling, tile binning and depth keys
             (bit-exact target for the GPU binning/sort).
  render.py  FP64 forward renderer written as the plain definition: ray-plane
             intersection (Sec. 3.1, Eq. 1-2), per-primitive texture lookup
             (Sec. 3.2-3.3, Eq. 4-6), normal mapping (Eq. 7), alpha compositing
             of the G-buffer (Eq. 3, Eq. 8-9), deferred split-sum shading
             (Eq. 10-12) -- plus a brute-force variant, an ambiguity mask and
             fragment counters.
  shading.py FP64 cube-map / LUT sampling and the shading function.
  grad.py    gradients of the forward by autograd (FP64) and central
             finite differences.
  loss.py    the image term of the training loss (Sec. 3.6): 0.8 L1 +
             0.2 (1 - SSIM), SSIM written out with an 11x11 Gaussian window,
             and its gradient by autograd.

Parity status per function is stated in each module header.
"""
