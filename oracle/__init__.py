"""FP64 CPU oracle for the DINR stochastic training step.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously correct
restatement of the paper's method (Sec. III "Our Approach", Appendix A
"Linear Projection", Appendix B "Network Architecture", Appendix C
"Training Parameters") used to check the CUDA library. Only the test suite,
the package smoke check and the benchmark's CPU-baseline leg may import it;
the product path never does, and this package imports nothing from the CUDA
library.

Modules:
  geometry  projection index decode, per-view rays, FOV chord, samples,
            coordinate normalisation
  network   Fourier encoding, coordinate MLP, its hand-derived backward
  step      forward model, loss, gradient, Adam, full training step,
            re-projection and voxel queries, finite differences
  phantom   closed-form line integrals of ellipsoid phantoms and Gaussian
            blobs, midpoint projection of an arbitrary analytic field
  sampler   the keyed Feistel bijection that draws minibatches

Parity status of each function is stated in its docstring; every function
is pinned by the CPU tests against closed forms, special cases, brute force
or finite differences (see tests/test_oracle_*.py).
"""
from . import geometry, network, step, phantom, sampler  # noqa: F401
