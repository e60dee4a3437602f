"""Plain, slow, FP64 CPU oracle of compressed NeNMF.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or run
anything in this package: only the tests, the smoke check and the benchmark's
CPU-baseline leg use it. It shares no code with the CUDA library; the two meet
only through the seeded inputs of `synth`.

Modules
  nenmf      Sec. 2 (NeNMF inner Nesterov loop, alpha series, stopping test),
             Alg. 1 (compressed NMF strategy), eq. (2)-(3) (plain NeNMF)
  subspace   Alg. 2 (randomized subspace iteration), Sec. 3 (random projection)
  philox     counter-based Gaussian sketch generator (Philox4x32-10 and
             Box-Muller, written from their published definitions)
  bruteforce exhaustive active-set NNLS for tiny problems (a pin, not a method)
  metrics    eq. (4) relative reconstruction error
"""

from . import bruteforce, metrics, nenmf, philox, subspace  # noqa: F401
