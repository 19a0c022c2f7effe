"""FP64 CPU oracle of the SCAO real-time pipeline -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously-correct statement of what the GPU
path computes, used to check it.  Only the test suite, the package smoke test
and the CPU-baseline leg of the benchmark may import it; the product path
(the CUDA library and its Python binding) never does, and shares no code,
headers, tables or helpers with it.

Modules
  pipeline  pixel calibration, centre-of-gravity slopes, slope packing, dense
            reconstruction (MVM) and the leaky integrator (Sec. 2.1, Fig. 3)
  quant     reduced-precision storage of the control matrix (BF16, FP8 E4M3
            with per-row scales) -- the 16-bit storage idea of Sec. 2.3.4
  mlp       the learned slope predictor: feature gather, forward, analytic
            backward and Adam, all in FP64

Parity status of each function is stated in its module header.
"""
from . import pipeline, quant, mlp  # noqa: F401
