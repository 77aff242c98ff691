"""GB300 X-engine for a large-N FX radio correlator (arXiv:1411.3751 setting).

The compute path is the CUDA library ``libcorr`` (C ABI in ``include/corr.h``); ``corr`` is its
Python binding and ``synth`` the seeded input generator used by the tests and the benchmark.
"""

__version__ = "0.1.0"
