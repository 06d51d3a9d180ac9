"""GB300-native compact Runge-Kutta flux reconstruction (cRK-FR) for
non-conservative hyperbolic systems.

The compute path is the C-ABI library ``libcrkfr.so`` (CUDA, sm_103a, FP64),
built from ``csrc/`` and declared in ``include/crkfr.h``.  ``crkfr`` is the
thin ctypes binding over it; ``workloads`` holds the seeded input recipes.
Importing the package does not load the library; the first call does, and
fails loudly if it is missing.
"""
