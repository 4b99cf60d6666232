"""GB300-native regular path query engine (cuRPQ problem, arXiv 2602.20748).

The compute path lives in the CUDA library built from ``csrc/``; the Python
module ``rpq`` is a thin ctypes binding with the same entry points as the C
ABI declared in ``include/rpq.h``.  ``synth`` draws seeded synthetic inputs.
"""
