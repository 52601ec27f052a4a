"""GB300-native dense state-vector simulator (Kelly, arXiv:1805.00988).

The compute path is the CUDA library built from ``csrc/`` (C ABI declared in
``include/qsim_gb300.h``); ``sim`` is its thin ctypes binding and loads the
library on import, failing loudly when it has not been built.  ``circuits``
holds the seeded input generators and imports nothing else.
"""
