"""GB300-native hot path of ImaSk (stochastic multiresolution image sketching).

The compute path is the CUDA library ``libimask.so`` behind a C ABI
(``include/imask.h``); ``paper_2412_10249_gb300.imask`` is its thin ctypes
binding.  Importing this package loads nothing; the binding loads the
library on first use and raises if it is missing.
"""
