"""GB300-native randomized Tucker decomposition (rHKron-re, rSTHKron).

The compute path is ``libtucker.so`` (CUDA kernels for sm_103a behind a C
ABI); ``paper_2211_13028_gb300.tucker`` is its thin ctypes binding.  Importing
this package does not load the library; the binding loads it on first use and
raises if it is missing.
"""
