"""GB300-native corner-transfer (CTM) move for a 2-site iPEPS.

The compute path lives in the CUDA shared library ``libctm`` (C ABI declared in
``include/ctm.h``); ``paper_2306_08212_gb300.ctm`` is its thin ctypes binding.
Importing the package does not load the library; ``ctm.load()`` does, and fails
loudly when it is missing.
"""
