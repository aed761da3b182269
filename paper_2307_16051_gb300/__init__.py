"""GB300-native three-precision Newton solver (C. T. Kelley, "Newton's Method in
Three Precisions", arXiv 2307.16051).

The solver lives in a C-ABI CUDA library (``libnewton3p.so``, sources under
``csrc/``); ``paper_2307_16051_gb300.nl`` is its thin ctypes binding.  The
library is loaded on first use and any failure to find it is an error: there
is no CPU path.
"""
