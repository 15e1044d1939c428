"""GB300-native finite element assembly engine (P1/P2 tetrahedra).

The compute path lives in the CUDA library ``libfea.so`` (sources in
``csrc/``, C-ABI in ``include/fea.h``); ``fea`` is its thin ctypes binding.
"""
