"""GB300-native vertex-star FDM/sparse relaxation (arXiv 2107.14758).

The compute path lives in the CUDA library ``libfdmpc.so`` (C-ABI declared
in ``include/fdmpc.h``); :mod:`.fdmpc` is its thin ctypes binding.
"""
