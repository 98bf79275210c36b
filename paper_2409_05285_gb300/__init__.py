"""GB300-native finite-temperature PEPS-VMC cooling step (arXiv:2409.05285).

The compute path lives in the CUDA library built from ``csrc/`` (C ABI declared in
``include/peps_vmc.h``); ``binding`` is a thin ctypes layer over it.
"""
