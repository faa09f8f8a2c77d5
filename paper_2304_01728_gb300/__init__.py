"""GB300-native DPG multigrid solver for 3D time-harmonic acoustics.

The solver lives in the C-ABI library ``libdpgmg.so`` (CUDA, sm_103a) built
from ``csrc/``; ``dpgmg`` is its ctypes binding and ``workloads`` the seeded
synthetic problem generators.
"""
