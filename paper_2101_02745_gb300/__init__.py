"""GB300-native (sm_103a) particle-in-cell step for the neutrino fast flavour
instability (Richers, Willcox, Ford & Myers, arXiv:2101.02745).

The compute path is a CUDA library behind a C ABI (include/emu.h); ``emu``
is its ctypes binding and ``workloads`` the seeded synthetic inputs.
"""
__all__ = ["emu", "workloads"]
