"""GB300-native EnKF-MC analysis: C-ABI library (libenkfmc.so) with sm_103a kernels.

`binding` loads the library and exposes its entry points; `filter` wraps one
problem for torch tensors.  Nothing here computes on the CPU.
"""
__all__ = ["binding", "filter"]
