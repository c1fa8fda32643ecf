"""GB300-native EnKF-MC analysis: C-ABI library (libenkfmc.so) with sm_103a kernels.

`binding` loads the library and exposes its entry points as a `Handle`;
`autograd` wraps one analysis in a torch.autograd.Function.  Nothing here
computes on the CPU.
"""
__all__ = ["binding", "autograd"]
