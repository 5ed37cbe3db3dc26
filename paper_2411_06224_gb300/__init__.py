"""GB300-native Newton-step linear solver of StiffGIPC (arXiv 2411.06224).

Hash-key assembly of duplicate 3x3 Hessian blocks, the connectivity-enhanced
MAS preconditioner built on the device, and multi-RHS PCG, as hand-written
sm_103a CUDA behind the C ABI in include/gipc_mas_pcg.h.  ``binding`` holds
the thin Python marshalling layer (ctypes, same names as the C calls),
``autograd`` the torch.autograd wrapper of the adjoint, ``autotune`` the
launch-shape tuner and ``replicas`` the multi-rank timing helper.
"""

from .build import LIB_PATH, build  # noqa: F401
