"""GB300 (sm_103a) isogeometric single-layer BEM: H^2 assembly, matvec and GMRES.

The compute path is the CUDA library ``libbembel.so`` behind the C ABI of
``include/bembel.h``; ``capi`` is its ctypes binding with the same names.
"""
from .capi import *  # noqa: F401,F403
from .capi import BembelError, Geometry, Operator, lib  # noqa: F401
