"""GB300 (sm_103a) double-MRT lattice Boltzmann melting with interfacial
tracking (Li, Yang & Zhang, arXiv:1604.03478).

The compute path is the CUDA library ``liblbm_melt.so`` behind the C ABI of
``include/lbm_melt.h``; this package holds its ctypes binding (``_abi``), a
small convenience wrapper (``Cavity``) and the in-tree build (``build``).
PyTorch is used only for device buffers and streams.
"""
from .cavity import Cavity, LbmError, default_rates  # noqa: F401
from .ensemble import Ensemble  # noqa: F401
from . import _abi  # noqa: F401
