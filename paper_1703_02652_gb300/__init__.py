"""GB300-native (sm_103a) lattice Boltzmann solver for 3D solid-liquid phase change.

The hot path -- the coupled D3Q19 MRT/SRT flow and D3Q7 MRT/SRT enthalpy update of
Li & He (Sec. 2.2-2.5) -- is hand-written CUDA in ``csrc/`` behind the C ABI of
``include/lbpc.h``; this package is its thin Python binding.
"""
from .binding import LbpcError, lib  # noqa: F401
from .lbpc import LBPC  # noqa: F401
from .autograd import LiquidVolume, liquid_volume  # noqa: F401
