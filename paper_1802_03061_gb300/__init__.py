"""GB300 (sm_103a) implementation of the homogeneous-medium fast method for
the integral formulation of the steady radiative transfer equation (Fan, An,
Ying): FFT-applied Nystrom operators (Sec. 2.3.1, 3.3.1) inside a device
GMRES, with FP32/BF16 inner solves and FP64 refinement.

The compute path is the CUDA library ``_build/librte.so`` behind the C ABI
of ``include/rte.h``; ``_binding`` mirrors it function by function and
``Plan`` adds torch-tensor conveniences (allocation and streams only).
"""
from . import _binding
from ._binding import RteError, make_opts  # noqa: F401
from .plan import Aniso3D, Batch, Inhom, Plan  # noqa: F401
