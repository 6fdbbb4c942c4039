"""libchamfer: GB300 (sm_103a) Chamfer-Estimate (Bakshi et al., 2023).

The compute path is the CUDA library libchamfer.so (C ABI in include/chamfer.h);
`binding` marshals torch tensors / numpy arrays into it; `build` compiles it.
"""
from .binding import *  # noqa: F401,F403
from .binding import ChamferError, lib  # noqa: F401
