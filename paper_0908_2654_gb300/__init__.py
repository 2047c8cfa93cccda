"""GB300-native implicit solve of flux-limited-diffusion radiation, hydrogen ionisation and
gas photo-heating (one operator-split step of Norman, Reynolds & So, arXiv:0908.2654).

The compute path is the CUDA library ``lib/librtfld.so`` (C ABI in include/rt.h); this
package holds its ctypes binding (``_rt``), unit conversion (``units``), a(t) for drivers
(``cosmology``), the step driver (``solver.Solver``) and the build script (``build``).
"""
from . import _rt  # noqa: F401
