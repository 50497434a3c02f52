"""GB300 (sm_103a) Fourier Disparity Layers: layer construction and rendering.

The compute path is libfdl.so (include/fdl.h), hand-written CUDA; the Python
modules only marshal torch tensors and streams into it.
"""

from ._lib import FdlError, load  # noqa: F401
from .fdl import (  # noqa: F401
    FitWorkspace,
    RenderSpec,
    aperture_table,
    calib_grad,
    fit,
    fit_spectra,
    irfft2,
    pack_requests,
    refocus,
    refocus_specs,
    render,
    rfft2,
    workspace,
)
