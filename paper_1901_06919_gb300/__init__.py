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
    calib_grad_shifts,
    fit,
    fit_general,
    fit_spectra,
    irfft2,
    pack_requests,
    pack_views,
    refocus,
    refocus_specs,
    sync_status,
    render,
    render_shifts,
    rfft2,
    workspace,
)
from .pipeline import FitRenderPipeline  # noqa: F401,E402
