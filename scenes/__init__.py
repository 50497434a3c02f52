"""Seeded synthetic light-field scenes.

This package is the one module shared by the FP64 oracle (``oracle/``) and the
CUDA path (``paper_1901_06919_gb300``): it only makes inputs.  It holds none of
the layer-construction or rendering arithmetic; the only Fourier work in it is
the exact sub-pixel translation used to synthesise views of a layered scene
(the scene model of Sec. IV-A), done with numpy's own FFT.
"""

from .lightfield import (  # noqa: F401
    view_grid,
    noise_1f,
    layered_scene,
    occluding_planes,
    random_layer_spectra,
    jittered_grid,
)
