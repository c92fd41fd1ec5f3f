"""GB300-native object-centric 2D Gaussian Splatting rasterizer.

The compute path is the CUDA library ``libocgs.so`` (C ABI in ``include/ocgs.h``):
surfel projection, tile binning with an on-device radix sort, front-to-back
compositing of colour / accumulated opacity / depth / normal and its backward
pass, the background loss on accumulated opacity (Eq. 1) and the
occlusion-aware pruning sweep (Sec. 4.3) of arXiv 2501.08174.  This package
is the thin PyTorch binding; it fails loudly if the library is missing.
"""
from .api import (FRONT_FRACTION, PARAM_KEYS, ForwardState, Rasterizer, RenderFunction,  # noqa: F401
                  camera_array, n_pixels, pixel_offsets, render)
from ._lib import OcgsError  # noqa: F401

__all__ = ["Rasterizer", "RenderFunction", "render", "ForwardState", "OcgsError", "PARAM_KEYS",
           "FRONT_FRACTION", "n_pixels", "pixel_offsets", "camera_array"]
