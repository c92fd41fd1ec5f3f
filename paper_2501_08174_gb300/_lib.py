"""ctypes declarations of the libocgs C ABI (include/ocgs.h).

Loading fails loudly when the shared library has not been built: there is
no CPU fallback anywhere in the product path.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libocgs.so")

STATUS = ["OCGS_OK", "OCGS_ERR_ARG", "OCGS_ERR_OOM", "OCGS_ERR_CUDA", "OCGS_ERR_TIMEOUT",
          "OCGS_ERR_NONFINITE", "OCGS_ERR_CAPACITY", "OCGS_ERR_STATE"]
OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NONFINITE, ERR_CAPACITY, ERR_STATE = range(8)


class Gaussians(C.Structure):
    _fields_ = [("xyz", C.c_void_p), ("quat", C.c_void_p), ("scale", C.c_void_p),
                ("opacity", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64),
                ("sh_degree", C.c_int32), ("reserved", C.c_int32)]


class Gaussians3d(C.Structure):
    _fields_ = [("xyz", C.c_void_p), ("quat", C.c_void_p), ("scale", C.c_void_p),
                ("opacity", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64),
                ("sh_degree", C.c_int32), ("reserved", C.c_int32)]


class GaussiansOut(C.Structure):
    _fields_ = [("xyz", C.c_void_p), ("quat", C.c_void_p), ("scale", C.c_void_p),
                ("opacity", C.c_void_p), ("sh", C.c_void_p)]


class Camera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 16), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("near_plane", C.c_float), ("reserved", C.c_int32)]


class Image(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("alpha", C.c_void_p), ("depth", C.c_void_p),
                ("normal", C.c_void_p), ("depth2", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("persistent", C.c_int32),
                ("pixels_per_thread", C.c_int32), ("front_fraction", C.c_float), ("batch", C.c_int32)]


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * 16), ("launches", C.c_int64 * 16)]


class StateInfo(C.Structure):
    _fields_ = [("n_pairs", C.c_int64), ("n_pixels", C.c_int64), ("n_tiles", C.c_int64),
                ("n_views", C.c_int64), ("n_evals", C.c_int64)]


STAGES = ["preprocess", "depth_sort", "binning", "tile_sort", "raster_fwd", "loss", "raster_bwd",
          "preprocess_bwd", "prune", "adam"]


class TuneResult(C.Structure):
    _fields_ = [("best", Options), ("best_ms", C.c_double), ("n_tried", C.c_int32), ("from_cache", C.c_int32)]


class AdamConfig(C.Structure):
    _fields_ = [("lr", C.c_double * 5), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
                ("step", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("n_gaussians", C.c_int64), ("n_views", C.c_int64), ("n_pixels", C.c_int64),
                ("n_visible", C.c_int64), ("n_pairs", C.c_int64), ("n_tiles", C.c_int64),
                ("tile_w", C.c_int32), ("tile_h", C.c_int32)]


# every exported entry point: name -> (restype, argtypes)
SIGNATURES = {
    "ocgs_status_str": (C.c_char_p, [C.c_int]),
    "ocgs_last_error": (C.c_char_p, [C.c_void_p]),
    "ocgs_abi_version": (C.c_int32, []),
    "ocgs_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p]),
    "ocgs_destroy": (C.c_int, [C.c_void_p]),
    "ocgs_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ocgs_set_options": (C.c_int, [C.c_void_p, C.POINTER(Options)]),
    "ocgs_set_coverage": (C.c_int, [C.c_void_p, C.c_int32]),
    "ocgs_get_options": (C.c_int, [C.c_void_p, C.POINTER(Options)]),
    "ocgs_get_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "ocgs_sync": (C.c_int, [C.c_void_p]),
    "ocgs_render": (C.c_int, [C.c_void_p, C.POINTER(Gaussians), C.POINTER(Camera), C.c_int32,
                              C.POINTER(Image), C.c_void_p, C.POINTER(C.c_void_p)]),
    "ocgs_render_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Gaussians),
                                       C.POINTER(Image), C.POINTER(GaussiansOut)]),
    "ocgs_state_release": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ocgs_background_loss": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Camera),
                                       C.c_int32, C.c_float, C.c_void_p, C.c_void_p]),
    "ocgs_background_loss_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Camera), C.c_int32, C.c_float,
                                               C.c_void_p, C.c_void_p, C.c_void_p]),
    "ocgs_accumulate_contribution": (C.c_int, [C.c_void_p, C.POINTER(Gaussians), C.POINTER(Camera),
                                               C.c_int32, C.c_void_p]),
    "ocgs_render_3d": (C.c_int, [C.c_void_p, C.POINTER(Gaussians3d), C.POINTER(Camera), C.c_int32,
                                 C.POINTER(Image), C.c_void_p]),
    "ocgs_accumulate_contribution_3d": (C.c_int, [C.c_void_p, C.POINTER(Gaussians3d), C.POINTER(Camera),
                                                  C.c_int32, C.c_void_p]),
    "ocgs_prune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_float, C.POINTER(Gaussians),
                             C.POINTER(GaussiansOut), C.POINTER(C.c_int64), C.c_void_p, C.c_int64,
                             C.POINTER(C.c_int64)]),
    "ocgs_adam_step": (C.c_int, [C.c_void_p, C.POINTER(Gaussians), C.POINTER(GaussiansOut),
                                 C.POINTER(GaussiansOut), C.POINTER(GaussiansOut), C.POINTER(AdamConfig)]),
    "ocgs_ssim": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Camera), C.c_int32,
                            C.c_float, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ocgs_masked_psnr": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Camera), C.c_int32,
                                   C.c_float, C.c_void_p]),
    "ocgs_depth_distortion": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Camera),
                                        C.c_int32, C.c_float, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ocgs_normal_consistency": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Camera),
                                          C.c_int32, C.c_float, C.c_float, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p]),
    "ocgs_masked_l1": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Camera),
                                 C.c_int32, C.c_float, C.c_void_p, C.c_void_p]),
    "ocgs_autotune": (C.c_int, [C.c_void_p, C.POINTER(Gaussians), C.POINTER(Camera), C.c_int32, C.c_char_p,
                                C.POINTER(TuneResult)]),
    "ocgs_contribution_graph_create": (C.c_int, [C.c_void_p, C.POINTER(Gaussians), C.POINTER(Camera), C.c_int32,
                                                 C.c_void_p, C.c_float, C.POINTER(C.c_void_p)]),
    "ocgs_graph_launch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ocgs_graph_destroy": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ocgs_state_query": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(StateInfo)]),
    "ocgs_kernel_launches": (C.c_int64, []),
    "ocgs_profile_enable": (C.c_int, [C.c_void_p, C.c_int32]),
    "ocgs_profile_read": (C.c_int, [C.c_void_p, C.POINTER(Profile)]),
}

_lib = None


def load() -> C.CDLL:
    """Load libocgs.so (built in-tree by ``paper_2501_08174_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libocgs.so is not built ({LIB_PATH}); run __graft_entry__.build() "
                               "or python -m paper_2501_08174_gb300.build")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class OcgsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        self.code = code
        name = STATUS[code] if 0 <= code < len(STATUS) else str(code)
        super().__init__(f"{name}: {msg}")
