"""CPU checks of the C ABI: the library builds, loads and exports what the header declares.

No compute call is made here; the GPU tests exercise the entry points.
"""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ocgs.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2501_08174_gb300 import _lib, build
    build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ocgs_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("ocgs_create", "ocgs_destroy", "ocgs_render", "ocgs_render_backward",
                 "ocgs_background_loss", "ocgs_accumulate_contribution", "ocgs_prune"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2501_08174_gb300 import _lib
    assert set(declared_functions()) == set(_lib.SIGNATURES)


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """ctypes mirrors of the ABI structs have the C compiler's sizes and offsets."""
    from paper_2501_08174_gb300 import _lib
    src = tmp_path / "layout.c"
    structs = {"ocgs_gaussians": _lib.Gaussians, "ocgs_gaussians_out": _lib.GaussiansOut,
               "ocgs_camera": _lib.Camera, "ocgs_image": _lib.Image, "ocgs_options": _lib.Options,
               "ocgs_stats": _lib.Stats, "ocgs_profile": _lib.Profile, "ocgs_state_info": _lib.StateInfo,
               "ocgs_tune_result": _lib.TuneResult, "ocgs_adam_config": _lib.AdamConfig,
               "ocgs_gaussians3d": _lib.Gaussians3d}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ocgs.h"', 'int main(void){']
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.split("\n") if l)
    for cname, py in structs.items():
        assert int(out[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(out[f"{cname}.{f}"]) == getattr(py, f).offset, f"{cname}.{f}"


def test_status_strings_and_version(lib):
    assert lib.ocgs_abi_version() == 4
    assert lib.ocgs_status_str(0) == b"OCGS_OK"
    assert lib.ocgs_status_str(5) == b"OCGS_ERR_NONFINITE"
    assert lib.ocgs_status_str(99) == b"OCGS_ERR_UNKNOWN"


def test_null_arguments_are_rejected_without_a_device(lib):
    # argument checks precede any CUDA call
    assert lib.ocgs_create(None, 0, None) == 1
    assert lib.ocgs_destroy(None) == 1
    assert lib.ocgs_render(None, None, None, 1, None, None, None) == 1
    assert lib.ocgs_prune(None, None, 0.0, None, None, None, None, 0, None) == 1


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="only meaningful without a GPU")
def test_create_without_gpu_fails_loudly(lib):
    ctx = C.c_void_p()
    assert lib.ocgs_create(C.byref(ctx), 0, None) == 3  # OCGS_ERR_CUDA, no fallback
    from paper_2501_08174_gb300 import OcgsError, Rasterizer
    with pytest.raises(OcgsError):
        Rasterizer(0)


def test_noalloc_limits_are_checked_before_any_device_work(lib):
    # the allocation-free background loss validates its sizes on the host first, so these
    # placeholder pointers are never read and no device is needed
    import synthetic
    from paper_2501_08174_gb300 import _lib, camera_array

    def call(sizes, gamma=0.5, alpha=C.c_void_p(16), loss=C.c_void_p(16)):
        cams = [synthetic.make_camera((0.0, -3.0, 0.0), w, h) for w, h in sizes]
        return lib.ocgs_background_loss_noalloc(alpha, C.c_void_p(16), camera_array(cams), len(cams), gamma,
                                                loss, None, None)

    assert call([(16384, 16384)] * 2) == _lib.ERR_CAPACITY     # 2 x 65,536 blocks of 4,096 pixels
    assert call([(4, 4)] * 1025) == _lib.ERR_CAPACITY          # more than 1,024 views
    assert call([(0, 4)]) == _lib.ERR_ARG
    assert call([(4, 16385)]) == _lib.ERR_ARG
    assert call([(4, 4)], gamma=float("nan")) == _lib.ERR_ARG
    assert call([(4, 4)], alpha=None) == _lib.ERR_ARG
    assert call([(4, 4)], loss=None) == _lib.ERR_ARG
    assert lib.ocgs_background_loss_noalloc(C.c_void_p(16), C.c_void_p(16), None, 0, 0.5, C.c_void_p(16),
                                            None, None) == _lib.ERR_ARG
