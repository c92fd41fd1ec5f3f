"""The allocation-free background loss against the context entry point (GPU).

Callers that cannot allocate device memory use ocgs_background_loss_noalloc,
whose scratch is a fixed static device array.  It must give the same loss and
adjoint as ocgs_background_loss on two calls in a row (the second call sees
the array the first one left behind), and refuse requests beyond its limits
before touching the device.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_08174_gb300 import build
    build.build()
    from paper_2501_08174_gb300 import Rasterizer, _lib
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rast = Rasterizer(dev)
    yield dev, rast, _lib.load(), _lib
    rast.close()


def _cams(sizes):
    import synthetic
    return [synthetic.make_camera((0.0, -3.0, 0.0), w, h) for w, h in sizes]


def _noalloc(lib, _lib, alpha, mask, cams, gamma, d_alpha):
    from paper_2501_08174_gb300 import camera_array
    loss = torch.empty(len(cams), dtype=torch.float64, device=alpha.device)
    st = lib.ocgs_background_loss_noalloc(C.c_void_p(alpha.data_ptr()), C.c_void_p(mask.data_ptr()),
                                          camera_array(cams), len(cams), float(gamma),
                                          C.c_void_p(loss.data_ptr()),
                                          C.c_void_p(d_alpha.data_ptr()) if d_alpha is not None else None,
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _lib.OK, _lib.STATUS[st]
    return loss


@pytest.mark.parametrize("sizes,gamma,seed", [(((64, 48), (333, 97), (800, 800)), 0.5, 1),
                                              (((1600, 1200), (17, 5)), 0.25, 2)])
def test_noalloc_loss_matches_context_entry_point_twice(setup, sizes, gamma, seed):
    dev, rast, lib, _lib = setup
    cams = _cams(sizes)
    P = sum(w * h for w, h in sizes)
    rng = np.random.default_rng(seed)
    for call in range(2):  # two calls in a row, different data each time
        alpha = torch.tensor(rng.uniform(0, 1, P).astype(np.float32), device=dev)
        mask = torch.tensor((rng.uniform(0, 1, P) < 0.3).astype(np.uint8), device=dev)
        base = torch.tensor(rng.normal(size=P).astype(np.float32), device=dev)
        d_ref = base.clone()
        ref = rast.background_loss(alpha, mask, cams, gamma=gamma, d_alpha=d_ref)
        d_new = base.clone()
        got = _noalloc(lib, _lib, alpha, mask, cams, gamma, d_new)
        torch.cuda.synchronize()
        # same kernels and block layout: identical up to the tolerance the other tests use
        np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=1e-12, atol=0)
        np.testing.assert_allclose(d_new.cpu().numpy(), d_ref.cpu().numpy(), rtol=0, atol=1e-7)
        assert torch.isfinite(got).all() and (got > 0).all(), call


def test_noalloc_loss_without_adjoint(setup):
    dev, rast, lib, _lib = setup
    cams = _cams(((128, 128),))
    rng = np.random.default_rng(3)
    alpha = torch.tensor(rng.uniform(0, 1, 128 * 128).astype(np.float32), device=dev)
    mask = torch.tensor((rng.uniform(0, 1, 128 * 128) < 0.5).astype(np.uint8), device=dev)
    got = _noalloc(lib, _lib, alpha, mask, cams, 0.5, None)
    ref = rast.background_loss(alpha, mask, cams, gamma=0.5)
    torch.cuda.synchronize()
    np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=1e-12, atol=0)


def test_noalloc_rejects_requests_beyond_its_limits(setup):
    dev, rast, lib, _lib = setup
    from paper_2501_08174_gb300 import camera_array
    small = torch.zeros(16, device=dev)
    m = torch.zeros(16, dtype=torch.uint8, device=dev)
    loss = torch.zeros(1100, dtype=torch.float64, device=dev)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(cams):
        return lib.ocgs_background_loss_noalloc(C.c_void_p(small.data_ptr()), C.c_void_p(m.data_ptr()),
                                                camera_array(cams), len(cams), 0.5,
                                                C.c_void_p(loss.data_ptr()), None, stream)
    # the checks come before any device work, so these pointers are never read
    assert call(_cams(((16384, 16384),) * 2)) == _lib.ERR_CAPACITY   # 2 x 65536 blocks > 65536
    assert call(_cams(((4, 4),) * 1025)) == _lib.ERR_CAPACITY         # more than 1024 views
    assert call(_cams(((0, 4),))) == _lib.ERR_ARG


def test_noalloc_full_view_table_matches_context_entry_point(setup):
    """1024 views (the table's limit) of ragged sizes: every view's loss, the block prefix the
    device-side set-up builds and the adjoint agree with the context entry point."""
    dev, rast, lib, _lib = setup
    rng = np.random.default_rng(4)
    sizes = [(int(w), int(h)) for w, h in rng.integers(1, 90, size=(1024, 2))]
    sizes[7] = (4097, 1)  # a view that needs two loss blocks
    cams = _cams(sizes)
    P = sum(w * h for w, h in sizes)
    alpha = torch.tensor(rng.uniform(0, 1, P).astype(np.float32), device=dev)
    mask = torch.tensor((rng.uniform(0, 1, P) < 0.4).astype(np.uint8), device=dev)
    d_ref = torch.zeros(P, device=dev)
    ref = rast.background_loss(alpha, mask, cams, gamma=0.5, d_alpha=d_ref)
    d_new = torch.zeros(P, device=dev)
    got = _noalloc(lib, _lib, alpha, mask, cams, 0.5, d_new)
    torch.cuda.synchronize()
    np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=1e-12, atol=0)
    np.testing.assert_allclose(d_new.cpu().numpy(), d_ref.cpu().numpy(), rtol=0, atol=1e-7)
