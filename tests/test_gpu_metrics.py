"""SSIM of masked images (the D-SSIM part of Eq. 2's photometric loss, and the masked
SSIM of Sec. 5) and the masked PSNR of Sec. 5 on the GPU, against the FP64 oracle.

Tolerances: the windowed statistics are 121-term FP32 sums and the variances subtract
squared means, so single values of the SSIM map carry errors of a few 1e-6 on images
with intensities in [0, 1]; the per-view means stay within 1e-5.  The gradient is the
same window applied to three adjoint maps, compared at the parity bar for gradients
(1e-3 relative, infinity norm).  PSNR is summed in FP64 from the FP32 inputs: 1e-6 dB.
"""
import numpy as np
import pytest
import torch

import oracle
from _helpers import GRAD_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rast():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_08174_gb300 import Rasterizer, build
    build.build()
    r = Rasterizer(torch.device("cuda", 0))
    yield r
    r.close()


def _cams(sizes):
    return [dict(viewmat=np.eye(4), fx=50.0, fy=50.0, cx=w / 2, cy=h / 2, width=w, height=h, near_plane=0.2)
            for w, h in sizes]


def _images(rng, sizes, smooth=False):
    rgbs, tgts, masks = [], [], []
    for w, h in sizes:
        t = rng.uniform(size=(h, w, 3))
        if smooth:
            from scipy import ndimage
            t = ndimage.gaussian_filter(t, sigma=(3, 3, 0))
            t = (t - t.min()) / (t.max() - t.min())
        r = np.clip(t + rng.normal(scale=0.1, size=t.shape), 0.0, 1.0)
        yy, xx = np.mgrid[0:h, 0:w]
        m = ((xx - w / 2) ** 2 + (yy - h / 2) ** 2 <= (0.4 * min(w, h)) ** 2).astype(np.uint8)
        rgbs.append(r.astype(np.float32))
        tgts.append(t.astype(np.float32))
        masks.append(m)
    return rgbs, tgts, masks


def _flat(arrs, dev, dtype):
    return torch.tensor(np.concatenate([a.reshape(-1) for a in arrs]).astype(dtype), device=dev)


def _ssim_check(rast, sizes, seed, smooth=False, weight=0.2, base_value=0.25):
    rng = np.random.default_rng(seed)
    dev = rast.device
    rgbs, tgts, masks = _images(rng, sizes, smooth)
    cams = _cams(sizes)
    rgb, tgt, mask = _flat(rgbs, dev, np.float32), _flat(tgts, dev, np.float32), _flat(masks, dev, np.uint8)
    base = torch.full_like(rgb, base_value)    # the adjoint is accumulated onto what is there
    d_rgb = base.clone()
    s_all, s_m = rast.ssim(rgb, tgt, mask, cams, weight=weight, d_rgb=d_rgb)
    torch.cuda.synchronize()
    got = (d_rgb - base).double().cpu().numpy()
    ref_grads = []
    for v in range(len(sizes)):
        ra, rm, rg = oracle.masked_ssim(rgbs[v].astype(np.float64), tgts[v].astype(np.float64), masks[v], weight)
        assert float(s_all[v]) == pytest.approx(ra, abs=1e-5), (v, float(s_all[v]), ra)
        assert float(s_m[v]) == pytest.approx(rm, abs=1e-5), (v, float(s_m[v]), rm)
        ref_grads.append(rg.reshape(-1))
    ref = np.concatenate(ref_grads)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= GRAD_TOL, err
    return got, ref


def test_ssim_and_its_adjoint_on_ragged_views(rast):
    _ssim_check(rast, [(37, 29), (64, 48), (17, 45), (5, 3)], seed=1)


def test_ssim_full_size_view(rast):
    # at 1600x1200 each value's gradient is ~1e-8, below the float32 spacing at 0.25: start from 0
    _ssim_check(rast, [(1600, 1200)], seed=2, smooth=True, base_value=0.0)


def test_ssim_of_identical_images(rast):
    rng = np.random.default_rng(3)
    sizes = [(40, 30), (33, 21)]
    _, tgts, masks = _images(rng, sizes)
    dev = rast.device
    t = _flat(tgts, dev, np.float32)
    mask = _flat(masks, dev, np.uint8)
    d = torch.zeros_like(t)
    s_all, s_m = rast.ssim(t, t.clone(), mask, _cams(sizes), weight=1.0, d_rgb=d)
    torch.cuda.synchronize()
    np.testing.assert_allclose(s_all.cpu().numpy(), 1.0, atol=1e-6)
    np.testing.assert_allclose(s_m.cpu().numpy(), 1.0, atol=1e-6)
    assert float(d.abs().max()) <= 1e-5   # SSIM is stationary at x2 = x1


def test_masked_psnr(rast):
    rng = np.random.default_rng(4)
    sizes = [(31, 22), (16, 16), (20, 9)]
    rgbs, tgts, masks = _images(rng, sizes)
    masks[1][:] = 0                        # no mask pixel: undefined
    rgbs[2] = tgts[2].copy()               # identical: +inf
    dev = rast.device
    got = rast.masked_psnr(_flat(rgbs, dev, np.float32), _flat(tgts, dev, np.float32), _flat(masks, dev, np.uint8),
                           _cams(sizes)).cpu().numpy()
    ref = oracle.masked_psnr(rgbs[0].astype(np.float64), tgts[0].astype(np.float64), masks[0])
    assert got[0] == pytest.approx(ref, abs=1e-6)
    assert np.isnan(got[1]) and got[2] == np.inf


def test_metric_arguments_are_checked(rast):
    from paper_2501_08174_gb300 import _lib
    sizes = [(8, 8)]
    dev = rast.device
    x = torch.zeros(8 * 8 * 3, device=dev)
    m = torch.ones(64, dtype=torch.uint8, device=dev)
    with pytest.raises(_lib.OcgsError) as e:
        rast.masked_psnr(x, x, m, _cams(sizes), max_i=0.0)
    assert e.value.code == _lib.ERR_ARG
    with pytest.raises(ValueError):
        rast.ssim(x[:-3], x, m, _cams(sizes))
