"""The per-view losses of Eq. 1 and Eq. 2 on the GPU against the FP64 oracle.

Masked L1 (Eq. 2, L1 part): the kernel takes each difference of two FP32
values in FP64 (exact here) and sums in FP64, so the per-view loss agrees
with the oracle up to the FP64 summation order (1e-12 relative).  Its adjoint
adds +-weight/(3 h w) per masked value, a constant formed with two FP32
roundings (3 h w, then the division), so from a zero start it is within
3e-7 relative of the oracle's FP64 value, exactly 0 where R = I or M = 0;
with a non-zero start it is that zero-start value added in FP32.

Background loss (Eq. 1): alpha (1 - M) is exact in FP64, so the same 1e-12
bar holds; its adjoint gamma (1 - M)/(h w) has the same two roundings.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

SIZES = ((37, 23), (64, 48), (129, 5), (800, 600), (1, 1))  # ragged; 800x600 spans many loss blocks


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_08174_gb300 import build
    build.build()
    return torch.device("cuda", 0)


@pytest.fixture(scope="module")
def rast(dev):
    from paper_2501_08174_gb300 import Rasterizer
    r = Rasterizer(dev)
    yield r
    r.close()


def _cams():
    return [synthetic.make_camera((0.0, -3.0, 0.0), w, h) for w, h in SIZES]


def _views(cams):
    off = [0]
    for c in cams:
        off.append(off[-1] + c["width"] * c["height"])
    return off


def _images(seed, P, mask_kind, tie_frac=0.1):
    rng = np.random.default_rng(seed)
    rgb = rng.uniform(0.0, 1.0, size=(P, 3)).astype(np.float32)
    target = rng.uniform(0.0, 1.0, size=(P, 3)).astype(np.float32)
    ties = rng.uniform(size=(P, 3)) < tie_frac
    target[ties] = rgb[ties]  # exact ties: the adjoint must be 0 there
    ties = rgb == target        # (with any tie the draws made by chance)
    if mask_kind == "random":
        mask = (rng.uniform(size=P) < 0.6).astype(np.uint8)
    elif mask_kind == "ones":
        mask = np.ones(P, np.uint8)
    else:
        mask = np.zeros(P, np.uint8)
    return rgb, target, mask, ties


@pytest.mark.parametrize("mask_kind,seed", [("random", 1), ("ones", 2), ("zeros", 3)])
def test_masked_l1_matches_oracle_per_view(rast, dev, mask_kind, seed):
    cams = _cams()
    off = _views(cams)
    P = off[-1]
    rgb, target, mask, ties = _images(seed, P, mask_kind)
    weight = 0.7
    t = lambda a: torch.tensor(a, device=dev)
    d0 = torch.zeros(P, 3, device=dev)
    loss = rast.masked_l1(t(rgb), t(target), t(mask), cams, weight=weight, d_rgb=d0).cpu().numpy()
    base = torch.tensor(np.random.default_rng(seed + 10).normal(size=(P, 3)).astype(np.float32), device=dev)
    d1 = base.clone()
    loss1 = rast.masked_l1(t(rgb), t(target), t(mask), cams, weight=weight, d_rgb=d1).cpu().numpy()
    torch.cuda.synchronize()
    g0 = d0.double().cpu().numpy()
    for v in range(len(cams)):
        lo, hi = off[v], off[v + 1]
        ref_loss, ref_grad = oracle.masked_l1(rgb[lo:hi], target[lo:hi], mask[lo:hi], weight=weight)
        assert loss[v] == pytest.approx(ref_loss, rel=1e-12, abs=1e-300), (v, loss[v], ref_loss)
        np.testing.assert_allclose(g0[lo:hi], ref_grad, rtol=3e-7, atol=0, err_msg=f"view {v}")
        # the sign adjoint is exactly zero at ties and outside the mask, on both sides
        zero = ties[lo:hi] | (mask[lo:hi, None] == 0)
        assert (g0[lo:hi][zero] == 0).all() and (ref_grad[zero] == 0).all(), v
        assert (g0[lo:hi][~zero] != 0).all(), v
    if mask_kind == "zeros":
        assert (loss == 0).all()
    if mask_kind == "ones":  # the plain mean absolute error of each view
        for v in range(len(cams)):
            lo, hi = off[v], off[v + 1]
            mae = np.abs(rgb[lo:hi].astype(np.float64) - target[lo:hi]).mean()
            assert loss[v] == pytest.approx(mae, rel=1e-12)
    # a second call accumulates into d_rgb and returns the same losses bit for bit
    np.testing.assert_array_equal(loss1, loss)
    assert torch.equal(d1, base + d0)


def test_masked_l1_without_adjoint_and_weight_only_scales_it(rast, dev):
    cams = _cams()
    P = _views(cams)[-1]
    rgb, target, mask, _ = _images(5, P, "random")
    t = lambda a: torch.tensor(a, device=dev)
    a = rast.masked_l1(t(rgb), t(target), t(mask), cams, weight=1.0).cpu().numpy()
    d = torch.zeros(P, 3, device=dev)
    b = rast.masked_l1(t(rgb), t(target), t(mask), cams, weight=0.25, d_rgb=d).cpu().numpy()
    d1 = torch.zeros(P, 3, device=dev)
    rast.masked_l1(t(rgb), t(target), t(mask), cams, weight=1.0, d_rgb=d1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a, b)  # the weight scales the adjoint only
    np.testing.assert_allclose(d.cpu().numpy(), 0.25 * d1.cpu().numpy(), rtol=3e-7, atol=0)


@pytest.mark.parametrize("gamma,seed", [(0.5, 6), (1.0, 7)])
def test_background_loss_matches_oracle_per_view(rast, dev, gamma, seed):
    cams = _cams()
    off = _views(cams)
    P = off[-1]
    rng = np.random.default_rng(seed)
    alpha = rng.uniform(0.0, 1.0, size=P).astype(np.float32)
    mask = (rng.uniform(size=P) < 0.5).astype(np.uint8)
    d = torch.zeros(P, device=dev)
    loss = rast.background_loss(torch.tensor(alpha, device=dev), torch.tensor(mask, device=dev), cams,
                                gamma=gamma, d_alpha=d).cpu().numpy()
    torch.cuda.synchronize()
    dn = d.double().cpu().numpy()
    for v in range(len(cams)):
        lo, hi = off[v], off[v + 1]
        assert loss[v] == pytest.approx(oracle.background_loss(alpha[lo:hi], mask[lo:hi]), rel=1e-12, abs=1e-300)
        np.testing.assert_allclose(dn[lo:hi], oracle.background_loss_grad(mask[lo:hi], gamma), rtol=3e-7, atol=0)
