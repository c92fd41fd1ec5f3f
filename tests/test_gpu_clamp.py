"""The 0.99 clamp of alpha (Sec. 4.3 compositing) on the GPU.

Records with o < 0.989 can never reach the clamp, and the backward takes a
clamp-free form of the blend for them, per record.  These tests check both
rasterizers' clamped form against the FP64 oracle on scenes whose opaque
surfels do reach the clamp (the other GPU scenes have o <= 0.95).
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from _helpers import FWD_TOL, KEYS, forward_errors, gpu_at, grad_errors, masked, oracle_adjoint, to_device, \
    worst_element

pytestmark = pytest.mark.gpu

W, H = 48, 40


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


def _append(g: dict, extra: dict) -> dict:
    out = {k: np.concatenate([g[k], extra[k]]).astype(np.float32) for k in KEYS}
    out["sh_degree"] = g["sh_degree"]
    return out


def _opaque_scene(seed: int = 701):
    """A small random scene in which half the surfels have o in [0.97, 0.999], in front of
    which four large surfels of opacity 0.999 face the camera (their centre pixels blend
    alpha = min(0.99, o G) at the clamp)."""
    sc = synthetic.small_scene(seed, 400, W, H, degree=1)
    g, cam = sc["gaussians"], sc["cameras"][0]
    rng = np.random.default_rng(seed)
    n = len(g["opacity"])
    hi = rng.random(n) < 0.5
    g["opacity"] = np.where(hi, rng.uniform(0.97, 0.999, size=n), g["opacity"]).astype(np.float32)
    R = np.asarray(cam["viewmat"], np.float64)[:3, :3]
    centre = -R.T @ np.asarray(cam["viewmat"], np.float64)[:3, 3]
    fwd = -centre / np.linalg.norm(centre)
    right, up = R[0], R[1]
    pts = np.stack([centre + fwd * (1.2 + 0.1 * i) + right * dx + up * dy
                    for i, (dx, dy) in enumerate(((0.15, 0.1), (-0.2, 0.05), (0.05, -0.2), (-0.1, -0.1)))])
    k = g["sh"].shape[1]
    extra = dict(xyz=pts, quat=synthetic.quats_with_normal(rng, np.repeat(fwd[None], 4, 0)),
                 scale=np.full((4, 2), 0.4), opacity=np.full(4, 0.999),
                 sh=rng.normal(0.0, 0.3, size=(4, k, 3)))
    return _append(g, extra), cam


def test_clamped_forward_matches_oracle(rast, dev):
    g_np, cam = _opaque_scene()
    out, _ = rast.render(to_device(g_np, dev), [cam])
    torch.cuda.synchronize()
    ref = oracle.render(g_np, cam)
    ok = ~ref["fragile"]
    assert ok.mean() > 0.97
    errs = forward_errors(gpu_at(out, np.arange(W * H)), ref, ok)
    assert max(errs.values()) <= FWD_TOL, errs


def test_single_opaque_surfel_is_clamped(rast, dev):
    """One large surfel of opacity 0.9999 facing the camera: near its centre o G > 0.99, so the
    blended alpha is the clamp, 0.99, on the GPU and in the oracle."""
    rng = np.random.default_rng(704)
    cam = synthetic.make_camera(np.array([0.011, -3.0, 0.013]), 33, 31)
    g_np = dict(xyz=np.zeros((1, 3), np.float32),
                quat=synthetic.quats_with_normal(rng, np.array([[0.0, 1.0, 0.0]])).astype(np.float32),
                scale=np.full((1, 2), 1.5, np.float32), opacity=np.array([0.9999], np.float32),
                sh=np.zeros((1, 1, 3), np.float32), sh_degree=0)
    out, _ = rast.render(to_device(g_np, dev), [cam])
    torch.cuda.synchronize()
    ref = oracle.render(g_np, cam)
    clamped = np.abs(ref["alpha"] - 0.99) <= 1e-12
    assert clamped.sum() >= 9
    a = out["alpha"].double().cpu().numpy()
    assert np.abs(a[clamped] - 0.99).max() <= 1e-6
    errs = forward_errors(gpu_at(out, np.arange(33 * 31)), ref, ~ref["fragile"])
    assert max(errs.values()) <= FWD_TOL, errs


def test_clamped_backward_matches_oracle_adjoint(rast, dev):
    g_np, cam = _opaque_scene(702)
    g = to_device(g_np, dev)
    out, state = rast.render(g, [cam])
    P = W * H
    rng = np.random.default_rng(7)
    d_out = dict(rgb=rng.normal(size=(P, 3)), alpha=rng.normal(size=P), depth=np.zeros(P),
                 normal=np.zeros((P, 3)))
    ok = ~oracle.render(g_np, cam)["fragile_grad"]
    assert ok.mean() > 0.95
    d_out = {k: masked(v, ok) for k, v in d_out.items()}
    ref, ref32 = oracle_adjoint(g_np, cam, d_out)
    grads = rast.render_backward(state, g, {k: torch.tensor(d_out[k], dtype=torch.float32, device=dev)
                                            for k in ("rgb", "alpha")})
    errs = grad_errors(grads, ref, ref32)
    assert max(errs.values()) <= 1.0, (errs, {k: worst_element(grads, ref, k, ref32) for k in KEYS})
