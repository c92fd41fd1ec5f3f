"""The 2DGS regularisers of Eq. 3 on the GPU against the FP64 oracle: the Q = sum w z^2
plane of the forward, the backward with its cotangent, the depth distortion and the
normal consistency with their adjoints, and the parameter gradients they produce.
Both losses are also compared with the oracle's losses on the oracle's own planes.

The regularisers are checked in two parts: their arithmetic on the GPU's own planes
(FP64 sums of FP32 planes: 1e-6 relative on the losses; 1e-4 of the largest entry on the
FP32 adjoints, whose normal-consistency part goes through central differences of the
expected depth and a normalisation), and the planes themselves against the oracle
(forward bar 1e-4).  Parameter gradients meet the element-wise gradient bar (_helpers.grad_bar).
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from _helpers import FWD_TOL, KEYS, add_grads, grad_errors, oracle_adjoint, to_device, worst_element

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rast():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_08174_gb300 import Rasterizer, build
    build.build()
    r = Rasterizer(torch.device("cuda", 0), tile=(16, 16), persistent=True, pixels_per_thread=4)
    yield r
    r.close()


@pytest.fixture(scope="module")
def scene():
    sc = synthetic.small_scene(611, 2500, 56, 44, degree=1, n_views=3, scale_range=(0.06, 0.25))
    refs = [oracle.render(sc["gaussians"], cam) for cam in sc["cameras"]]
    return sc, refs


def _host(t):
    return t.double().cpu().numpy()


def test_depth2_plane_and_unchanged_outputs(rast, scene):
    sc, refs = scene
    dev = rast.device
    g = to_device(sc["gaussians"], dev)
    out, _ = rast.render(g, sc["cameras"], keep_state=False, depth2=True)
    plain, _ = rast.render(g, sc["cameras"], keep_state=False)
    torch.cuda.synchronize()
    for k in ("rgb", "alpha", "depth", "normal"):
        assert torch.equal(out[k], plain[k]), k      # the extra plane changes nothing else
    from paper_2501_08174_gb300 import pixel_offsets
    off = pixel_offsets(sc["cameras"])
    for v, ref in enumerate(refs):
        ok = ~ref["fragile"]
        got = _host(out["depth2"][off[v]:off[v + 1]])
        assert np.abs(got[ok] - ref["depth2"][ok]).max() <= FWD_TOL


def test_backward_with_a_depth2_cotangent(rast, scene):
    sc, refs = scene
    dev = rast.device
    g = to_device(sc["gaussians"], dev)
    cam = sc["cameras"][0]
    P = cam["width"] * cam["height"]
    rng = np.random.default_rng(3)
    ref0 = refs[0]
    keep = ~ref0["fragile_grad"]
    d = dict(rgb=np.zeros((P, 3)), alpha=rng.normal(size=P) * keep, depth=np.zeros(P),
             normal=np.zeros((P, 3)), depth2=rng.normal(size=P) * keep)
    ref, ref32 = oracle_adjoint(sc["gaussians"], cam, d)
    out, st = rast.render(g, [cam], depth2=True)
    grads = rast.render_backward(st, g, {k: torch.tensor(d[k], dtype=torch.float32, device=dev)
                                         for k in ("alpha", "depth2")})
    st.release()
    errs = grad_errors(grads, ref, ref32)
    assert max(errs.values()) <= 1.0, (errs, {k: worst_element(grads, ref, k, ref32) for k in KEYS})


def test_depth_distortion_loss_adjoint_and_parameter_gradient(rast, scene):
    sc, refs = scene
    dev = rast.device
    cams = sc["cameras"]
    g = to_device(sc["gaussians"], dev)
    from paper_2501_08174_gb300 import pixel_offsets
    off = pixel_offsets(cams)
    P = off[-1]
    out, st = rast.render(g, cams, depth2=True)
    grads_img = {k: torch.zeros(P, device=dev) for k in ("alpha", "depth", "depth2")}
    loss = rast.depth_distortion(out["alpha"], out["depth"], out["depth2"], cams, weight=0.7, grads=grads_img)
    torch.cuda.synchronize()
    own = {k: v.clone() for k, v in grads_img.items()}
    keep_all = torch.tensor(np.concatenate([~r["fragile_grad"] for r in refs]), device=dev)
    for v in grads_img.values():
        v.mul_(keep_all)                       # no cotangent at fragile pixels, on either side
    pgrads = rast.render_backward(st, g, grads_img)
    st.release()
    torch.cuda.synchronize()
    grads_ref, grads_ref32 = {}, {}
    for v, cam in enumerate(cams):
        sl = slice(off[v], off[v + 1])
        # the kernel's arithmetic on its own planes
        l_own, ga, gd, gq = oracle.depth_distortion(_host(out["alpha"][sl]), _host(out["depth"][sl]),
                                                    _host(out["depth2"][sl]), weight=0.7)
        assert float(loss[v]) == pytest.approx(l_own, rel=1e-6, abs=1e-12)
        for got, want in ((own["alpha"][sl], ga), (own["depth"][sl], gd), (own["depth2"][sl], gq)):
            assert np.abs(_host(got) - want).max() <= 1e-4 * np.abs(want).max() + 1e-12
        # the oracle's own loss on its planes, and its parameter gradient through the render
        ref = refs[v]
        l_ref, ra, rd, rq = oracle.depth_distortion(ref["alpha"], ref["depth"], ref["depth2"], weight=0.7)
        assert float(loss[v]) == pytest.approx(l_ref, rel=1e-3, abs=1e-6)
        keep = ~ref["fragile_grad"]
        n = cam["width"] * cam["height"]
        d = dict(rgb=np.zeros((n, 3)), alpha=ra * keep, depth=rd * keep, normal=np.zeros((n, 3)), depth2=rq * keep)
        gr, gr32 = oracle_adjoint(sc["gaussians"], cam, d)
        grads_ref, grads_ref32 = add_grads(grads_ref, gr), add_grads(grads_ref32, gr32)
    errs = grad_errors(pgrads, grads_ref, grads_ref32)
    assert max(errs.values()) <= 1.0, (errs, {k: worst_element(pgrads, grads_ref, k, grads_ref32) for k in KEYS})


def test_normal_consistency_loss_and_adjoint(rast, scene):
    sc, refs = scene
    dev = rast.device
    cams = sc["cameras"]
    g = to_device(sc["gaussians"], dev)
    from paper_2501_08174_gb300 import pixel_offsets
    off = pixel_offsets(cams)
    P = off[-1]
    out, st = rast.render(g, cams)
    gi = dict(alpha=torch.zeros(P, device=dev), depth=torch.zeros(P, device=dev), normal=torch.zeros(P, 3, device=dev))
    loss = rast.normal_consistency(out["alpha"], out["depth"], out["normal"], cams, weight=0.05, a_min=0.5, grads=gi)
    torch.cuda.synchronize()
    own = {k: v.clone() for k, v in gi.items()}
    keep_all = torch.tensor(np.concatenate([~r["fragile_grad"] for r in refs]), device=dev)
    gi["alpha"].mul_(keep_all)
    gi["depth"].mul_(keep_all)
    gi["normal"].mul_(keep_all[:, None])       # no cotangent at fragile pixels, on either side
    pgrads = rast.render_backward(st, g, gi)
    st.release()
    torch.cuda.synchronize()
    counted = 0
    grads_ref, grads_ref32 = {}, {}
    for v, cam in enumerate(cams):
        sl = slice(off[v], off[v + 1])
        a, dp, nr = _host(out["alpha"][sl]), _host(out["depth"][sl]), _host(out["normal"][sl])
        counted += int((a > 0.5).sum())
        l_own, ga, gd, gn = oracle.normal_consistency(a, dp, nr, cam, weight=0.05, a_min=0.5)
        assert float(loss[v]) == pytest.approx(l_own, rel=1e-5, abs=1e-9)
        for got, want in ((own["alpha"][sl], ga), (own["depth"][sl], gd), (own["normal"][sl], gn)):
            assert np.abs(_host(got) - want).max() <= 1e-4 * np.abs(want).max() + 1e-12
        # the oracle's own loss on its planes: no pixel lies within the forward bar of a_min, so
        # both sides count the same pixels; plane errors of 1e-4 relative move this loss by
        # < 1e-4 relative on this scene, so the 1e-3 bar of the depth distortion applies
        ref = refs[v]
        assert np.abs(ref["alpha"] - 0.5).min() > FWD_TOL
        l_ref = oracle.normal_consistency(ref["alpha"], ref["depth"], ref["normal"], cam, weight=0.05, a_min=0.5)[0]
        assert float(loss[v]) == pytest.approx(l_ref, rel=1e-3, abs=1e-6)
        # the parameter gradient of these cotangents through the oracle's adjoint
        n = cam["width"] * cam["height"]
        d = dict(rgb=np.zeros((n, 3)), alpha=_host(gi["alpha"][sl]), depth=_host(gi["depth"][sl]),
                 normal=_host(gi["normal"][sl]).reshape(n, 3))
        gr, gr32 = oracle_adjoint(sc["gaussians"], cam, d)
        grads_ref, grads_ref32 = add_grads(grads_ref, gr), add_grads(grads_ref32, gr32)
    assert counted > 200                      # the scene has covered pixels to check
    errs = grad_errors(pgrads, grads_ref, grads_ref32)
    assert max(errs.values()) <= 1.0, (errs, {k: worst_element(pgrads, grads_ref, k, grads_ref32) for k in KEYS})
