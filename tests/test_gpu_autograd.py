"""The differentiable entry point (RenderFunction / render) through torch autograd.

A torch loss over the rendered planes, differentiated by ``.backward()`` or
``torch.autograd.grad``, must give the FP64 oracle's adjoint of the same loss
at the gradient bar, with unused outputs passing None cotangents; the
wrapper must refuse a second backward through one render and a parameter
changed in place between the forward and the backward.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from _helpers import KEYS, add_grads, grad_errors, masked, oracle_adjoint, to_device, worst_element

pytestmark = pytest.mark.gpu


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
    r = Rasterizer(dev, tile=(16, 16), persistent=True, pixels_per_thread=4)
    yield r
    r.close()


@pytest.fixture(scope="module")
def scene():
    sc = synthetic.small_scene(1101, 700, 56, 44, degree=2, n_views=2)
    sc["cameras"][1] = synthetic.make_camera(
        sc["cameras"][1]["viewmat"][:3, :3].T @ -sc["cameras"][1]["viewmat"][:3, 3], 37, 61)
    return sc


def _leaves(g_np, dev):
    return {k: v.requires_grad_(True) for k, v in to_device(g_np, dev).items()}


def _cotangents(sc, planes, seed):
    """Per view, random cotangents of the planes named (zero for the others), with no
    cotangent on either side at pixels the oracle flags as fragile."""
    rng = np.random.default_rng(seed)
    out = []
    for cam in sc["cameras"]:
        P = cam["width"] * cam["height"]
        ok = ~oracle.render(sc["gaussians"], cam)["fragile_grad"]
        d = dict(rgb=rng.normal(size=(P, 3)), alpha=rng.normal(size=P), depth=rng.normal(size=P),
                 normal=rng.normal(size=(P, 3)))
        out.append({k: (masked(v, ok) if k in planes else np.zeros_like(v)) for k, v in d.items()})
    return out


def _oracle_grads(sc, d_views):
    tot, tot32 = {}, {}
    for cam, d in zip(sc["cameras"], d_views):
        ref, ref32 = oracle_adjoint(sc["gaussians"], cam, d)
        tot, tot32 = add_grads(tot, ref), add_grads(tot32, ref32)
    return tot, tot32


def _cat(d_views, key, dev):
    return torch.tensor(np.concatenate([d[key] for d in d_views]), dtype=torch.float32, device=dev)


@pytest.mark.parametrize("planes", [("rgb", "alpha"), ("rgb", "alpha", "depth", "normal"), ("depth",)])
def test_backward_through_render_gives_the_oracle_adjoint(rast, dev, scene, planes):
    from paper_2501_08174_gb300 import render
    d_views = _cotangents(scene, planes, seed=len(planes))
    leaves = _leaves(scene["gaussians"], dev)
    rgb, alpha, depth, normal = render(rast, leaves, scene["cameras"])
    outs = dict(rgb=rgb, alpha=alpha, depth=depth, normal=normal)
    # a torch loss over the planes used; the others get None cotangents
    loss = sum((outs[k] * _cat(d_views, k, dev)).sum() for k in planes)
    loss.backward()
    ref, ref32 = _oracle_grads(scene, d_views)
    got = {k: leaves[k].grad for k in KEYS}
    errs = grad_errors(got, ref, ref32)
    errs = {k: e for k, e in errs.items() if np.abs(ref[k]).max() > 0}  # depth alone leaves sh at zero
    bad = {k: worst_element(got, ref, k, ref32) for k, e in errs.items() if e > 1.0}
    assert max(errs.values()) <= 1.0, (errs, bad)
    if "rgb" not in planes:
        assert float(leaves["sh"].grad.abs().max()) == 0.0


def test_autograd_grad_matches_render_backward(rast, dev, scene):
    """torch.autograd.grad through render() against the binding's own render_backward with the
    same cotangents (the same kernels; only the atomic order may differ)."""
    from paper_2501_08174_gb300 import render
    d_views = _cotangents(scene, ("rgb", "alpha"), seed=7)
    leaves = _leaves(scene["gaussians"], dev)
    rgb, alpha, _, _ = render(rast, leaves, scene["cameras"])
    loss = (rgb * _cat(d_views, "rgb", dev)).sum() + (alpha * _cat(d_views, "alpha", dev)).sum()
    got = torch.autograd.grad(loss, [leaves[k] for k in KEYS])
    g = {k: v.detach() for k, v in leaves.items()}
    out, st = rast.render(g, scene["cameras"])
    direct = rast.render_backward(st, g, {"rgb": _cat(d_views, "rgb", dev), "alpha": _cat(d_views, "alpha", dev)})
    st.release()
    assert torch.equal(out["rgb"], rgb.detach()) and torch.equal(out["alpha"], alpha.detach())
    for k, a in zip(KEYS, got):
        b = direct[k]
        assert (a - b).abs().max().item() <= 1e-5 * max(b.abs().max().item(), 1e-30), k


def test_second_backward_through_one_render_is_refused(rast, dev, scene):
    from paper_2501_08174_gb300 import render
    leaves = _leaves(scene["gaussians"], dev)
    rgb, alpha, _, _ = render(rast, leaves, scene["cameras"])
    loss = rgb.sum() + alpha.sum()
    loss.backward(retain_graph=True)
    first = leaves["opacity"].grad.clone()
    assert float(first.abs().max()) > 0
    with pytest.raises(RuntimeError, match="released"):
        loss.backward()


def test_in_place_change_between_forward_and_backward_is_refused(rast, dev, scene):
    from paper_2501_08174_gb300 import render
    leaves = _leaves(scene["gaussians"], dev)
    rgb, _, _, _ = render(rast, leaves, scene["cameras"])
    with torch.no_grad():
        leaves["opacity"].mul_(0.5)  # e.g. an optimiser step before the backward
    with pytest.raises(RuntimeError, match="modified by an inplace operation"):
        rgb.sum().backward()
