"""Tile binning of a thin support ellipse (an almost edge-on surfel), Sec. 4.3.

The binning keeps a (tile, surfel) pair only where the surfel's support
{rho <= rb}, bounded by a conic, reaches a pixel centre of the tile.  For a
surfel seen nearly edge-on the conic is a thin ellipse, and its determinant
a c - b^2 taken as a difference of products keeps only a few correct digits in
FP32: for the surfel below it came out 3.7 % too large and the support's tip
0.9 px too short.  The camera here puts that tip, where the FP64 definition
still blends alpha of about 0.0066, at the top rows of a tile that no other part
of the support reaches, so a binning that loses the tip leaves those pixels
empty.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from _helpers import FWD_TOL, forward_errors, gpu_at, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_08174_gb300 import build
    build.build()
    return torch.device("cuda", 0)


def _edge_on_scene():
    """Surfel 430675 of the 500k-surfel, 16-view scene (seed 4) and its view 9 (1600 x 1200),
    with the principal point moved up 9 px: the support's tip, rows 1129-1130 of that view,
    becomes rows 1120-1121, the first rows of a tile row."""
    cam = synthetic.make_camera([0.6569143762968417, 2.2229545214543696, 1.9044518103013544], 1600, 1200)
    cam["cy"] = cam["cy"] - 9.0
    g = dict(xyz=np.array([[1.6903904676437378, -1.0359622240066528, -2.7195851802825928]], np.float32),
             quat=np.array([[0.8243237733840942, 0.19206833839416504, 0.4418884515762329,
                             -0.2972114682197571]], np.float32),
             scale=np.array([[0.010471999645233154, 0.07593058794736862]], np.float32),
             opacity=np.array([0.585666835308075], np.float32),
             sh=np.array([[[1.2, 0.8, 0.4]]], np.float32), sh_degree=0)
    return g, cam


@pytest.mark.parametrize("tile", [(16, 16), (16, 8)])
def test_thin_support_tip_is_binned(dev, tile):
    from paper_2501_08174_gb300 import Rasterizer
    g_np, cam = _edge_on_scene()
    W = cam["width"]
    ys, xs = np.meshgrid(np.arange(1116, 1126), np.arange(224, 256), indexing="ij")
    pix = (ys * W + xs).reshape(-1)
    ref = oracle.render(g_np, cam, pixels=pix)
    tip = (ys.reshape(-1) >= 1120) & (ref["alpha"] > 1.0 / 255.0)
    assert tip.sum() >= 1 and ref["alpha"][pix == 1120 * W + 238] > 0.006  # the case is the one described
    r = Rasterizer(dev, tile=tile)
    out, st = r.render(to_device(g_np, dev), [cam])
    torch.cuda.synchronize()
    gpu = gpu_at(out, pix)
    st.release()
    r.close()
    ok = ~ref["fragile"]
    assert ok[tip].all()
    errs = forward_errors(gpu, ref, ok)
    assert max(errs.values()) <= FWD_TOL, errs


@pytest.fixture(scope="module")
def c4(dev):
    sc = synthetic.config4()
    return sc["gaussians"], sc["cameras"]


def _render_both(dev, render, n):
    """render(rast, score) under the exact coverage, then with every tile of each record's
    screen rectangle: (outputs, score, pairs) of each."""
    from paper_2501_08174_gb300 import Rasterizer
    r = Rasterizer(dev, tile=(16, 16), persistent=True, pixels_per_thread=4)
    res = []
    for rect in (False, True):
        r.set_coverage(rect)
        score = torch.zeros(n, device=dev)
        out = render(r, score)
        torch.cuda.synchronize()
        res.append(({k: v.cpu() for k, v in out.items()}, score.cpu(), r.stats()["n_pairs"]))
    r.close()
    return res


@pytest.mark.parametrize("front", [0.1, 0.0])
def test_support_test_drops_no_blend(dev, c4, front):
    """On the 500k-surfel, 16-view scene, binning every tile of each record's screen rectangle
    and staging every record for every band (no support test) renders the same bits and the
    same contribution record as the exact coverage: the support test drops only pairs that
    blend no pixel.  One pass and two passes."""
    g_np, cams = c4
    g = to_device(g_np, dev)

    def render(r, score):
        r.set_options(tile=(16, 16), persistent=True, pixels_per_thread=4, front_fraction=front)
        out, st = r.render(g, cams, score=score)
        st.release()
        return out

    (a, sa, ka), (b, sb, kb) = _render_both(dev, render, g_np["opacity"].shape[0])
    assert kb > 1.5 * ka, (ka, kb)
    for k in a:
        assert torch.equal(a[k], b[k]), k
    assert torch.equal(sa, sb)


def test_support_test_drops_no_blend_3d(dev, c4):
    """The same for the 3DGS variant (Appendix B): projected 3D Gaussians, whose support
    conic is the covariance's."""
    g_np, cams = c4
    rng = np.random.default_rng(44)
    n = g_np["opacity"].shape[0]
    third = np.exp(rng.uniform(np.log(0.01), np.log(0.1), size=(n, 1)))
    g3 = dict(g_np, scale=np.concatenate([np.asarray(g_np["scale"], np.float64), third], 1))
    g = {k: torch.tensor(np.asarray(g3[k], np.float32), device=dev) for k in ("xyz", "quat", "scale", "opacity", "sh")}

    def render(r, score):
        return r.render_3d(g, cams, score=score)

    (a, sa, ka), (b, sb, kb) = _render_both(dev, render, n)
    assert kb > ka, (ka, kb)
    for k in ("rgb", "alpha", "depth"):
        assert torch.equal(a[k], b[k]), k
    assert torch.equal(sa, sb)


def test_support_test_drops_no_blend_1m_64views(dev):
    """The same check on the 1M-surfel, 64-view scene (1600x1200 views; 40 % of the surfels on
    tangent shells, many seen almost edge-on), in two passes with the Q plane as the training
    iteration renders it."""
    sc = synthetic.config5()
    g_np, cams = sc["gaussians"], sc["cameras"]
    g = to_device(g_np, dev)

    def render(r, score):
        out, st = r.render(g, cams, score=score, depth2=True)
        st.release()
        return out

    (a, sa, ka), (b, sb, kb) = _render_both(dev, render, g_np["opacity"].shape[0])
    assert kb > ka, (ka, kb)
    for k in a:
        assert torch.equal(a[k], b[k]), k
    assert torch.equal(sa, sb)
