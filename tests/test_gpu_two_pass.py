"""Two-pass binning of persistent renders (the front of the depth order first,
then the tiles left open, rendered again from their complete lists): every
result equals the one-pass render's.

Forward planes, blending positions and contribution scores are compared bit for
bit.  Parameter gradients are sums of per-tile atomic additions whose order
follows the tile queue, so they are compared to 1e-5 of each group's largest
entry.
"""
import numpy as np
import pytest
import torch

import synthetic
from _helpers import KEYS, to_device

pytestmark = pytest.mark.gpu

FRACTIONS = (0.0, 1e-6, 0.02, 0.08, 0.3, 1.0)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_08174_gb300 import build
    build.build()
    return torch.device("cuda", 0)


def opaque_scene(seed=901, n=40_000, views=((0.0, -3.0, 0.0), (2.1, -2.1, 0.4), (0.3, 0.5, 2.9)),
                 sizes=((128, 96), (97, 75), (80, 80))):
    """An opaque object ball inside a sparse background shell: the ball's tiles stop early, the
    background's run to the end of their lists."""
    rng = np.random.default_rng(seed)
    g = synthetic.object_scene(rng, n, 1)
    cams = [synthetic.make_camera(np.array(p), w, h) for p, (w, h) in zip(views, sizes)]
    return g, cams


def _run(dev, g, cams, fraction, tile=(16, 16), ppt=4, d_out=None):
    from paper_2501_08174_gb300 import Rasterizer, n_pixels
    r = Rasterizer(dev, tile=tile, persistent=True, pixels_per_thread=ppt, front_fraction=fraction)
    n = g["opacity"].shape[0]
    score = torch.zeros(n, device=dev)
    out, st = r.render(g, cams, score=score, depth2=True)
    res = {k: v.clone() for k, v in out.items()}
    res["score"] = score
    res["n_evals"] = st.info()["n_evals"]
    res["n_pairs"] = r.stats()["n_pairs"]
    if d_out is not None:
        res["grads"] = r.render_backward(st, g, d_out)
    st.release()
    torch.cuda.synchronize()
    r.close()
    return res


def _cotangents(dev, P, seed):
    gen = torch.Generator(device="cpu").manual_seed(seed)
    return {k: torch.randn(shape, generator=gen).to(dev) for k, shape in
            (("rgb", (P, 3)), ("alpha", (P,)), ("depth", (P,)), ("normal", (P, 3)), ("depth2", (P,)))}


def test_two_pass_equals_one_pass(dev):
    from paper_2501_08174_gb300 import n_pixels
    gn, cams = opaque_scene()
    g = to_device(gn, dev)
    d_out = _cotangents(dev, n_pixels(cams), 5)
    base = _run(dev, g, cams, 0.0, d_out=d_out)
    for f in FRACTIONS[1:]:
        cur = _run(dev, g, cams, f, d_out=d_out)
        for k in ("rgb", "alpha", "depth", "normal", "depth2", "score"):
            assert torch.equal(base[k], cur[k]), (f, k)
        assert cur["n_evals"] == base["n_evals"], f
        for k in KEYS:
            a, b = base["grads"][k], cur["grads"][k]
            assert float((a - b).abs().max()) <= 1e-5 * float(a.abs().max()) + 1e-30, (f, k)
        if f == 1.0:
            assert cur["n_pairs"] == base["n_pairs"]


def test_two_pass_bins_fewer_pairs_behind_an_opaque_ball(dev):
    """Without the background shell the front of the depth order is the ball's near side, which
    stops the interior tiles: fewer pairs in all, the same images."""
    rng = np.random.default_rng(904)
    gn = synthetic.object_scene(rng, 40_000, 1, object_frac=1.0)
    cams = [synthetic.make_camera(np.array(p), 256, 256) for p in ((0.0, -3.0, 0.0), (2.1, -2.1, 0.4))]
    g = to_device(gn, dev)
    base = _run(dev, g, cams, 0.0)
    cur = _run(dev, g, cams, 0.3)
    for k in ("rgb", "alpha", "depth", "normal", "depth2", "score"):
        assert torch.equal(base[k], cur[k]), k
    assert cur["n_pairs"] < base["n_pairs"], (cur["n_pairs"], base["n_pairs"])


@pytest.mark.parametrize("tile,ppt", [((16, 8), 2), ((8, 8), 1), ((32, 8), 2)])
def test_two_pass_other_tile_shapes(dev, tile, ppt):
    gn, cams = opaque_scene(seed=902, n=15_000)
    g = to_device(gn, dev)
    base = _run(dev, g, cams, 0.0, tile=tile, ppt=ppt)
    cur = _run(dev, g, cams, 0.05, tile=tile, ppt=ppt)
    for k in ("rgb", "alpha", "depth", "normal", "depth2", "score"):
        assert torch.equal(base[k], cur[k]), k


def test_two_pass_pruning_sweeps_equal_one_pass(dev):
    """The image-free sweeps (2DGS and the 3DGS variant) continue from T and the stop flags alone."""
    from paper_2501_08174_gb300 import Rasterizer
    gn, cams = opaque_scene(seed=905, n=30_000)
    g = to_device(gn, dev)
    rng = np.random.default_rng(906)
    g3 = dict(g)
    g3["scale"] = torch.cat([g["scale"], torch.tensor(np.exp(rng.uniform(np.log(0.01), np.log(0.1),
                                                                         size=(len(gn["opacity"]), 1))),
                                                      dtype=torch.float32, device=dev)], 1).contiguous()
    res = {}
    for f in (0.0, 0.05, 0.3):
        r = Rasterizer(dev, tile=(16, 16), persistent=True, pixels_per_thread=4, front_fraction=f)
        res[f] = (r.accumulate_contribution(g, cams), r.accumulate_contribution_3d(g3, cams))
        torch.cuda.synchronize()
        r.close()
    for f in (0.05, 0.3):
        assert torch.equal(res[0.0][0], res[f][0]), f
        assert torch.equal(res[0.0][1], res[f][1]), f
    assert float(res[0.0][0].max()) > 0.5 and float(res[0.0][1].max()) > 0.5


def test_two_pass_with_nothing_visible(dev):
    """Every Gaussian behind the camera: no record has a screen box, the first pass is the
    whole render and the image is background."""
    gn, _ = opaque_scene(seed=903, n=500)
    gn = dict(gn)
    gn["xyz"] = np.asarray(gn["xyz"]) * 0.1 + np.array([0.0, -5.0, 0.0])
    cams = [synthetic.make_camera(np.array([0.0, -3.0, 0.0]), 40, 30)]
    g = to_device(gn, dev)
    cur = _run(dev, g, cams, 0.08)
    assert cur["n_pairs"] == 0
    assert float(cur["alpha"].abs().max()) == 0.0


def test_front_fraction_is_checked(dev):
    from paper_2501_08174_gb300 import Rasterizer, _lib
    r = Rasterizer(dev)
    for bad in (-0.1, 1.5, float("nan")):
        with pytest.raises(_lib.OcgsError) as e:
            r.set_options(tile=(16, 16), persistent=True, pixels_per_thread=4, front_fraction=bad)
        assert e.value.code == _lib.ERR_ARG
    r.close()
