"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Sizes are small enough for the oracle to finish in seconds yet span several
tiles with ragged image edges.  Pixels where the oracle reports that an FP32
evaluation may take a discrete decision the other way (a candidate within a
relative 1e-5 of the rho = 9 cut, the 1/255 floor, the 1e-4 transmittance
stop or the filter/surfel switch) are excluded and counted; they must stay a
small fraction.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from _helpers import (FWD_TOL, KEYS, OUT_KEYS, forward_errors, gpu_at, grad_errors, masked, oracle_adjoint,
                      to_device, worst_element)

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
    r = Rasterizer(dev)
    yield r
    r.close()


def _render_np(rast, g, cams):
    out, state = rast.render(g, cams)
    torch.cuda.synchronize()
    return out, state


@pytest.mark.parametrize("seed,n,w,h,deg", [(101, 600, 70, 45, 1), (102, 900, 53, 61, 3), (103, 300, 33, 17, 0),
                                            (104, 1500, 96, 72, 2)])
def test_forward_matches_oracle(rast, dev, seed, n, w, h, deg):
    sc = synthetic.small_scene(seed, n, w, h, degree=deg)
    g_np, cam = sc["gaussians"], sc["cameras"][0]
    out, _ = _render_np(rast, to_device(g_np, dev), [cam])
    ref = oracle.render(g_np, cam)
    ok = ~ref["fragile"]
    assert ok.mean() > 0.98
    errs = forward_errors(gpu_at(out, np.arange(w * h)), ref, ok)
    assert max(errs.values()) <= FWD_TOL, errs
    assert ref["alpha"].max() > 0.5  # the scene is not empty
    tf = out["alpha"].double().cpu().numpy()
    np.testing.assert_allclose(1.0 - tf, ref["t_final"], atol=FWD_TOL)


def test_forward_config1_and_background_loss(rast, dev):
    sc = synthetic.config1()
    g_np, cam, mask = sc["gaussians"], sc["cameras"][0], sc["masks"][0]
    out, _ = _render_np(rast, to_device(g_np, dev), [cam])
    ref = oracle.render(g_np, cam)
    ok = ~ref["fragile"]
    errs = forward_errors(gpu_at(out, np.arange(128 * 128)), ref, ok)
    assert max(errs.values()) <= FWD_TOL, errs
    m = torch.tensor(mask.reshape(-1), device=dev)
    d_alpha = torch.zeros(128 * 128, device=dev)
    loss = rast.background_loss(out["alpha"], m, [cam], gamma=0.5, d_alpha=d_alpha).item()
    a = out["alpha"].double().cpu().numpy().reshape(128, 128)
    assert loss == pytest.approx(oracle.background_loss(a, mask), rel=1e-12, abs=1e-15)
    np.testing.assert_allclose(d_alpha.cpu().numpy().reshape(128, 128), oracle.background_loss_grad(mask, 0.5),
                               rtol=1e-6, atol=0)
    ref_loss = oracle.background_loss(ref["alpha"].reshape(128, 128), mask)
    assert abs(loss - ref_loss) <= FWD_TOL


@pytest.mark.parametrize("seed,n,w,h,deg", [(201, 500, 48, 40, 2), (202, 300, 37, 29, 3), (203, 200, 20, 36, 0)])
def test_backward_matches_oracle_adjoint(rast, dev, seed, n, w, h, deg):
    sc = synthetic.small_scene(seed, n, w, h, degree=deg)
    g_np, cam = sc["gaussians"], sc["cameras"][0]
    g = to_device(g_np, dev)
    out, state = _render_np(rast, g, [cam])
    P = w * h
    rng = np.random.default_rng(seed)
    d_out = dict(rgb=rng.normal(size=(P, 3)), alpha=rng.normal(size=P), depth=rng.normal(size=P),
                 normal=rng.normal(size=(P, 3)))
    probe = oracle.render(g_np, cam)
    ok = ~probe["fragile_grad"]
    assert ok.mean() > 0.97
    d_out = {k: masked(v, ok) for k, v in d_out.items()}
    ref, ref32 = oracle_adjoint(g_np, cam, d_out)
    grads = rast.render_backward(state, g, {k: torch.tensor(v, dtype=torch.float32, device=dev)
                                            for k, v in d_out.items()})
    errs = grad_errors(grads, ref, ref32)
    assert max(errs.values()) <= 1.0, (errs, {k: worst_element(grads, ref, k, ref32) for k in KEYS})


def test_backward_single_plane_cotangents(rast, dev):
    """Each output plane alone (others NULL) gives the oracle's gradient of that plane."""
    sc = synthetic.small_scene(211, 400, 40, 32, degree=1)
    g_np, cam = sc["gaussians"], sc["cameras"][0]
    g = to_device(g_np, dev)
    out, state = _render_np(rast, g, [cam])
    P = 40 * 32
    rng = np.random.default_rng(5)
    ok = ~oracle.render(g_np, cam)["fragile_grad"]
    full = dict(rgb=rng.normal(size=(P, 3)), alpha=rng.normal(size=P), depth=rng.normal(size=P),
                normal=rng.normal(size=(P, 3)))
    for key in OUT_KEYS:
        d = {k: (masked(v, ok) if k == key else np.zeros_like(v)) for k, v in full.items()}
        ref, ref32 = oracle_adjoint(g_np, cam, d)
        grads = rast.render_backward(state, g, {key: torch.tensor(d[key], dtype=torch.float32, device=dev)})
        errs = grad_errors(grads, ref, ref32)
        # opacity-only and colour-only planes leave some parameter groups at exactly zero
        errs = {k: e for k, e in errs.items() if np.abs(ref[k]).max() > 0}
        assert max(errs.values()) <= 1.0, (key, errs)


def test_tile_shapes_and_persistent_queue_give_identical_results(dev):
    from paper_2501_08174_gb300 import Rasterizer
    sc = synthetic.small_scene(301, 800, 77, 51, degree=2, n_views=3)
    g = to_device(sc["gaussians"], dev)
    cams = sc["cameras"]
    base = None
    combos = [(t, k, 32) for t in ((16, 16), (16, 8), (8, 8), (32, 8)) for k in (1, 2)] + [((16, 16), 4, 32)]
    # Gaussians per batch where the shape offers it
    combos += [((16, 16), 4, 16), ((16, 16), 4, 64), ((16, 16), 2, 16), ((16, 16), 2, 64), ((16, 8), 4, 16),
               ((16, 8), 4, 64)]
    for tile, ppt, batch in combos:
        for persistent in (False, True):
            r = Rasterizer(dev, tile=tile, persistent=persistent, pixels_per_thread=ppt, batch=batch)
            score = torch.zeros(len(sc["gaussians"]["opacity"]), device=dev)
            out, _ = r.render(g, cams, score=score, keep_state=False)
            torch.cuda.synchronize()
            cur = {k: v.cpu() for k, v in out.items()}
            cur["score"] = score.cpu()
            if base is None:
                base = cur
            else:
                for k in base:
                    assert torch.equal(base[k], cur[k]), (tile, ppt, batch, persistent, k)
            r.close()
    # the two-pass split of persistent renders
    for front in (0.0, 0.02, 0.3, 1.0):
        r = Rasterizer(dev, tile=(16, 16), persistent=True, pixels_per_thread=4, front_fraction=front)
        score = torch.zeros(len(sc["gaussians"]["opacity"]), device=dev)
        out, _ = r.render(g, cams, score=score, keep_state=False)
        torch.cuda.synchronize()
        cur = {k: v.cpu() for k, v in out.items()}
        cur["score"] = score.cpu()
        for k in base:
            assert torch.equal(base[k], cur[k]), (front, k)
        r.close()


def test_batched_views_equal_per_view_launches(rast, dev):
    sc = synthetic.small_scene(401, 700, 64, 48, degree=3, n_views=4)
    sc["cameras"][1] = synthetic.make_camera(sc["cameras"][1]["viewmat"][:3, :3].T @ -sc["cameras"][1]["viewmat"][:3, 3], 40, 56)
    g = to_device(sc["gaussians"], dev)
    cams = sc["cameras"]
    out_b, st_b = rast.render(g, cams)
    P = sum(c["width"] * c["height"] for c in cams)
    rng = np.random.default_rng(1)
    d_np = dict(rgb=rng.normal(size=(P, 3)), alpha=rng.normal(size=P), depth=rng.normal(size=P),
                normal=rng.normal(size=(P, 3)))
    d = {k: torch.tensor(v, dtype=torch.float32, device=dev) for k, v in d_np.items()}
    gb = rast.render_backward(st_b, g, d)
    off = 0
    gsum = {k: torch.zeros_like(g[k]) for k in KEYS}
    for cam in cams:
        n = cam["width"] * cam["height"]
        o, st = rast.render(g, [cam])
        for k in OUT_KEYS:
            assert torch.equal(o[k], out_b[k][off:off + n]), k
        rast.render_backward(st, g, {k: v[off:off + n].contiguous() for k, v in d.items()}, grads=gsum)
        off += n
    torch.cuda.synchronize()
    for k in KEYS:
        a, b = gb[k].double(), gsum[k].double()
        assert (a - b).abs().max().item() <= 1e-5 * max(b.abs().max().item(), 1e-30), k


def test_contribution_score_matches_oracle(rast, dev):
    sc = synthetic.small_scene(501, 3000, 48, 40, degree=1, n_views=3, scale_range=(0.08, 0.3))
    g_np = sc["gaussians"]
    score = rast.accumulate_contribution(to_device(g_np, dev), sc["cameras"]).cpu().numpy()
    refs = [oracle.render(g_np, c) for c in sc["cameras"]]
    ref = np.max([r["score"] for r in refs], axis=0)
    assert sum(r["fragile"].sum() for r in refs) < 0.01 * sum(r["fragile"].size for r in refs)
    assert np.abs(score - ref).max() <= 1e-5
    assert ((score > 0) == (ref > 0)).all()
    assert (ref == 0).sum() > 10  # some surfels are hidden or off screen


def test_prune_keep_set_and_compaction(rast, dev):
    sc = synthetic.small_scene(601, 2000, 56, 56, degree=2, n_views=4, scale_range=(0.05, 0.25))
    g_np = sc["gaussians"]
    g = to_device(g_np, dev)
    score = rast.accumulate_contribution(g, sc["cameras"])
    ref_score = np.max([oracle.render(g_np, c)["score"] for c in sc["cameras"]], axis=0)
    tau = 0.01
    keep_ref, near_ref = oracle.keep_set(ref_score, tau)
    kept, border, n_border = rast.prune(g, score, tau)
    s = score.cpu().numpy()
    keep_gpu = s > tau
    near = np.abs(ref_score - tau) <= 1e-6
    assert (keep_gpu[~near] == keep_ref[~near]).all()
    np.testing.assert_array_equal(np.sort(border.cpu().numpy()), np.nonzero(np.abs(s - tau) <= 1e-6)[0])
    for k in KEYS:
        np.testing.assert_array_equal(kept[k].cpu().numpy(), np.asarray(g_np[k], np.float32)[keep_gpu])
    # the paper's rule: threshold 0 keeps exactly the surfels used in blending
    kept0, _, _ = rast.prune(g, score, 0.0)
    assert kept0["xyz"].shape[0] == int((ref_score > 0).sum())


# ----------------------------------------------------------------------------- edge cases
def test_empty_scene_renders_background(rast, dev):
    cam = synthetic.make_camera((0, -3, 0), 33, 21)
    g = {k: torch.zeros((0,) + s, device=dev) for k, s in
         (("xyz", (3,)), ("quat", (4,)), ("scale", (2,)), ("opacity", ()), ("sh", (1, 3)))}
    out, st = rast.render(g, [cam])
    torch.cuda.synchronize()
    assert out["alpha"].abs().max().item() == 0 and out["rgb"].abs().max().item() == 0
    grads = rast.render_backward(st, g, {"alpha": torch.ones(33 * 21, device=dev)})
    assert grads["xyz"].numel() == 0


def test_invalid_arguments_are_rejected(rast, dev):
    from paper_2501_08174_gb300 import OcgsError
    sc = synthetic.small_scene(701, 50, 16, 16)
    g = to_device(sc["gaussians"], dev)
    bad = dict(sc["cameras"][0])
    bad["width"] = 0
    with pytest.raises(OcgsError, match="ERR_ARG"):
        rast.render(g, [bad])
    bad = dict(sc["cameras"][0])
    bad["near"] = 0.0
    with pytest.raises(OcgsError, match="ERR_ARG"):
        rast.render(g, [bad])
    with pytest.raises(OcgsError, match="ERR_ARG"):
        rast.set_options(tile=(12, 12))
    rast.set_options(tile=(16, 16))


def test_nonfinite_parameters_are_reported_and_skipped(rast, dev):
    sc = synthetic.small_scene(702, 300, 32, 32, degree=1)
    g_np = {k: (np.array(v, copy=True) if k != "sh_degree" else v) for k, v in sc["gaussians"].items()}
    g_np["xyz"][7, 1] = np.nan
    from paper_2501_08174_gb300 import OcgsError
    with pytest.raises(OcgsError, match="NONFINITE"):
        rast.render(to_device(g_np, dev), sc["cameras"])
    # the same image as without that surfel
    keep = np.ones(300, bool)
    keep[7] = False
    g2 = {k: np.asarray(v)[keep] for k, v in g_np.items() if k != "sh_degree"}
    out2, _ = rast.render(to_device(g2, dev), sc["cameras"], keep_state=False)
    assert torch.isfinite(out2["rgb"]).all()


def test_surfel_behind_camera_and_edge_on(rast, dev):
    cam = synthetic.make_camera((0.0, -3.0, 0.0), 41, 41)
    q_face = [np.cos(np.pi / 4), np.sin(np.pi / 4), 0, 0]
    q_edge = [1.0, 0.0, 0.0, 0.0]  # normal +z: seen exactly edge-on from the -y axis
    sh = lambda rgb: ((np.asarray(rgb) - 0.5) * 2 * np.sqrt(np.pi)).reshape(1, 3)
    g_np = dict(xyz=np.array([[0, -4.0, 0], [0.1, 0.0, 0.05], [-0.2, 0.3, 0.1]]),
                quat=np.array([q_face, q_edge, q_face]), scale=np.array([[0.3, 0.3], [0.2, 0.2], [0.1, 0.05]]),
                opacity=np.array([0.9, 0.8, 0.7]), sh=np.stack([sh([1, 0, 0]), sh([0, 1, 0]), sh([0, 0, 1])]),
                sh_degree=0)
    out, _ = _render_np(rast, to_device(g_np, dev), [cam])
    ref = oracle.render(g_np, cam)
    ok = ~ref["fragile"]
    errs = forward_errors(gpu_at(out, np.arange(41 * 41)), ref, ok)
    assert max(errs.values()) <= FWD_TOL, errs
    assert ref["alpha"].max() > 0.1


def test_autotune_picks_valid_options_and_caches_them(dev, tmp_path):
    from paper_2501_08174_gb300 import Rasterizer
    sc = synthetic.small_scene(801, 1200, 96, 80, degree=2, n_views=2)
    g = to_device(sc["gaussians"], dev)
    r = Rasterizer(dev)
    before, _ = r.render(g, sc["cameras"], keep_state=False)
    before = {k: v.clone() for k, v in before.items()}
    cache = tmp_path / "tune.txt"
    res = r.autotune(g, sc["cameras"], cache_path=cache)
    assert res["n_tried"] >= 14 and not res["from_cache"] and res["ms"] > 0
    assert res["batch"] in (16, 32, 64) and 0.0 <= res["front_fraction"] <= 1.0
    after, _ = r.render(g, sc["cameras"], keep_state=False)
    torch.cuda.synchronize()
    for k in OUT_KEYS:  # options change the time, never the result
        assert torch.equal(before[k], after[k]), k
    r2 = Rasterizer(dev)
    res2 = r2.autotune(g, sc["cameras"], cache_path=cache)
    assert res2["from_cache"] and res2["tile"] == res["tile"] and res2["pixels_per_thread"] == res["pixels_per_thread"]
    assert res2["batch"] == res["batch"] and res2["front_fraction"] == pytest.approx(res["front_fraction"])
    assert r2.options() == dict(tile=res["tile"], persistent=res["persistent"],
                                pixels_per_thread=res["pixels_per_thread"], front_fraction=res2["front_fraction"],
                                batch=res["batch"])
    r.close()
    r2.close()


def test_captured_sweep_equals_eager_sweep_and_reports_overflow(dev):
    from paper_2501_08174_gb300 import OcgsError, Rasterizer
    sc = synthetic.small_scene(901, 3000, 64, 48, degree=1, n_views=20, scale_range=(0.05, 0.2))
    g = to_device(sc["gaussians"], dev)
    cams = sc["cameras"]
    for opts in (dict(), dict(tile=(16, 8), persistent=False, pixels_per_thread=2)):
        r = Rasterizer(dev, **opts)
        eager = r.accumulate_contribution(g, cams).clone()
        graph = r.contribution_graph(g, cams, headroom=1.0)
        got = graph.launch()
        r.sync()
        assert torch.equal(got, eager)
        got.fill_(7.0)  # the graph zeroes the score itself
        graph.launch()
        r.sync()
        assert torch.equal(got, eager)
        # parameters change in place between launches: the graph sees the new values
        g["opacity"].mul_(0.5)
        graph.launch()
        r.sync()
        assert torch.equal(graph.score, r.accumulate_contribution(g, cams))
        g["opacity"].mul_(2.0)
        # larger surfels need more pairs than the capacity: reported, not faulted
        g["scale"].mul_(3.0)
        graph.launch()
        with pytest.raises(OcgsError, match="CAPACITY"):
            r.sync()
        g["scale"].div_(3.0)
        graph.close()
        r.close()


@pytest.mark.parametrize("opts", [dict(), dict(tile=(16, 16), persistent=True, pixels_per_thread=4)])
def test_config3_geometry_keep_set_matches_oracle(dev, opts):
    """Config 3's geometry scaled down (three closed tangent shells of 900 surfels around 400
    interior surfels, 8 hemisphere views of 64x64).  Scores are compared within 1e-5 and the
    keep-set at tau = 0.01 exactly (borderline scores listed) for every surfel whose score is
    certain in float32: not itself at a fragile threshold at any pixel and with its largest
    weight at a firm pixel; the others (listed, a few percent at most) keep their firm lower
    bound.  The paper's rule (tau = 0) is checked the same way, and the interior hidden behind
    the shells is pruned."""
    from paper_2501_08174_gb300 import Rasterizer
    sc = synthetic.config3(seed=33, n_views=8, width=64, height=64, shell_counts=(900, 900, 900),
                           n_interior=400, shell_scale=(0.09, 0.12))
    g_np = sc["gaussians"]
    refs = [oracle.render(g_np, c) for c in sc["cameras"]]
    ref = np.max([r["score"] for r in refs], axis=0)
    firm = np.max([r["score_firm"] for r in refs], axis=0)
    uncertain = np.any([r["at_edge"] for r in refs], axis=0) | (ref > firm)
    assert sum(r["fragile"].sum() for r in refs) < 0.01 * sum(r["fragile"].size for r in refs)
    assert uncertain.mean() < 0.03, int(uncertain.sum())
    r = Rasterizer(dev, **opts)
    g = to_device(g_np, dev)
    score = r.accumulate_contribution(g, sc["cameras"])
    s = score.cpu().numpy()
    sure = ~uncertain
    assert np.abs(s - ref)[sure].max() <= 1e-5
    assert (s[uncertain] >= firm[uncertain] - 1e-5).all()
    tau = 0.01
    keep_ref, near_ref = oracle.keep_set(ref, tau)
    kept, border, n_border = r.prune(g, score, tau)
    keep_gpu = s > tau
    near = np.abs(ref - tau) <= 1e-6
    checked = sure & ~near
    assert (keep_gpu[checked] == keep_ref[checked]).all(), np.nonzero(keep_gpu[checked] != keep_ref[checked])
    np.testing.assert_array_equal(np.sort(border.cpu().numpy()), np.nonzero(np.abs(s - tau) <= 1e-6)[0])
    kept_ref = oracle.prune(g_np, keep_gpu)
    for k in KEYS:
        np.testing.assert_array_equal(kept[k].cpu().numpy(), np.asarray(kept_ref[k], np.float32))
    assert ((s > 0) == (ref > 0))[sure].all()          # the paper's "used in blending" rule
    interior = slice(sc["n_shell"], None)
    assert not keep_gpu[interior].any() and keep_ref[:sc["n_shell"]].mean() > 0.5
    r.close()
