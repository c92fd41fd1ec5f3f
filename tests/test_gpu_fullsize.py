"""Full-size workloads on the GPU, in the launch configuration bench.py times
(16x16 tiles, 4 pixels per thread, persistent tile queue).

The FP64 oracle cannot render whole 500k-surfel frames, so it is evaluated on
seeded pixel samples: forward outputs element by element at the samples, and
gradients of losses whose cotangents are non-zero only at the samples (the
same loss on both sides).  Whole-frame properties (Sum w + T = 1 via alpha,
score bounds, batched == chunked sweeps) are checked at every pixel.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from _helpers import (FWD_TOL, GRAD_TOL, KEYS, OUT_KEYS, add_grads, forward_errors, grad_errors, oracle_adjoint,
                      to_device, worst_element)

pytestmark = pytest.mark.gpu

BENCH_OPTS = dict(tile=(16, 16), persistent=True, pixels_per_thread=4)


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
    r = Rasterizer(dev, **BENCH_OPTS)
    yield r
    r.close()


def _sample(cam, n, seed):
    rng = np.random.default_rng(seed)
    P = cam["width"] * cam["height"]
    return np.sort(rng.choice(P, size=n, replace=False))


def _gather(out, idx):
    t = torch.as_tensor(idx, device=out["alpha"].device)
    return {k: out[k][t].double().cpu().numpy() for k in OUT_KEYS}


@pytest.fixture(scope="module")
def c2(rast, dev):
    sc = synthetic.config2()
    g = to_device(sc["gaussians"], dev)
    out, state = rast.render(g, sc["cameras"])
    torch.cuda.synchronize()
    return sc, g, out, state


# ----------------------------------------------------------------------------- config 2: 100k surfels, 800x800, SH3
def test_c2_forward_at_sampled_pixels(c2):
    sc, g, out, _ = c2
    cam = sc["cameras"][0]
    px = _sample(cam, 1024, 20)
    ref = oracle.render(sc["gaussians"], cam, pixels=px)
    ok = ~ref["fragile"]
    assert ok.mean() > 0.98
    errs = forward_errors(_gather(out, px), ref, ok)
    assert max(errs.values()) <= FWD_TOL, errs
    a = out["alpha"]
    assert float(a.min()) >= 0.0 and float(a.max()) < 1.0 and bool(torch.isfinite(out["depth"]).all())


def test_c2_gradient_of_sampled_l1_plus_background_loss(rast, dev, c2):
    """Masked-L1 + 0.5 L_b, both restricted to a pixel sample, against the oracle adjoint."""
    sc, g, out, state = c2
    cam, mask = sc["cameras"][0], sc["masks"][0].reshape(-1)
    P = cam["width"] * cam["height"]
    px = _sample(cam, 512, 21)
    px = px[~oracle.render(sc["gaussians"], cam, pixels=px)["fragile_grad"]]
    rng = np.random.default_rng(22)
    target = rng.uniform(0.0, 1.0, size=(len(px), 3))
    c = out["rgb"][torch.as_tensor(px, device=dev)].double().cpu().numpy()
    d_rgb = np.sign(c - target) * mask[px, None] / (3 * len(px))
    d_alpha = 0.5 * (1.0 - mask[px]) / P
    d_ref = dict(rgb=d_rgb, alpha=d_alpha, depth=np.zeros(len(px)), normal=np.zeros((len(px), 3)))
    ref, ref32 = oracle_adjoint(sc["gaussians"], cam, d_ref, pixels=px)
    full_rgb = torch.zeros(P, 3, device=dev)
    full_a = torch.zeros(P, device=dev)
    idx = torch.as_tensor(px, device=dev)
    full_rgb[idx] = torch.tensor(d_rgb, dtype=torch.float32, device=dev)
    full_a[idx] = torch.tensor(d_alpha, dtype=torch.float32, device=dev)
    grads = rast.render_backward(state, g, {"rgb": full_rgb, "alpha": full_a})
    errs = grad_errors(grads, ref, ref32)
    assert max(errs.values()) <= 1.0, (errs, {k: worst_element(grads, ref, k, ref32) for k in KEYS})


def test_c2_gradient_against_central_differences(rast, dev, c2):
    """32 parameters: GPU gradient vs central differences of the FP64 oracle forward."""
    sc, g, out, state = c2
    cam = sc["cameras"][0]
    P = cam["width"] * cam["height"]
    px = _sample(cam, 96, 23)
    probe = oracle.render(sc["gaussians"], cam, pixels=px)
    px = px[~probe["fragile_grad"]]
    rng = np.random.default_rng(24)
    d = dict(rgb=rng.normal(size=(len(px), 3)), alpha=rng.normal(size=len(px)), depth=rng.normal(size=len(px)),
             normal=np.zeros((len(px), 3)))
    full = {k: torch.zeros((P,) + v.shape[1:], device=dev) for k, v in d.items()}
    idx = torch.as_tensor(px, device=dev)
    for k, v in d.items():
        full[k][idx] = torch.tensor(v, dtype=torch.float32, device=dev)
    grads = rast.render_backward(state, g, full)
    gnp = {k: grads[k].double().cpu().numpy().reshape(-1) for k in KEYS}
    params = {k: np.array(sc["gaussians"][k], np.float64, copy=True) for k in KEYS}
    params["sh_degree"] = sc["gaussians"]["sh_degree"]

    def loss(pp):
        r = oracle.render(pp, cam, pixels=px)
        return sum(float(np.sum(r[k] * d[k])) for k in ("rgb", "alpha", "depth", "normal")), r["n_blended"]

    base_sig = probe["n_blended"][~probe["fragile_grad"]]
    picks = []
    for k, n in (("xyz", 7), ("quat", 7), ("scale", 6), ("opacity", 6), ("sh", 6)):
        order = np.argsort(-np.abs(gnp[k]))[:60]
        picks += [(k, int(j)) for j in rng.choice(order, size=n, replace=False)]
    checked = 0
    for k, j in picks:
        flat = params[k].reshape(-1)
        x0 = flat[j]
        h = 1e-6 * max(1.0, abs(x0))
        flat[j] = x0 + h
        lp, sp = loss(params)
        flat[j] = x0 - h
        lm, sm = loss(params)
        flat[j] = x0
        if not (np.array_equal(sp, base_sig) and np.array_equal(sm, base_sig)):
            continue  # a discrete decision moved: no derivative there
        fd = (lp - lm) / (2 * h)
        floor = 1e-2 * np.abs(gnp[k]).max()
        assert abs(gnp[k][j] - fd) <= GRAD_TOL * max(abs(fd), floor), (k, j, gnp[k][j], fd)
        checked += 1
    assert checked >= 24


# ----------------------------------------------------------------------------- config 3: pruning sweep, 300k x 100 views
@pytest.fixture(scope="module")
def c3(rast, dev):
    sc = synthetic.config3()
    g = to_device(sc["gaussians"], dev)
    score = rast.accumulate_contribution(g, sc["cameras"])
    torch.cuda.synchronize()
    return sc, g, score


def test_c3_interior_is_pruned_and_keep_set_is_the_threshold(rast, c3):
    sc, g, score = c3
    s = score.cpu().numpy()
    assert s.min() >= 0.0 and s.max() <= 0.99 + 1e-7
    tau = 0.01
    interior = s[sc["n_shell"]:]
    assert (interior <= tau).mean() >= 0.99          # hidden behind three opaque shells
    assert (s[:60_000] > tau).mean() > 0.3            # the outer shell is seen where the hemisphere cameras look
    kept, border, n_border = rast.prune(g, score, tau)
    keep = s > tau
    assert kept["xyz"].shape[0] == int(keep.sum())
    np.testing.assert_array_equal(kept["opacity"].cpu().numpy(), sc["gaussians"]["opacity"][keep])
    np.testing.assert_array_equal(np.sort(border.cpu().numpy()), np.nonzero(np.abs(s - tau) <= 1e-6)[0])
    assert n_border == int((np.abs(s - tau) <= 1e-6).sum())


def test_c3_sweep_is_the_max_over_view_subsets(rast, dev, c3):
    sc, g, score = c3
    a = rast.accumulate_contribution(g, sc["cameras"][:37])
    b = rast.accumulate_contribution(g, sc["cameras"][37:])
    torch.cuda.synchronize()
    assert torch.equal(torch.maximum(a, b), score)


def test_c3_sampled_oracle_scores_are_lower_bounds(c3):
    """The oracle's max weight over a pixel sample can only be below the sweep's max over all pixels."""
    sc, g, score = c3
    s = score.cpu().numpy()
    for v in (0, 50):
        cam = sc["cameras"][v]
        px = _sample(cam, 256, 30 + v)
        ref = oracle.render(sc["gaussians"], cam, pixels=px)
        assert (ref["score"] <= s + 1e-5).all()
        seen = ref["score"] > 1e-3
        assert seen.sum() > 10


# ----------------------------------------------------------------------------- config 4: 500k x 16 uneven views
def test_c4_batched_forward_and_gradient_at_sampled_pixels(rast, dev):
    sc = synthetic.config4()
    cams = sc["cameras"]
    g = to_device(sc["gaussians"], dev)
    out, state = rast.render(g, cams)
    from paper_2501_08174_gb300 import pixel_offsets
    off = pixel_offsets(cams)
    P = off[-1]
    full = {k: torch.zeros((P, 3) if k in ("rgb", "normal") else (P,), device=dev) for k in OUT_KEYS}
    grads_ref, grads_ref32 = {}, {}
    rng = np.random.default_rng(40)
    worst = 0.0
    for v, cam in enumerate(cams):
        px = _sample(cam, 256, 400 + v)
        d = dict(rgb=rng.normal(size=(len(px), 3)), alpha=rng.normal(size=len(px)), depth=rng.normal(size=len(px)),
                 normal=rng.normal(size=(len(px), 3)))
        probe = oracle.render(sc["gaussians"], cam, pixels=px)
        keep = ~probe["fragile_grad"]  # give fragile pixels no cotangent on either side
        d = {k: np.where(keep.reshape((-1,) + (1,) * (x.ndim - 1)), x, 0.0) for k, x in d.items()}
        errs = forward_errors(_gather(out, px + off[v]), probe, ~probe["fragile"])
        worst = max(worst, max(errs.values()))
        ref, ref32 = oracle_adjoint(sc["gaussians"], cam, d, pixels=px)
        idx = torch.as_tensor(px + off[v], device=dev)
        for k in OUT_KEYS:
            full[k][idx] = torch.tensor(d[k], dtype=torch.float32, device=dev)
        grads_ref, grads_ref32 = add_grads(grads_ref, ref), add_grads(grads_ref32, ref32)
    assert worst <= FWD_TOL, worst
    grads = rast.render_backward(state, g, full)
    errs = grad_errors(grads, grads_ref, grads_ref32)
    assert max(errs.values()) <= 1.0, (errs, {k: worst_element(grads, grads_ref, k, grads_ref32) for k in KEYS})
    a = out["alpha"]
    assert float(a.min()) >= 0.0 and float(a.max()) < 1.0


# ----------------------------------------------------------------------------- config 5: training iteration, 1M x 64 views
def test_c5_training_iteration_at_sampled_pixels(rast, dev):
    """One full iteration at the config-5 size (1M surfels, 64 views 1600x1200) in the launch
    configuration bench.py times: the batched forward at sampled pixels against the oracle
    (128 pixels on each of eight views); the gradient of a colour + opacity loss restricted
    to those samples against the oracle adjoint (the backward instantiation without depth
    and normal cotangents, as in the training step); the Adam update against the oracle applied to the GPU's own gradient at
    sampled elements; the pruning of parameters and of both moments with one keep-set."""
    sc = synthetic.config5()
    cams = sc["cameras"]
    g_np = sc["gaussians"]
    g = to_device(g_np, dev)
    N = g["xyz"].shape[0]
    from paper_2501_08174_gb300 import pixel_offsets
    off = pixel_offsets(cams)
    P = off[-1]
    score = torch.zeros(N, device=dev)
    out, state = rast.render(g, cams, score=score)
    full_rgb = torch.zeros(P, 3, device=dev)
    full_alpha = torch.zeros(P, device=dev)
    grads_ref, grads_ref32 = {}, {}
    rng = np.random.default_rng(50)
    worst = 0.0
    for v in (0, 9, 18, 27, 36, 45, 54, 63):
        cam = cams[v]
        px = _sample(cam, 128, 500 + v)
        d = dict(rgb=rng.normal(size=(len(px), 3)), alpha=rng.normal(size=len(px)), depth=np.zeros(len(px)),
                 normal=np.zeros((len(px), 3)))
        probe = oracle.render(g_np, cam, pixels=px)
        keep = ~probe["fragile_grad"]  # no cotangent on either side at fragile pixels
        d = {k: np.where(keep.reshape((-1,) + (1,) * (x.ndim - 1)), x, 0.0) for k, x in d.items()}
        errs = forward_errors(_gather(out, px + off[v]), probe, ~probe["fragile"])
        worst = max(worst, max(errs.values()))
        ref, ref32 = oracle_adjoint(g_np, cam, d, pixels=px)
        idx = torch.as_tensor(px + off[v], device=dev)
        full_rgb[idx] = torch.tensor(d["rgb"], dtype=torch.float32, device=dev)
        full_alpha[idx] = torch.tensor(d["alpha"], dtype=torch.float32, device=dev)
        grads_ref, grads_ref32 = add_grads(grads_ref, ref), add_grads(grads_ref32, ref32)
    assert worst <= FWD_TOL, worst
    grads = rast.render_backward(state, g, {"rgb": full_rgb, "alpha": full_alpha})
    state.release()
    errs = grad_errors(grads, grads_ref, grads_ref32)
    assert max(errs.values()) <= 1.0, (errs, {k: worst_element(grads, grads_ref, k, grads_ref32) for k in KEYS})

    lr = dict(xyz=1.6e-4, quat=1e-3, scale=5e-3, opacity=5e-2, sh=2.5e-3)
    params = {k: v.clone() for k, v in g.items()}
    m = {k: torch.zeros_like(v) for k, v in g.items()}
    vv = {k: torch.zeros_like(v) for k, v in g.items()}
    rast.adam_step(params, grads, m, vv, lr, step=1)
    tau = 0.01
    kept = [rast.prune(d, score, tau)[0] for d in (params, m, vv)]
    torch.cuda.synchronize()
    sel = {k: torch.as_tensor(rng.choice(grads[k].numel(), size=4096, replace=False), device=dev) for k in KEYS}

    def at(d):
        return {k: d[k].reshape(-1)[sel[k]].double().cpu().numpy() for k in KEYS}

    z = {k: np.zeros(4096) for k in KEYS}
    p_o, m_o, v_o = oracle.adam_step(at(g), at(grads), z, z, lr, step=1)
    got_p, got_m = at(params), at(m)
    for k in KEYS:
        np.testing.assert_allclose(got_p[k], p_o[k], rtol=0, atol=2e-6, err_msg=k)
        np.testing.assert_allclose(got_m[k], m_o[k], rtol=1e-6, atol=1e-30, err_msg=k)
    keep = score > tau
    n_keep = int(keep.sum())
    assert 0 < n_keep < N
    for d, kd in zip((params, m, vv), kept):
        for k in KEYS:
            assert kd[k].shape[0] == n_keep
            assert torch.equal(kd[k], d[k][keep]), k
