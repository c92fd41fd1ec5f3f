"""The training iteration on the GPU: the fused Adam update against the FP64
oracle, and one full iteration (batched forward with the contribution record,
masked L1 + background loss, backward, Adam, pruning of the parameters and of
the optimiser moments with the same keep-set).

Adam tolerance: every element goes through ~10 FP32 roundings per step
(two moment FMAs, two bias-correction products, sqrt, add, product, divide,
subtract), each within 2^-24 relative.  m is a signed sum of gradients and can
cancel, so its error is bounded relative to the same recurrence run on |g|
(1e-6 of it over 5 steps); v has no cancellation (1e-5 relative); parameters
of magnitude <= 5 with steps of lr <= 5e-2 stay within 2e-6 absolute.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from _helpers import FWD_TOL, KEYS, to_device

pytestmark = pytest.mark.gpu

LR = dict(xyz=1.6e-4, quat=1e-3, scale=5e-3, opacity=5e-2, sh=2.5e-3)


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


def _arrays(rng, n, deg, scale=1.0):
    shapes = dict(xyz=(n, 3), quat=(n, 4), scale=(n, 2), opacity=(n,), sh=(n, (deg + 1) ** 2, 3))
    return {k: (scale * rng.normal(size=s)).astype(np.float32) for k, s in shapes.items()}


def _dev(d, dev):
    return {k: torch.tensor(v, device=dev) for k, v in d.items()}


def _host(d):
    return {k: v.double().cpu().numpy() for k, v in d.items()}


@pytest.mark.parametrize("n,deg", [(1001, 3), (7, 0), (64, 2)])
def test_adam_matches_oracle_over_five_steps(rast, dev, n, deg):
    rng = np.random.default_rng(n)
    p = _arrays(rng, n, deg)
    zero = {k: np.zeros_like(v) for k, v in p.items()}
    p_d, m_d, v_d = _dev(p, dev), _dev(zero, dev), _dev(zero, dev)
    p_o, m_o, v_o = ({k: v.astype(np.float64) for k, v in d.items()} for d in (p, zero, zero))
    m_abs = {k: np.zeros(v.shape) for k, v in p.items()}  # the m recurrence on |g|
    for t in range(1, 6):
        g = _arrays(rng, n, deg, scale=10.0 ** rng.uniform(-3, 1))
        rast.adam_step(p_d, _dev(g, dev), m_d, v_d, LR, step=t, beta1=0.9, beta2=0.999, eps=1e-15)
        p_o, m_o, v_o = oracle.adam_step(p_o, g, m_o, v_o, LR, step=t, beta1=0.9, beta2=0.999, eps=1e-15)
        m_abs = {k: 0.9 * m_abs[k] + 0.1 * np.abs(g[k]) for k in m_abs}
    torch.cuda.synchronize()
    gp, gm, gv = _host(p_d), _host(m_d), _host(v_d)
    for k in KEYS:
        np.testing.assert_allclose(gp[k], p_o[k], rtol=0, atol=2e-6, err_msg=k)
        assert np.all(np.abs(gm[k] - m_o[k]) <= 1e-6 * m_abs[k] + 1e-30), k
        np.testing.assert_allclose(gv[k], v_o[k], rtol=1e-5, atol=1e-30, err_msg=k)


def test_adam_unaligned_arrays_take_the_scalar_path_with_the_same_result(rast, dev):
    """Arrays that start 4 bytes past a 16-byte boundary give bit-identical results."""
    rng = np.random.default_rng(5)
    n, deg = 333, 1
    p = _arrays(rng, n, deg)
    g = _arrays(rng, n, deg)

    def shifted(d):
        out = {}
        for k, v in d.items():
            buf = torch.zeros(v.size + 1, device=dev)
            view = buf[1:].view(v.shape)
            view.copy_(torch.tensor(v, device=dev))
            out[k] = view
        return out

    zero = {k: np.zeros_like(v) for k, v in p.items()}
    a_p, a_m, a_v = _dev(p, dev), _dev(zero, dev), _dev(zero, dev)
    b_p, b_m, b_v = shifted(p), shifted(zero), shifted(zero)
    for t in (1, 2):
        rast.adam_step(a_p, _dev(g, dev), a_m, a_v, LR, step=t)
        rast.adam_step(b_p, shifted(g), b_m, b_v, LR, step=t)
    torch.cuda.synchronize()
    assert b_p["xyz"].data_ptr() % 16 != 0
    for k in KEYS:
        assert torch.equal(a_p[k], b_p[k]) and torch.equal(a_m[k], b_m[k]) and torch.equal(a_v[k], b_v[k]), k


def test_adam_reports_non_finite_gradients(dev):
    from paper_2501_08174_gb300 import Rasterizer, _lib
    r = Rasterizer(dev)
    try:
        rng = np.random.default_rng(6)
        p = _dev(_arrays(rng, 10, 0), dev)
        g = _arrays(rng, 10, 0)
        g["opacity"][3] = np.nan
        zero = {k: torch.zeros_like(v) for k, v in p.items()}
        r.adam_step(p, _dev(g, dev), zero, {k: torch.zeros_like(v) for k, v in p.items()}, 1e-3, step=1)
        with pytest.raises(_lib.OcgsError) as e:
            r.sync()
        assert e.value.code == _lib.ERR_NONFINITE
        assert torch.isnan(p["opacity"][3]) and torch.isfinite(p["opacity"][:3]).all()
    finally:
        r.close()


def test_adam_rejects_bad_configuration(rast, dev):
    from paper_2501_08174_gb300 import _lib
    rng = np.random.default_rng(7)
    p = _dev(_arrays(rng, 4, 0), dev)
    g = _dev(_arrays(rng, 4, 0), dev)
    z = {k: torch.zeros_like(v) for k, v in p.items()}
    for kw in (dict(beta1=1.0), dict(beta2=-0.1), dict(eps=0.0), dict(step=0)):
        args = dict(lr=1e-3, step=1)
        args.update(kw)
        with pytest.raises(_lib.OcgsError) as e:
            rast.adam_step(p, g, z, {k: torch.zeros_like(v) for k, v in p.items()}, **args)
        assert e.value.code == _lib.ERR_ARG, kw


def test_training_iteration_updates_and_prunes_consistently(rast, dev):
    """Render (with the contribution record) -> masked L1 + 0.5 L_b -> backward ->
    Adam -> prune params, m and v at tau.  Checks: forward against the oracle,
    the Adam update against the oracle applied to the GPU's own gradients, and
    the three pruned sets against the keep-set of the score."""
    sc = synthetic.small_scene(901, 1200, 96, 72, degree=2, n_views=3)
    cams = sc["cameras"]
    g_np = sc["gaussians"]
    g = to_device(g_np, dev)
    from paper_2501_08174_gb300 import pixel_offsets
    off = pixel_offsets(cams)
    P = off[-1]
    N = g["xyz"].shape[0]
    rng = np.random.default_rng(9)
    target = torch.tensor(rng.uniform(0, 1, size=(P, 3)).astype(np.float32), device=dev)
    mask_np = np.concatenate([synthetic.disc_mask(c["width"], c["height"], 25).reshape(-1) for c in cams])
    mask = torch.tensor(mask_np.astype(np.uint8), device=dev)

    score = torch.zeros(N, device=dev)
    out, st = rast.render(g, cams, score=score)
    d_rgb = torch.zeros(P, 3, device=dev)
    d_alpha = torch.zeros(P, device=dev)
    rast.masked_l1(out["rgb"], target, mask, cams, weight=1.0, d_rgb=d_rgb)
    rast.background_loss(out["alpha"], mask, cams, gamma=0.5, d_alpha=d_alpha)
    grads = rast.render_backward(st, g, {"rgb": d_rgb, "alpha": d_alpha})
    st.release()
    params = {k: v.clone() for k, v in g.items()}
    m = {k: torch.zeros_like(v) for k, v in g.items()}
    v = {k: torch.zeros_like(v) for k, v in g.items()}
    rast.adam_step(params, grads, m, v, LR, step=1)
    tau = 0.01
    kept_p, _, _ = rast.prune(params, score, tau)
    kept_m, _, _ = rast.prune(m, score, tau)
    kept_v, _, _ = rast.prune(v, score, tau)
    torch.cuda.synchronize()

    # forward against the oracle on view 1
    ref = oracle.render(g_np, cams[1])
    ok = ~ref["fragile"]
    lo, hi = off[1], off[2]
    for k in ("rgb", "alpha", "depth", "normal"):
        a = out[k][lo:hi].double().cpu().numpy()
        assert np.abs(a[ok] - ref[k][ok]).max() <= FWD_TOL, k
    # Adam on the GPU's gradients, FP64
    g64 = _host(grads)
    p_o, m_o, v_o = oracle.adam_step({k: np.asarray(g_np[k], np.float64) for k in KEYS}, g64,
                                     {k: np.zeros_like(x) for k, x in g64.items()},
                                     {k: np.zeros_like(x) for k, x in g64.items()}, LR, step=1)
    keep = score.cpu().numpy() > tau
    assert 0 < keep.sum() < N
    for k in KEYS:
        np.testing.assert_allclose(_host(params)[k], p_o[k], rtol=0, atol=2e-6, err_msg=k)
        assert torch.equal(kept_p[k], params[k][torch.as_tensor(keep, device=dev)]), k
        assert torch.equal(kept_m[k], m[k][torch.as_tensor(keep, device=dev)]), k
        assert torch.equal(kept_v[k], v[k][torch.as_tensor(keep, device=dev)]), k
