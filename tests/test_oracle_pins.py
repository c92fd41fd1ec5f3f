"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test fixes a plausible mistake in the oracle: a wrong rotation or SH
sign (library routines), a wrong intersection (closed forms and an
independent world-space ray-plane solve), a wrong compositing order,
termination or cut-off (hand-computed stacks), a wrong adjoint (central
finite differences), and a wrong loss or pruning rule (hand sums).
"""
import json
import math
import os

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation
from scipy import special

import oracle
import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SQ2PI = 2.0 * math.sqrt(math.pi)


def surfels(xyz, quat, scale, opacity, rgb):
    """Degree-0 surfels whose rendered colour is exactly ``rgb``."""
    xyz = np.asarray(xyz, np.float64).reshape(-1, 3)
    n = len(xyz)
    return dict(xyz=xyz, quat=np.asarray(quat, np.float64).reshape(n, 4),
                scale=np.asarray(scale, np.float64).reshape(n, 2),
                opacity=np.asarray(opacity, np.float64).reshape(n),
                sh=((np.asarray(rgb, np.float64).reshape(n, 1, 3) - 0.5) * SQ2PI), sh_degree=0)


# rotation about +x by 90 deg maps the surfel normal +z to -y: facing a camera on the -y axis
Q_FACE = [math.cos(math.pi / 4), math.sin(math.pi / 4), 0.0, 0.0]


def cam65(width=65, height=65):
    return synthetic.make_camera((0.0, -3.0, 0.0), width, height)


def pix(cam, ix, iy):
    return np.array([iy * cam["width"] + ix])


# ----------------------------------------------------------------------------- library pins
def test_quaternion_matches_scipy():
    rng = np.random.default_rng(0)
    q = rng.normal(size=(64, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    ours = oracle.quat_to_rotmat(torch.tensor(q)).numpy()
    ref = Rotation.from_quat(q, scalar_first=True).as_matrix()
    np.testing.assert_allclose(ours, ref, atol=1e-13)


def test_sh_basis_matches_scipy_complex_harmonics():
    rng = np.random.default_rng(1)
    d = rng.normal(size=(50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(d[:, 2])
    phi = np.arctan2(d[:, 1], d[:, 0])
    ours = oracle.sh_basis(torch.tensor(d), 3).numpy()
    col = 0
    for l in range(4):
        for m in range(-l, l + 1):
            y = special.sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                ref = math.sqrt(2.0) * y.real
            elif m < 0:
                ref = math.sqrt(2.0) * y.imag
            else:
                ref = y.real
            np.testing.assert_allclose(ours[:, col], ref, atol=1e-13, err_msg=f"l={l} m={m}")
            col += 1


# ----------------------------------------------------------------------------- closed forms
def test_fronto_parallel_centre_hit():
    cam = cam65()
    rgb = [0.2, 0.7, 0.4]
    g = surfels([0, 0, 0], Q_FACE, [0.1, 0.1], 0.6, rgb)
    r = oracle.render(g, cam, pix(cam, 32, 32))
    np.testing.assert_allclose(r["alpha"], [0.6], atol=1e-14)
    np.testing.assert_allclose(r["rgb"][0], 0.6 * np.array(rgb), atol=1e-14)
    np.testing.assert_allclose(r["depth"], [0.6 * 3.0], atol=1e-13)
    np.testing.assert_allclose(r["normal"][0], [0.0, 0.0, -0.6], atol=1e-14)
    np.testing.assert_allclose(r["t_final"], [0.4], atol=1e-14)


def test_opacity_clamp_at_centre():
    cam = cam65()
    g = surfels([0, 0, 0], Q_FACE, [0.1, 0.1], 1.0, [1, 1, 1])
    r = oracle.render(g, cam, pix(cam, 32, 32))
    np.testing.assert_allclose(r["alpha"], [0.99], atol=1e-14)


@pytest.mark.parametrize("s,dx,branch", [(0.2, 3, "surfel"), (0.1, 2, "surfel"), (0.005, 1, "filter")])
def test_fronto_parallel_falloff(s, dx, branch):
    """Ray through pixel offset dx meets the plane z = 3 at X = dx z / f: u = X / s."""
    cam = cam65()
    o = 0.8
    g = surfels([0, 0, 0], Q_FACE, [s, s], o, [0.5, 0.5, 0.5])
    r = oracle.render(g, cam, pix(cam, 32 + dx, 32))
    rho3 = (dx * 3.0 / (cam["fx"] * s)) ** 2
    rho2 = 2.0 * dx * dx
    rho = min(rho3, rho2)
    assert (rho3 <= rho2) == (branch == "surfel")
    a = o * math.exp(-0.5 * rho)
    np.testing.assert_allclose(r["alpha"], [a], rtol=1e-12)
    np.testing.assert_allclose(r["depth"], [a * 3.0], rtol=1e-12)


def test_oblique_surfel_matches_ray_plane_intersection():
    """Tilted surfel: depth and (u, v) from the textbook ray-plane intersection."""
    cam = synthetic.make_camera((0.0, -3.0, 0.0), 48, 40)
    rng = np.random.default_rng(5)
    q = Rotation.from_euler("xyz", [70, 25, 10], degrees=True).as_quat(scalar_first=True)
    s = np.array([0.35, 0.2])
    o = 0.7
    centre = np.array([0.05, 0.1, -0.04])
    g = surfels(centre, q, s, o, [0.3, 0.3, 0.3])
    R = Rotation.from_quat(q, scalar_first=True).as_matrix()
    vm = cam["viewmat"]
    r_cw, t_cw = vm[:3, :3], vm[:3, 3]
    p = r_cw @ centre + t_cw
    U, V = r_cw @ (s[0] * R[:, 0]), r_cw @ (s[1] * R[:, 1])
    n = np.cross(U, V)
    px = np.arange(48 * 40)
    r = oracle.render(g, cam, px, prefilter=False)
    for k, pidx in enumerate(px):
        x, y = pidx % 48 + 0.5, pidx // 48 + 0.5
        d = np.array([(x - cam["cx"]) / cam["fx"], (y - cam["cy"]) / cam["fy"], 1.0])
        t = n @ p / (n @ d)                 # camera depth of the hit (d has unit z)
        X = t * d
        u = (X - p) @ U / (U @ U)
        v = (X - p) @ V / (V @ V)
        rho3 = u * u + v * v
        c = np.array([cam["fx"] * p[0] / p[2] + cam["cx"], cam["fy"] * p[1] / p[2] + cam["cy"]])
        rho2 = ((x - c[0]) ** 2 + (y - c[1]) ** 2) * 2.0
        rho = min(rho3, rho2)
        a = min(0.99, o * math.exp(-0.5 * rho))
        if rho > 9 or a < 1 / 255:
            a = 0.0
        z = t if rho3 <= rho2 else p[2]
        np.testing.assert_allclose(r["alpha"][k], a, atol=1e-12)
        np.testing.assert_allclose(r["depth"][k], a * z, atol=1e-11)
    assert (r["alpha"] > 0).sum() > 100


def test_two_splat_ordering_and_swap():
    cam = cam65()
    c1, c2 = np.array([1.0, 0.2, 0.1]), np.array([0.1, 0.3, 0.9])
    o1, o2 = 0.6, 0.7
    # surfel 0 at depth 2 (world y = -1), surfel 1 at depth 3 (y = 0)
    g = surfels([[0, -1, 0], [0, 0, 0]], [Q_FACE, Q_FACE], [[0.3, 0.3]] * 2, [o1, o2], [c1, c2])
    r = oracle.render(g, cam, pix(cam, 32, 32))
    np.testing.assert_allclose(r["rgb"][0], o1 * c1 + (1 - o1) * o2 * c2, atol=1e-14)
    np.testing.assert_allclose(r["depth"], [o1 * 2.0 + (1 - o1) * o2 * 3.0], atol=1e-13)
    g2 = surfels([[0, 0, 0], [0, -1, 0]], [Q_FACE, Q_FACE], [[0.3, 0.3]] * 2, [o1, o2], [c1, c2])
    r2 = oracle.render(g2, cam, pix(cam, 32, 32))
    np.testing.assert_allclose(r2["rgb"][0], o2 * c2 + (1 - o2) * o1 * c1, atol=1e-14)
    # equal depth: ties resolve to ascending index
    g3 = surfels([[0, 0, 0], [0, 0, 0]], [Q_FACE, Q_FACE], [[0.3, 0.3]] * 2, [o1, o2], [c1, c2])
    r3 = oracle.render(g3, cam, pix(cam, 32, 32))
    np.testing.assert_allclose(r3["rgb"][0], o1 * c1 + (1 - o1) * o2 * c2, atol=1e-14)


@pytest.mark.parametrize("o,expect", [(0.95, 3), (0.8, 5), (0.5, 13)])
def test_termination_blends_closed_form_count(o, expect):
    """A stack of equal surfels blends k = floor(log 1e-4 / log(1 - o)) of them."""
    cam = cam65()
    m = 20
    xyz = [[0, -1.0 + 0.02 * i, 0] for i in range(m)]
    g = surfels(xyz, [Q_FACE] * m, [[0.4, 0.4]] * m, [o] * m, [[0.5, 0.5, 0.5]] * m)
    r = oracle.render(g, cam, pix(cam, 32, 32))
    k = math.floor(math.log(1e-4) / math.log(1 - o))
    assert k == expect
    assert r["n_blended"][0] == k
    np.testing.assert_allclose(r["t_final"], [(1 - o) ** k], rtol=1e-12)
    np.testing.assert_allclose(r["alpha"], [1 - (1 - o) ** k], rtol=1e-12)


@pytest.mark.parametrize("rho_target,blended", [(8.9, True), (9.1, False)])
def test_support_cutoff(rho_target, blended):
    cam = cam65()
    dx = 4
    s = dx * 3.0 / (cam["fx"] * math.sqrt(rho_target))   # rho3 = rho_target < rho2 = 32
    g = surfels([0, 0, 0], Q_FACE, [s, s], 0.9, [0.5, 0.5, 0.5])
    r = oracle.render(g, cam, pix(cam, 32 + dx, 32))
    expect = 0.9 * math.exp(-0.5 * rho_target) if blended else 0.0
    np.testing.assert_allclose(r["alpha"], [expect], rtol=1e-10, atol=1e-15)


@pytest.mark.parametrize("factor,blended", [(1.01, True), (0.99, False)])
def test_alpha_floor(factor, blended):
    cam = cam65()
    dx, s = 3, 0.15
    rho = (dx * 3.0 / (cam["fx"] * s)) ** 2
    o = factor * (1 / 255) / math.exp(-0.5 * rho)
    g = surfels([0, 0, 0], Q_FACE, [s, s], o, [0.5, 0.5, 0.5])
    r = oracle.render(g, cam, pix(cam, 32 + dx, 32))
    np.testing.assert_allclose(r["alpha"], [factor / 255 if blended else 0.0], rtol=1e-10, atol=1e-15)


def test_near_plane_cull():
    """A surfel whose 3-sigma square crosses the near plane is not rendered."""
    cam = cam65()
    # camera at y=-3 looks along +y; a surfel at depth 0.5 tilted so its square spans depth +-0.4
    q = Rotation.from_euler("x", 45, degrees=True).as_quat(scalar_first=True)
    g = surfels([0, -2.5, 0], q, [0.2, 0.2], 0.9, [1, 1, 1])
    r = oracle.render(g, cam)
    assert r["alpha"].max() == 0.0
    assert r["cull_margin"][0] < 0


# ----------------------------------------------------------------------------- invariants
def test_weights_plus_final_transmittance_is_one():
    sc = synthetic.small_scene(11, 300, 40, 33, degree=1)
    r = oracle.render(sc["gaussians"], sc["cameras"][0])
    np.testing.assert_allclose(r["alpha"] + r["t_final"], 1.0, atol=1e-12)
    assert r["alpha"].max() > 0.5


def test_prefilter_is_exact():
    sc = synthetic.small_scene(12, 400, 37, 29, degree=2)
    a = oracle.render(sc["gaussians"], sc["cameras"][0], prefilter=True, chunk=97)
    b = oracle.render(sc["gaussians"], sc["cameras"][0], prefilter=False, chunk=1000)
    for k in ("rgb", "alpha", "depth", "normal", "t_final"):
        np.testing.assert_allclose(a[k], b[k], atol=1e-13, err_msg=k)
    np.testing.assert_array_equal(a["n_blended"], b["n_blended"])
    np.testing.assert_array_equal(a["score"], b["score"])


def _brute_force(g, cam):
    """Independent per-pixel loop: world-space ray-plane solve, explicit projection."""
    vm = cam["viewmat"]
    r_cw, t_cw = vm[:3, :3], vm[:3, 3]
    origin = -r_cw.T @ t_cw
    q = g["quat"] / np.linalg.norm(g["quat"], axis=1, keepdims=True)
    Rs = Rotation.from_quat(q, scalar_first=True).as_matrix()
    n = len(q)
    W, H = cam["width"], cam["height"]
    out = np.zeros((H * W, 8))
    zc = np.array([(r_cw @ g["xyz"][i] + t_cw)[2] for i in range(n)])
    order = sorted(range(n), key=lambda i: (zc[i], i))
    deg = g["sh_degree"]
    for pidx in range(H * W):
        x, y = pidx % W + 0.5, pidx // W + 0.5
        d_cam = np.array([(x - cam["cx"]) / cam["fx"], (y - cam["cy"]) / cam["fy"], 1.0])
        d_w = r_cw.T @ d_cam
        T = 1.0
        acc = np.zeros(8)
        for i in order:
            p = g["xyz"][i]
            tu, tv, tw = Rs[i][:, 0], Rs[i][:, 1], Rs[i][:, 2]
            su, sv = g["scale"][i]
            pc = r_cw @ p + t_cw
            zmin = pc[2] - 3 * (abs((r_cw @ (su * tu))[2]) + abs((r_cw @ (sv * tv))[2]))
            if zmin <= cam["near"]:
                continue
            A = np.stack([d_w, -su * tu, -sv * tv], axis=1)
            try:
                t, u, v = np.linalg.solve(A, p - origin)
                rho3 = u * u + v * v
            except np.linalg.LinAlgError:
                rho3 = math.inf
            c = np.array([cam["fx"] * pc[0] / pc[2] + cam["cx"], cam["fy"] * pc[1] / pc[2] + cam["cy"]])
            rho2 = ((x - c[0]) ** 2 + (y - c[1]) ** 2) / 0.5
            rho = min(rho3, rho2)
            a = min(0.99, g["opacity"][i] * math.exp(-0.5 * rho))
            if rho > 9 or a < 1 / 255:
                continue
            if T * (1 - a) < 1e-4:
                break
            w = a * T
            z = (r_cw @ (origin + t * d_w) + t_cw)[2] if rho3 <= rho2 else pc[2]
            nc = r_cw @ tw
            if nc @ pc > 0:
                nc = -nc
            dirv = (p - origin) / np.linalg.norm(p - origin)
            basis = oracle.sh_basis(torch.tensor(dirv[None]), deg).numpy()[0]
            rgb = np.maximum(basis @ g["sh"][i] + 0.5, 0.0)
            acc += w * np.concatenate([rgb, [1.0, z], nc])
            T *= 1 - a
        out[pidx] = acc
    return out


@pytest.mark.parametrize("seed", [21, 22])
def test_brute_force_tiny_scene(seed):
    sc = synthetic.small_scene(seed, 8, 16, 16, degree=1, scale_range=(0.2, 0.6))
    g = sc["gaussians"]
    cam = synthetic.make_camera((0.3, -3.0, 0.4), 16, 16, f32=False)  # orthonormal, for the world-space solve
    g = {k: (np.asarray(v, np.float64) if k != "sh_degree" else v) for k, v in g.items()}
    r = oracle.render(g, cam, prefilter=False)
    bf = _brute_force(g, cam)
    np.testing.assert_allclose(r["rgb"], bf[:, 0:3], atol=1e-11)
    np.testing.assert_allclose(r["alpha"], bf[:, 3], atol=1e-11)
    np.testing.assert_allclose(r["depth"], bf[:, 4], atol=1e-10)
    np.testing.assert_allclose(r["normal"], bf[:, 5:8], atol=1e-11)
    assert r["alpha"].max() > 0.3


# ----------------------------------------------------------------------------- adjoint
def _loss(g, cam, d_out, px):
    r = oracle.render(g, cam, px, prefilter=False)
    return (np.sum(r["rgb"] * d_out["rgb"]) + np.sum(r["alpha"] * d_out["alpha"])
            + np.sum(r["depth"] * d_out["depth"]) + np.sum(r["normal"] * d_out["normal"])), r


def test_adjoint_matches_central_differences():
    sc = synthetic.small_scene(31, 6, 12, 10, degree=2, scale_range=(0.25, 0.6))
    g = {k: (np.asarray(v, np.float64).copy() if k != "sh_degree" else v) for k, v in sc["gaussians"].items()}
    cam = sc["cameras"][0]
    px = np.arange(12 * 10)
    rng = np.random.default_rng(3)
    d_out = dict(rgb=rng.normal(size=(len(px), 3)), alpha=rng.normal(size=len(px)),
                 depth=rng.normal(size=len(px)), normal=rng.normal(size=(len(px), 3)))
    r = oracle.render(g, cam, px, d_out=d_out, prefilter=False)
    grads = r["grads"]
    base_sig = r["n_blended"]
    checked = 0
    for key in ("xyz", "quat", "scale", "opacity", "sh"):
        flat = g[key].reshape(-1)
        gflat = grads[key].reshape(-1)
        for j in range(flat.size):
            x0 = flat[j]
            h = 1e-6 * max(1.0, abs(x0))
            flat[j] = x0 + h
            lp, rp = _loss(g, cam, d_out, px)
            flat[j] = x0 - h
            lm, rm = _loss(g, cam, d_out, px)
            flat[j] = x0
            if not (np.array_equal(rp["n_blended"], base_sig) and np.array_equal(rm["n_blended"], base_sig)):
                continue  # a discrete decision flipped: the derivative is not defined there
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gflat[j]) <= 1e-6 * max(1.0, abs(fd)), (key, j, fd, gflat[j])
            checked += 1
    assert checked > 100


# ----------------------------------------------------------------------------- background loss and pruning
def test_background_loss_hand_sum():
    with open(os.path.join(GOLDEN, "background_loss_4x4.json")) as f:
        case = json.load(f)
    a = np.array(case["alpha"])
    m = np.array(case["mask"])
    assert oracle.background_loss(a, m) == pytest.approx(case["loss"], abs=1e-15)
    np.testing.assert_allclose(oracle.background_loss_grad(m, 0.5), 0.5 * (1 - m) / 16, atol=0)


def test_parameter_layout_matches_the_storage_per_gaussian_of_table3():
    """58 float32 values per surfel at SH degree 3 (xyz 3, quaternion 4, two scales, opacity 1,
    48 SH coefficients), the layout the oracle, the generators and the library share, against the
    bytes per Gaussian the paper's storage figures imply; a third scale (59 values, 236 bytes)
    would miss them by 1.5 %."""
    with open(os.path.join(GOLDEN, "storage_per_gaussian_table3.json")) as f:
        case = json.load(f)
    g = synthetic.small_scene(3, 5, 8, 8, degree=3)["gaussians"]
    floats = sum(int(np.prod(np.asarray(g[k]).shape[1:])) for k in ("xyz", "quat", "scale", "opacity", "sh"))
    assert floats == 58
    for row in case["rows"]:
        per_gaussian = row["storage_mb"] * 1e6 / row["gaussians"]
        assert abs(per_gaussian - 4 * floats) < 0.5, row


def test_masked_l1_hand_sum():
    with open(os.path.join(GOLDEN, "masked_l1_2x2.json")) as f:
        case = json.load(f)
    loss, grad = oracle.masked_l1(case["rgb"], case["target"], case["mask"], weight=1.0)
    assert loss == pytest.approx(case["loss"], abs=1e-15)
    np.testing.assert_allclose(grad * 12.0, np.array(case["grad_times_12"], np.float64), atol=1e-15)
    _, g2 = oracle.masked_l1(case["rgb"], case["target"], case["mask"], weight=0.8)
    np.testing.assert_allclose(g2, 0.8 * grad, atol=1e-17)


def test_masked_l1_special_masks_and_central_differences():
    rng = np.random.default_rng(31)
    r = rng.uniform(0, 1, size=(60, 3))
    t = rng.uniform(0, 1, size=(60, 3))
    # an all-ones mask gives the plain mean absolute error, an all-zeros mask nothing
    loss, grad = oracle.masked_l1(r, t, np.ones(60))
    assert loss == pytest.approx(np.mean(np.abs(r - t)), abs=1e-15)
    np.testing.assert_allclose(grad, np.sign(r - t) / r.size, atol=0)
    loss0, grad0 = oracle.masked_l1(r, t, np.zeros(60))
    assert loss0 == 0.0 and not grad0.any()
    # the adjoint against central differences of the loss, away from the kinks
    m = (rng.uniform(size=60) < 0.6).astype(np.float64)
    _, grad = oracle.masked_l1(r, t, m)
    h = 1e-6
    for i, c in zip(rng.integers(0, 60, 40), rng.integers(0, 3, 40)):
        if abs(r[i, c] - t[i, c]) < 1e-3:
            continue
        rp, rm = r.copy(), r.copy()
        rp[i, c] += h
        rm[i, c] -= h
        fd = (oracle.masked_l1(rp, t, m)[0] - oracle.masked_l1(rm, t, m)[0]) / (2 * h)
        assert fd == pytest.approx(grad[i, c], abs=1e-9)


def test_hidden_surfel_scores_zero_and_lone_surfel_scores_opacity():
    cam = cam65()
    m = 6
    x_lone = 22.0 * 3.0 / cam["fx"]   # projects exactly onto the centre of pixel (54, 32)
    # an opaque stack in front (0.95 each): every pixel the hidden surfel reaches terminates first
    xyz = [[0, -1.0 + 0.02 * i, 0] for i in range(m)] + [[0, 0.5, 0], [x_lone, 0, 0]]
    scales = [[0.2, 0.2]] * m + [[0.05, 0.05], [0.02, 0.02]]
    g = surfels(xyz, [Q_FACE] * (m + 2), scales, [0.95] * m + [0.9, 0.7], [[0.5, 0.5, 0.5]] * (m + 2))
    score = oracle.contribution_score(g, [cam])
    assert score[m] == 0.0                              # hidden behind the stack
    assert score[m + 1] == pytest.approx(0.7, abs=1e-9)  # lone surfel, hit at its centre
    assert score[0] == pytest.approx(0.95, abs=1e-9)
    keep, near = oracle.keep_set(score, 0.0)
    assert not keep[m] and keep[m + 1] and keep[0]
    keep, near = oracle.keep_set(np.array([0.01, 0.0100000005, 0.02]), 0.01)
    np.testing.assert_array_equal(keep, [False, True, True])
    np.testing.assert_array_equal(near, [0, 1])


def test_lone_surfel_exact_score_at_centre_pixel():
    cam = cam65()
    g = surfels([0, 0, 0], Q_FACE, [0.1, 0.1], 0.42, [0.5, 0.5, 0.5])
    score = oracle.contribution_score(g, [cam])
    assert score[0] == pytest.approx(0.42, abs=1e-14)


# ----------------------------------------------------------------------------- Adam (Kingma & Ba, Algorithm 1)
def _adam_arrays(rng, n=5, deg=1):
    shapes = dict(xyz=(n, 3), quat=(n, 4), scale=(n, 2), opacity=(n,), sh=(n, (deg + 1) ** 2, 3))
    return {k: rng.normal(size=s) for k, s in shapes.items()}, shapes


def test_adam_first_step_is_lr_times_sign():
    """From zero moments the bias corrections give m_hat = g and v_hat = g^2, so the
    first step moves every element by lr g / (|g| + eps)."""
    rng = np.random.default_rng(0)
    p, shapes = _adam_arrays(rng)
    g, _ = _adam_arrays(rng)
    z = {k: np.zeros(s) for k, s in shapes.items()}
    lr = dict(xyz=1e-3, quat=2e-3, scale=5e-3, opacity=5e-2, sh=2.5e-3)
    eps = 1e-8
    p1, m1, v1 = oracle.adam_step(p, g, z, z, lr, step=1, beta1=0.9, beta2=0.999, eps=eps)
    for k in p:
        np.testing.assert_allclose(p1[k], p[k] - lr[k] * g[k] / (np.abs(g[k]) + eps), rtol=0, atol=1e-15)
        np.testing.assert_allclose(m1[k], 0.1 * g[k], rtol=1e-14)
        np.testing.assert_allclose(v1[k], 0.001 * g[k] ** 2, rtol=1e-12)


def test_adam_constant_gradient_moves_linearly():
    """With a constant gradient m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2, so each
    bias-corrected step is the same lr g / (|g| + eps): after t steps p = p0 - t lr g / (|g| + eps)."""
    rng = np.random.default_rng(1)
    p0, shapes = _adam_arrays(rng)
    g, _ = _adam_arrays(rng)
    m = {k: np.zeros(s) for k, s in shapes.items()}
    v = {k: np.zeros(s) for k, s in shapes.items()}
    p = p0
    for t in range(1, 8):
        p, m, v = oracle.adam_step(p, g, m, v, 1e-2, step=t, beta1=0.8, beta2=0.99, eps=1e-12)
    for k in p:
        np.testing.assert_allclose(p[k], p0[k] - 7 * 1e-2 * g[k] / (np.abs(g[k]) + 1e-12), rtol=0, atol=1e-12)
        np.testing.assert_allclose(m[k], (1 - 0.8 ** 7) * g[k], rtol=1e-12)


def test_adam_alternating_gradient_second_step():
    """Gradients g then -g: m_2 = -(1 - b1)^2 g and v_2 = (1 - b2)(1 + b2) g^2, so
    m_hat = -(1 - b1) g / (1 + b1), v_hat = g^2 and the second step is
    +lr (1 - b1) / (1 + b1) g / (|g| + eps)  (a swapped b1 / 1 - b1 fails this)."""
    rng = np.random.default_rng(2)
    p0, shapes = _adam_arrays(rng)
    g, _ = _adam_arrays(rng)
    neg = {k: -x for k, x in g.items()}
    z = {k: np.zeros(s) for k, s in shapes.items()}
    b1, b2, lr, eps = 0.7, 0.95, 0.1, 1e-12
    p1, m1, v1 = oracle.adam_step(p0, g, z, z, lr, 1, b1, b2, eps)
    p2, m2, v2 = oracle.adam_step(p1, neg, m1, v1, lr, 2, b1, b2, eps)
    for k in p0:
        np.testing.assert_allclose(m2[k], -(1 - b1) ** 2 * g[k], rtol=1e-12)
        np.testing.assert_allclose(v2[k], (1 - b2) * (1 + b2) * g[k] ** 2, rtol=1e-12)
        step2 = lr * (1 - b1) / (1 + b1) * g[k] / (np.abs(g[k]) + eps)
        np.testing.assert_allclose(p2[k] - p1[k], step2, rtol=1e-9, atol=1e-15)


def test_adam_zero_gradient_keeps_everything():
    rng = np.random.default_rng(3)
    p, shapes = _adam_arrays(rng)
    z = {k: np.zeros(s) for k, s in shapes.items()}
    p1, m1, v1 = oracle.adam_step(p, z, z, z, 0.5, step=3)
    for k in p:
        np.testing.assert_array_equal(p1[k], p[k])
        np.testing.assert_array_equal(m1[k], 0.0)
        np.testing.assert_array_equal(v1[k], 0.0)


# ----------------------------------------------------------------------------- SSIM / PSNR (Eq. 2's L_c, Sec. 5)
def test_ssim_window_blur_matches_scipy_gaussian_filter():
    """The windowed mean is SciPy's Gaussian filter of sigma 1.5 truncated at radius 5, zero outside."""
    from scipy import ndimage
    rng = np.random.default_rng(0)
    x = rng.uniform(size=(23, 17, 3))
    got = oracle.ssim_blur(torch.tensor(x)).numpy()
    for c in range(3):
        ref = ndimage.gaussian_filter(x[..., c], sigma=1.5, mode="constant", cval=0.0, truncate=5.0 / 1.5)
        np.testing.assert_allclose(got[..., c], ref, rtol=0, atol=1e-13)


def test_ssim_of_identical_images_is_one_and_stationary():
    rng = np.random.default_rng(1)
    x = rng.uniform(size=(19, 14, 3))
    m = (rng.uniform(size=(19, 14)) > 0.3).astype(np.uint8)
    s_all, s_m, grad = oracle.masked_ssim(x, x, m, weight=0.2)
    assert s_all == pytest.approx(1.0, abs=1e-14) and s_m == pytest.approx(1.0, abs=1e-14)
    np.testing.assert_allclose(grad, 0.0, atol=1e-12)   # SSIM is maximal at x2 = x1


def test_ssim_of_constant_images_in_the_interior():
    """Constant images a and b: away from the border the variances vanish and
    SSIM = (2ab + C1) / (a^2 + b^2 + C1)."""
    a, b = 0.7, 0.4
    s = oracle.ssim_map(torch.full((30, 30, 3), a, dtype=torch.float64),
                        torch.full((30, 30, 3), b, dtype=torch.float64)).numpy()
    expect = (2 * a * b + 1e-4) / (a * a + b * b + 1e-4)
    np.testing.assert_allclose(s[5:25, 5:25], expect, rtol=1e-12)


def test_ssim_map_matches_brute_force_windows():
    rng = np.random.default_rng(2)
    h, w = 9, 13
    x1, x2 = rng.uniform(size=(h, w, 3)), rng.uniform(size=(h, w, 3))
    g = [math.exp(-(k * k) / 4.5) for k in range(-5, 6)]
    gs = sum(g)
    g = [v / gs for v in g]
    got = oracle.ssim_map(torch.tensor(x1), torch.tensor(x2)).numpy()
    for y in range(h):
        for x in range(w):
            for c in range(3):
                m1 = m2 = e11 = e22 = e12 = 0.0
                for dy in range(-5, 6):
                    for dx in range(-5, 6):
                        yy, xx = y + dy, x + dx
                        if 0 <= yy < h and 0 <= xx < w:
                            wt = g[dy + 5] * g[dx + 5]
                            p, q = x1[yy, xx, c], x2[yy, xx, c]
                            m1 += wt * p; m2 += wt * q
                            e11 += wt * p * p; e22 += wt * q * q; e12 += wt * p * q
                v1, v2, cv = e11 - m1 * m1, e22 - m2 * m2, e12 - m1 * m2
                ref = (2 * m1 * m2 + 1e-4) * (2 * cv + 9e-4) / ((m1 * m1 + m2 * m2 + 1e-4) * (v1 + v2 + 9e-4))
                assert got[y, x, c] == pytest.approx(ref, abs=1e-12), (y, x, c)


def test_dssim_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    h, w = 10, 8
    r, t = rng.uniform(size=(h, w, 3)), rng.uniform(size=(h, w, 3))
    m = (rng.uniform(size=(h, w)) > 0.25).astype(np.uint8)
    _, _, grad = oracle.masked_ssim(r, t, m, weight=0.2)
    for flat in rng.choice(h * w * 3, size=24, replace=False):
        i = np.unravel_index(flat, r.shape)
        rp, rm = r.copy(), r.copy()
        rp[i] += 1e-6
        rm[i] -= 1e-6
        fd = (0.2 * (1 - oracle.masked_ssim(rp, t, m)[0]) - 0.2 * (1 - oracle.masked_ssim(rm, t, m)[0])) / 2e-6
        assert grad[i] == pytest.approx(fd, abs=1e-8), i
        if m[i[0], i[1]] == 0:
            assert grad[i] == 0.0                          # masked-out pixels get no gradient


def test_masked_psnr_hand_value():
    """Target 0.5 everywhere; one masked value off by 0.1 and an unmasked pixel off by 0.3:
    MSE = 0.01 / 9 over the 3 x 3 masked values, PSNR = 20 log10(30)."""
    t = np.full((2, 2, 3), 0.5)
    r = t.copy()
    r[0, 0, 0] = 0.6
    r[0, 1] = 0.8
    m = np.array([[1, 0], [1, 1]], np.uint8)
    assert oracle.masked_psnr(r, t, m) == pytest.approx(20 * math.log10(30.0), abs=1e-12)
    assert oracle.masked_psnr(t, t, m) == float("inf")


# ----------------------------------------------------------------------------- 2DGS regularisers (Eq. 3)
def test_depth2_and_depth_distortion_of_two_stacked_surfels():
    """Two fronto-parallel surfels hit at their centres at depths 3 and 3.5: w1 = o1,
    w2 = (1 - o1) o2, Q = w1 z1^2 + w2 z2^2 and the pixel's distortion
    sum_{i,j} w_i w_j (z_i - z_j)^2 = 2 w1 w2 (z1 - z2)^2."""
    cam = cam65()
    o1, o2 = 0.6, 0.7
    g = surfels([[0, 0, 0], [0, 0.5, 0]], [Q_FACE] * 2, [[0.1, 0.1]] * 2, [o1, o2], [[0.5, 0.5, 0.5]] * 2)
    r = oracle.render(g, cam, pix(cam, 32, 32))
    w1, w2 = o1, (1 - o1) * o2
    assert r["depth2"][0] == pytest.approx(w1 * 9.0 + w2 * 12.25, abs=1e-12)
    ld, ga, gd, gq = oracle.depth_distortion(r["alpha"], r["depth"], r["depth2"])
    assert ld == pytest.approx(2 * w1 * w2 * 0.25, abs=1e-12)
    one = oracle.render(surfels([0, 0, 0], Q_FACE, [0.1, 0.1], o1, [0.5] * 3), cam, pix(cam, 32, 32))
    assert oracle.depth_distortion(one["alpha"], one["depth"], one["depth2"])[0] == pytest.approx(0.0, abs=1e-12)


def test_depth_distortion_equals_brute_force_pairs():
    rng = np.random.default_rng(7)
    A, D, Q, ref = [], [], [], []
    for _ in range(6):
        n = int(rng.integers(1, 9))
        w, z = rng.uniform(0, 0.3, n), rng.uniform(1, 4, n)
        A.append(w.sum()); D.append((w * z).sum()); Q.append((w * z * z).sum())
        ref.append(sum(w[i] * w[j] * (z[i] - z[j]) ** 2 for i in range(n) for j in range(n)))
    ld, ga, gd, gq = oracle.depth_distortion(np.array(A), np.array(D), np.array(Q), weight=1.0)
    assert ld == pytest.approx(np.mean(ref), rel=1e-12)
    np.testing.assert_allclose(gq, 2 * np.array(A) / 6, rtol=1e-12)   # d/dQ of the mean of 2 (A Q - D^2)


def test_depth_distortion_pairs_brute_force_against_the_planes():
    """The brute-force pair sums over each pixel's blended entries: the squared reading equals
    2 (A Q - D^2) of the rendered planes at every pixel (which pins the Q plane and the closed
    form), and the printed |z_i - z_j| form of two stacked surfels is 2 w1 w2 |z1 - z2|."""
    sc = synthetic.small_scene(41, 250, 24, 20, degree=1, scale_range=(0.05, 0.3))
    r = oracle.render(sc["gaussians"], sc["cameras"][0], pair_powers=(1, 2))
    closed = 2.0 * (r["alpha"] * r["depth2"] - r["depth"] ** 2)
    np.testing.assert_allclose(r["distortion_pairs_2"], closed, rtol=1e-9, atol=1e-12)
    assert (r["n_blended"] >= 2).sum() > 50 and r["distortion_pairs_1"].max() > 0
    cam = cam65()
    o1, o2 = 0.6, 0.7
    g = surfels([[0, 0, 0], [0, 0.5, 0]], [Q_FACE] * 2, [[0.1, 0.1]] * 2, [o1, o2], [[0.5, 0.5, 0.5]] * 2)
    two = oracle.render(g, cam, pix(cam, 32, 32), pair_powers=(1, 2))
    w1, w2 = o1, (1 - o1) * o2
    assert two["distortion_pairs_1"][0] == pytest.approx(2 * w1 * w2 * 0.5, abs=1e-12)
    assert two["distortion_pairs_2"][0] == pytest.approx(2 * w1 * w2 * 0.25, abs=1e-12)


def test_prune_keeps_the_flagged_surfels_in_order():
    """A hand case: five surfels, keep-set {score > 0.01} of the scores below keeps rows 1 and 3
    (score 0.01 itself is not kept), each array sliced the same way, order preserved."""
    g = dict(xyz=np.arange(15.0).reshape(5, 3), quat=np.arange(20.0).reshape(5, 4),
             scale=np.arange(10.0).reshape(5, 2), opacity=np.array([0.1, 0.2, 0.3, 0.4, 0.5]),
             sh=np.arange(15.0).reshape(5, 1, 3), sh_degree=0)
    keep, near = oracle.keep_set(np.array([0.0, 0.5, 0.01, 0.02, 0.0099995]), 0.01)
    assert keep.tolist() == [False, True, False, True, False]
    assert near.tolist() == [2, 4]
    out = oracle.prune(g, keep)
    assert out["xyz"].tolist() == [[3.0, 4.0, 5.0], [9.0, 10.0, 11.0]]
    assert out["quat"].tolist() == [[4.0, 5.0, 6.0, 7.0], [12.0, 13.0, 14.0, 15.0]]
    assert out["scale"].tolist() == [[2.0, 3.0], [6.0, 7.0]]
    assert out["opacity"].tolist() == [0.2, 0.4]
    assert out["sh"].tolist() == [[[3.0, 4.0, 5.0]], [[9.0, 10.0, 11.0]]]
    assert out["sh_degree"] == 0


def _plane_images(cam, n, p0, a=0.8):
    """Planes of a surface with unit normal n through p0 (camera frame), seen with opacity a."""
    W, H = cam["width"], cam["height"]
    xs = (np.arange(W) + 0.5 - cam["cx"]) / cam["fx"]
    ys = (np.arange(H) + 0.5 - cam["cy"]) / cam["fy"]
    ray = np.stack([np.broadcast_to(xs[None, :], (H, W)), np.broadcast_to(ys[:, None], (H, W)), np.ones((H, W))], -1)
    t = (np.dot(n, p0)) / (ray @ n)
    alpha = np.full(H * W, a)
    return alpha, (a * t).reshape(-1), np.broadcast_to(a * np.asarray(n), (H * W, 3)).copy()


@pytest.mark.parametrize("n", [(0.0, 0.0, -1.0), (0.3, -0.2, -0.93)])
def test_normal_consistency_vanishes_on_a_plane(n):
    """Expected depth of a plane and its own normal as the rendered normal: N from the depth
    map equals the plane normal at every interior pixel, so A - N . N_r = 0."""
    cam = synthetic.make_camera((0.0, -3.0, 0.0), 24, 18)
    n = np.asarray(n) / np.linalg.norm(n)
    alpha, depth, normal = _plane_images(cam, n, np.array([0.0, 0.0, 3.0]))
    ln, ga, gd, gn = oracle.normal_consistency(alpha, depth, normal, cam)
    assert abs(ln) <= 1e-12
    valid = np.zeros((18, 24), bool)
    valid[1:-1, 1:-1] = True
    assert np.all(gn.reshape(18, 24, 3)[~valid] == 0.0)        # border pixels carry no term


def test_normal_consistency_gradient_matches_central_differences():
    cam = synthetic.make_camera((0.0, -3.0, 0.0), 12, 10)
    rng = np.random.default_rng(8)
    alpha, depth, normal = _plane_images(cam, np.array([0.2, 0.1, -0.97]) / np.linalg.norm([0.2, 0.1, -0.97]),
                                         np.array([0.0, 0.0, 3.0]))
    alpha = alpha + rng.uniform(0, 0.15, alpha.shape)
    depth = depth * (1 + rng.uniform(-0.02, 0.02, depth.shape))
    normal = normal + rng.normal(scale=0.05, size=normal.shape)
    ln, ga, gd, gn = oracle.normal_consistency(alpha, depth, normal, cam, weight=0.05)
    for arr, g in ((alpha, ga), (depth, gd), (normal, gn)):
        flat = arr.reshape(-1)
        for i in rng.choice(flat.size, size=8, replace=False):
            x0 = flat[i]
            flat[i] = x0 + 1e-6
            lp = oracle.normal_consistency(alpha, depth, normal, cam)[0]
            flat[i] = x0 - 1e-6
            lm = oracle.normal_consistency(alpha, depth, normal, cam)[0]
            flat[i] = x0
            assert g.reshape(-1)[i] == pytest.approx(0.05 * (lp - lm) / 2e-6, abs=1e-9)


# ----------------------------------------------------------------------------- 3DGS variant (Appendix B)
def _g3(xyz, scale, opacity, rgb, quat=None):
    xyz = np.asarray(xyz, np.float64).reshape(-1, 3)
    n = len(xyz)
    q = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)) if quat is None else np.asarray(quat, np.float64).reshape(n, 4)
    return dict(xyz=xyz, quat=q, scale=np.asarray(scale, np.float64).reshape(n, 3),
                opacity=np.asarray(opacity, np.float64).reshape(n),
                sh=((np.asarray(rgb, np.float64).reshape(n, 1, 3) - 0.5) * SQ2PI), sh_degree=0)


def test_ewa_isotropic_gaussian_on_the_axis():
    """An isotropic Gaussian of scale s at distance d on the optical axis projects to the
    image covariance ((f s / d)^2 + 0.3) I, so alpha at k pixels from the centre is
    o exp(-k^2 / (2 ((f s / d)^2 + 0.3)))."""
    cam = cam65()
    s, o = 0.04, 0.8
    g = _g3([0, 0, 0], [s, s, s], o, [0.3, 0.6, 0.9])
    var = (cam["fx"] * s / 3.0) ** 2 + 0.3
    for k in (0, 1, 2, 4):
        r = oracle.render_3d(g, cam, pix(cam, 32 + k, 32))
        a = o * math.exp(-0.5 * k * k / var)
        expect = a if (k * k / var <= 9.0 and a >= 1.0 / 255.0) else 0.0   # k = 4 lies past the cut
        assert r["alpha"][0] == pytest.approx(expect, abs=1e-13)
        assert r["depth"][0] == pytest.approx(3.0 * r["alpha"][0], abs=1e-12)
        np.testing.assert_allclose(r["rgb"][0], r["alpha"][0] * np.array([0.3, 0.6, 0.9]), atol=1e-13)


def test_ewa_covariance_is_the_linearised_projection():
    """J W Sigma W^T J^T equals the covariance pushed through the Jacobian of the pinhole
    projection of the world point, taken here by central differences."""
    cam = synthetic.make_camera((1.0, -3.0, 0.5), 80, 60)
    rng = np.random.default_rng(9)
    g = _g3(rng.uniform(-0.5, 0.5, (5, 3)), rng.uniform(0.02, 0.2, (5, 3)), [0.5] * 5, [[0.5] * 3] * 5,
            quat=rng.normal(size=(5, 4)))
    pr = oracle.project_ewa(g, cam)
    R, t = np.asarray(cam["viewmat"])[:3, :3], np.asarray(cam["viewmat"])[:3, 3]

    def proj(X):
        c = R @ X + t
        return np.array([cam["fx"] * c[0] / c[2] + cam["cx"], cam["fy"] * c[1] / c[2] + cam["cy"]])

    for i in range(5):
        X = g["xyz"][i]
        J = np.stack([(proj(X + h) - proj(X - h)) / 2e-6 for h in np.eye(3) * 1e-6], 1)   # [2,3]
        q = g["quat"][i] / np.linalg.norm(g["quat"][i])
        Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        S = Rq @ np.diag(g["scale"][i] ** 2) @ Rq.T
        ref = J @ S @ J.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(pr["cov2"][i].numpy(), ref, rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(pr["centre"][i].numpy(), proj(X), rtol=1e-12)


def test_ewa_hidden_gaussian_scores_zero():
    cam = cam65()
    g = _g3([[0, -1.0, 0], [0, -0.98, 0], [0, -0.96, 0], [0, 0.5, 0]], [[1.0, 0.01, 1.0]] * 3 + [[0.05] * 3],
            [0.97, 0.97, 0.97, 0.9], [[0.5] * 3] * 4)
    score = oracle.contribution_score_3d(g, [cam])
    assert score[3] == 0.0                                # behind three nearly opaque sheets
    assert score[0] == pytest.approx(0.97, abs=1e-12)     # the front sheet, hit at its centre
