"""Seeded synthetic inputs for the object-centric 2DGS rasterizer.

This module only *draws* inputs: surfel parameters, pinhole cameras and object
masks shaped like the paper's multi-view object captures (Sec. 5: DTU and
Mip-NeRF360 are replaced by synthetic object-centric scenes; no dataset item is
reproduced).  It holds none of the rasterizer's arithmetic (no projection,
ray-splat intersection, compositing, loss or pruning), so the FP64 oracle and
the CUDA path are both fed from here without sharing any method code.

Conventions of the data it produces:
  * parameters are float32 numpy arrays, one array per attribute
    (xyz [N,3], quat [N,4] as (w,x,y,z), scale [N,2], opacity [N],
    sh [N,(deg+1)^2,3]);
  * a camera is a dict with a row-major 4x4 world->camera ``viewmat``
    (OpenCV axes: +x right, +y down, +z forward), ``fx, fy, cx, cy``
    (pixels), ``width, height`` and ``near``;
  * a mask is a uint8 [H,W] array, 1 on the object (Sec. 4.2, M_i = 1 where
    the object is present).
"""
from __future__ import annotations

import math

import numpy as np

NEAR = 0.2
FOV_X_DEG = 60.0
RESOLUTIONS_C4 = ((640, 480), (800, 800), (1024, 768), (1600, 1200))


# ----------------------------------------------------------------------------- cameras
def look_at(position, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """World->camera 4x4 (OpenCV axes) for a camera at ``position`` facing ``target``."""
    c = np.asarray(position, np.float64)
    f = np.asarray(target, np.float64) - c
    f /= np.linalg.norm(f)
    up = np.asarray(up, np.float64)
    if abs(float(np.dot(f, up))) > 0.999:  # looking along the up axis: pick another up
        up = np.array([0.0, 1.0, 0.0])
    x = np.cross(f, up)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)  # points "down" in the image
    r_wc = np.stack([x, y, f], axis=1)  # columns: camera axes in world coordinates
    vm = np.eye(4)
    vm[:3, :3] = r_wc.T
    vm[:3, 3] = -r_wc.T @ c
    return vm


def _f32(x):
    """The nearest float32 value, as float64: the library's camera is float32, so both
    sides of a comparison see the same camera numbers."""
    return np.asarray(x, np.float32).astype(np.float64)


def make_camera(position, width: int, height: int, fov_x_deg: float = FOV_X_DEG,
                near: float = NEAR, target=(0.0, 0.0, 0.0), f32: bool = True) -> dict:
    """Pinhole camera with a horizontal field of view and the principal point at the centre.
    With ``f32`` (the default) every number is float32-representable, as the library holds
    it; without, the rotation is exactly orthonormal (for world-space checks of the oracle)."""
    rnd = _f32 if f32 else (lambda x: np.asarray(x, np.float64))
    fx = float(rnd((width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)))
    return dict(viewmat=rnd(look_at(position, target)), fx=fx, fy=fx, cx=float(rnd(width / 2.0)),
                cy=float(rnd(height / 2.0)), width=int(width), height=int(height), near=float(rnd(near)))


def hemisphere_positions(rng: np.random.Generator, n: int, radius: float) -> np.ndarray:
    """Camera centres uniform on the upper (z >= 0) hemisphere of the given radius."""
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d[:, 2] = np.abs(d[:, 2])
    return d * radius


# ----------------------------------------------------------------------------- surfels
def random_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random unit quaternions (normalised 4D Gaussian), (w,x,y,z)."""
    q = rng.normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def uniform_ball(rng: np.random.Generator, n: int, radius: float) -> np.ndarray:
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d * (radius * rng.random(n) ** (1.0 / 3.0))[:, None]


def uniform_shell(rng: np.random.Generator, n: int, r0: float, r1: float) -> np.ndarray:
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = (r0 ** 3 + (r1 ** 3 - r0 ** 3) * rng.random(n)) ** (1.0 / 3.0)
    return d * r[:, None]


def log_uniform(rng: np.random.Generator, shape, lo: float, hi: float) -> np.ndarray:
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=shape))


def quats_with_normal(rng: np.random.Generator, normals: np.ndarray) -> np.ndarray:
    """Unit quaternions whose rotation maps +z onto ``normals`` (random spin about it)."""
    n = normals / np.linalg.norm(normals, axis=1, keepdims=True)
    ez = np.array([0.0, 0.0, 1.0])
    axis = np.cross(np.broadcast_to(ez, n.shape), n)
    s = np.linalg.norm(axis, axis=1)
    cosang = np.clip(n[:, 2], -1.0, 1.0)
    ang = np.arctan2(s, cosang)
    axis = np.where(s[:, None] > 1e-12, axis / np.maximum(s, 1e-30)[:, None], np.array([1.0, 0.0, 0.0]))
    qa = np.concatenate([np.cos(ang / 2)[:, None], np.sin(ang / 2)[:, None] * axis], axis=1)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=len(n))
    qs = np.stack([np.cos(phi / 2), np.zeros_like(phi), np.zeros_like(phi), np.sin(phi / 2)], axis=1)
    # Hamilton product qa * qs (spin about the local z first, then align z with the normal)
    w1, x1, y1, z1 = qa.T
    w2, x2, y2, z2 = qs.T
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], axis=1)


def _pack(xyz, quat, scale, opacity, sh, degree) -> dict:
    return dict(xyz=np.ascontiguousarray(xyz, np.float32),
                quat=np.ascontiguousarray(quat, np.float32),
                scale=np.ascontiguousarray(scale, np.float32),
                opacity=np.ascontiguousarray(opacity, np.float32),
                sh=np.ascontiguousarray(sh, np.float32),
                sh_degree=int(degree))


def sh_dc_from_rgb(rgb: np.ndarray) -> np.ndarray:
    """Degree-0 coefficient whose rendered colour is ``rgb``.

    The degree-0 real SH function is the constant 1/(2 sqrt(pi)) and the
    renderer adds 0.5 to the SH sum, so c_00 = (rgb - 0.5) * 2 sqrt(pi).
    """
    return (rgb - 0.5) * (2.0 * math.sqrt(math.pi))


def object_scene(rng: np.random.Generator, n: int, degree: int, object_frac: float = 0.7,
                 object_radius: float = 0.8, shell=(2.0, 4.0), sh_sigma: float = 0.2,
                 scale_range=(0.01, 0.1)) -> dict:
    """Object sphere plus background shell (configs 2, 4, 5 of the workload list)."""
    n_obj = int(round(n * object_frac))
    xyz = np.concatenate([uniform_ball(rng, n_obj, object_radius),
                          uniform_shell(rng, n - n_obj, shell[0], shell[1])])
    k = (degree + 1) ** 2
    return _pack(xyz, random_quats(rng, n), log_uniform(rng, (n, 2), *scale_range),
                 rng.uniform(0.1, 0.9, size=n), rng.normal(0.0, sh_sigma, size=(n, k, 3)), degree)


# ----------------------------------------------------------------------------- masks
def disc_mask(width: int, height: int, radius_px: float) -> np.ndarray:
    """1 inside the disc of ``radius_px`` around the image centre (pixel centres at +0.5)."""
    x = np.arange(width) + 0.5 - width / 2.0
    y = np.arange(height) + 0.5 - height / 2.0
    return ((x[None, :] ** 2 + y[:, None] ** 2) <= radius_px ** 2).astype(np.uint8)


def sphere_mask(cam: dict, radius: float, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """1 where the pixel-centre ray of ``cam`` hits the sphere (the object's silhouette)."""
    w, h = cam["width"], cam["height"]
    vm = np.asarray(cam["viewmat"], np.float64)
    r_cw, t = vm[:3, :3], vm[:3, 3]
    origin = -r_cw.T @ t
    x = (np.arange(w) + 0.5 - cam["cx"]) / cam["fx"]
    y = (np.arange(h) + 0.5 - cam["cy"]) / cam["fy"]
    d_cam = np.stack(np.broadcast_arrays(x[None, :], y[:, None], np.ones((1, 1))), axis=-1)
    d = d_cam @ r_cw  # rows: r_cw^T d_cam
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    oc = origin - np.asarray(center, np.float64)
    b = d @ oc
    disc = b * b - (oc @ oc - radius * radius)
    hit = (disc >= 0) & ((-b + np.sqrt(np.maximum(disc, 0))) > 0)
    return hit.astype(np.uint8)


# ----------------------------------------------------------------------------- workloads
def config1(seed: int = 1) -> dict:
    """Plain forward, one 128x128 view, 2,000 surfels, SH degree 0, disc mask r=40 px."""
    rng = np.random.default_rng(seed)
    n = 2000
    rgb = rng.uniform(0.0, 1.0, size=(n, 1, 3))
    g = _pack(uniform_ball(rng, n, 1.0), random_quats(rng, n), log_uniform(rng, (n, 2), 0.01, 0.1),
              rng.uniform(0.1, 0.9, size=n), sh_dc_from_rgb(rgb), 0)
    cam = make_camera((0.0, -3.0, 0.0), 128, 128)
    return dict(name="c1_fwd_128px_2k", gaussians=g, cameras=[cam], masks=[disc_mask(128, 128, 40.0)])


def config2(seed: int = 2, n: int = 100_000, width: int = 800, height: int = 800) -> dict:
    """Forward + backward, one 800x800 view, 100k surfels, SH degree 3, sphere mask."""
    rng = np.random.default_rng(seed)
    g = object_scene(rng, n, 3)
    cam = make_camera((0.0, -3.0, 0.0), width, height)
    return dict(name=f"c2_fwdbwd_{width}px_{n // 1000}k", gaussians=g, cameras=[cam],
                masks=[sphere_mask(cam, 0.8)])


def config3(seed: int = 3, n_views: int = 100, width: int = 800, height: int = 800,
            shell_counts=(60_000, 60_000, 60_000), n_interior: int = 120_000,
            shell_scale=(0.04, 0.06)) -> dict:
    """Occlusion pruning sweep: three dense tangent shells hide an interior cloud.

    Shell radii 1.00, 0.97, 0.94; shell surfels are tangent to the sphere
    (normal radial), scales U(shell_scale) (default U(0.04, 0.06)), opacity
    0.95; the interior surfels sit in r < 0.7 with the config-2 scale law.
    Cameras sit on the upper hemisphere of radius 3 and look at the origin.
    A scaled-down scene keeps the shells closed with fewer, larger surfels.
    """
    rng = np.random.default_rng(seed)
    xyz, quat, scale, opac = [], [], [], []
    for r, m in zip((1.00, 0.97, 0.94), shell_counts):
        d = rng.normal(size=(m, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        xyz.append(d * r)
        quat.append(quats_with_normal(rng, d))
        scale.append(rng.uniform(shell_scale[0], shell_scale[1], size=(m, 2)))
        opac.append(np.full(m, 0.95))
    xyz.append(uniform_ball(rng, n_interior, 0.7))
    quat.append(random_quats(rng, n_interior))
    scale.append(log_uniform(rng, (n_interior, 2), 0.01, 0.1))
    opac.append(rng.uniform(0.1, 0.9, size=n_interior))
    n = sum(shell_counts) + n_interior
    sh = rng.normal(0.0, 0.2, size=(n, 16, 3))
    g = _pack(np.concatenate(xyz), np.concatenate(quat), np.concatenate(scale),
              np.concatenate(opac), sh, 3)
    cams = [make_camera(p, width, height) for p in hemisphere_positions(rng, n_views, 3.0)]
    return dict(name=f"c3_prune_{n // 1000}k_{n_views}v", gaussians=g, cameras=cams,
                n_shell=sum(shell_counts), n_interior=n_interior)


def config4(seed: int = 4, n: int = 500_000, n_views: int = 16, resolutions=RESOLUTIONS_C4) -> dict:
    """Batched fwd+bwd: 500k surfels SH3, 16 hemisphere views of uneven resolution."""
    rng = np.random.default_rng(seed)
    g = object_scene(rng, n, 3)
    res = [resolutions[i] for i in rng.integers(0, len(resolutions), size=n_views)]
    pos = hemisphere_positions(rng, n_views, 3.0)
    cams = [make_camera(p, w, h) for p, (w, h) in zip(pos, res)]
    return dict(name=f"c4_batched_{n // 1000}k_{n_views}v", gaussians=g, cameras=cams,
                masks=[sphere_mask(c, 0.8) for c in cams])


def config5(seed: int = 5, n: int = 1_000_000, n_views: int = 64, width: int = 1600,
            height: int = 1200) -> dict:
    """Training-iteration shape: 1M surfels (60% object / 40% shell), 64 views 1600x1200."""
    rng = np.random.default_rng(seed)
    g = object_scene(rng, n, 3, object_frac=0.6)
    cams = [make_camera(p, width, height) for p in hemisphere_positions(rng, n_views, 3.0)]
    return dict(name=f"c5_train_{n // 1000}k_{n_views}v", gaussians=g, cameras=cams,
                masks=[sphere_mask(c, 0.8) for c in cams])


def small_scene(seed: int, n: int, width: int, height: int, degree: int = 1,
                n_views: int = 1, scale_range=(0.03, 0.15), cam_radius: float = 3.0) -> dict:
    """A few-tile scene with ragged image edges, for element-by-element parity."""
    rng = np.random.default_rng(seed)
    k = (degree + 1) ** 2
    g = _pack(uniform_ball(rng, n, 1.0), random_quats(rng, n), log_uniform(rng, (n, 2), *scale_range),
              rng.uniform(0.1, 0.9, size=n), rng.normal(0.0, 0.3, size=(n, k, 3)), degree)
    if n_views == 1:
        pos = np.array([[0.3, -cam_radius, 0.4]])
    else:
        pos = hemisphere_positions(rng, n_views, cam_radius)
    cams = [make_camera(p, width, height) for p in pos]
    return dict(name=f"small_{n}_{width}x{height}_{n_views}v", gaussians=g, cameras=cams,
                masks=[sphere_mask(c, 0.6) for c in cams])
