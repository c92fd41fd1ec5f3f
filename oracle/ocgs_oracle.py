"""FP64 CPU oracle of the object-centric 2DGS rasterizer — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The product path (the CUDA library and
its Python binding) never imports, calls or falls back to it.

What it computes is the plain definition of the method, written in FP64
PyTorch CPU ops so that reverse-mode autograd gives the exact adjoint of the
same procedure with its discrete decisions (skip, stop, clamp, min branch,
normal flip) held fixed:

* per pixel, every non-culled surfel is a candidate; candidates are taken in
  ascending centre depth, ties by ascending index (the front-to-back
  compositing order of Sec. 4.3);
* the ray through the pixel centre meets the surfel plane at (u, v), found as
  the crossing of the two homogeneous pixel planes pulled back through the
  surfel's 3x3 splat-to-pixel matrix (2DGS ray-splat intersection, prior work
  the paper builds on, Sec. 3.2 and Sec. 5.1);
* rho = min(u^2 + v^2, |x - c|^2 / sigma_f^2) with sigma_f^2 = 1/2 px^2
  (screen-space low-pass filter), alpha = min(0.99, o exp(-rho/2));
  a candidate is skipped if rho > 9 or alpha < 1/255, and compositing stops
  at the first candidate for which T (1 - alpha) < 1e-4, which is not
  blended (Sec. 4.3: rendering ends once the pixel reaches an opacity close
  to 1, or the candidates are exhausted);
* blending weight w = alpha T; colour C = sum w rgb, accumulated opacity
  A = sum w (the A_i of Eq. 1), depth D = sum w z, normal N = sum w n;
* background loss L_b = (1/(h w)) sum A (1 - M) (Eq. 1);
* contribution score of a surfel = max blending weight over all pixels of
  all views; the surfel is "used" (visible, not occluded) iff the score is
  > 0 (Sec. 4.3), and the keep-set at threshold tau is {score > tau};
* one Adam update of the parameters (the optimiser of the training Sec. 5.1
  keeps; Kingma & Ba, 2015, Algorithm 1);
* the L1 part of the masked photometric loss of Eq. 2 with its adjoint;
* SSIM of masked images (the D-SSIM part of the photometric loss Eq. 2 masks,
  and the masked SSIM of Sec. 5) and the masked PSNR of Sec. 5;
* the 2DGS depth distortion and normal consistency of Eq. 3, from the composited
  planes (their readings: squared depth distances, expected-depth normals).

Readings of points the paper leaves to prior work (documented with the
project's design notes): culling of a surfel whose 3-sigma square reaches
the near plane; depth z = camera depth of the ray-plane hit when the surfel
term wins the min, else the centre depth; normals flipped to face the
camera; SH colour max(0, sum c_lm Y_lm(d) + 0.5) with the real SH basis with
Condon-Shortley phase.  Parity of these readings against the paper itself is
unpinned: the paper does not fix them.

Inputs are numpy arrays (see ``synthetic.py`` for the layout).
"""
from __future__ import annotations

import contextlib
import math
from typing import Optional

import numpy as np
import torch

DT = torch.float64

SIGMA_F2 = 0.5          # low-pass filter variance, px^2 (sigma_f = sqrt(2)/2 px)
RHO_CUT = 9.0           # support cut-off, rho <= 9 (3 sigma)
ALPHA_MIN = 1.0 / 255.0  # skip candidates below this opacity
ALPHA_MAX = 0.99        # opacity clamp
T_EPS = 1e-4            # stop once the transmittance would fall below this

FRAGILE_REL = 1e-5      # relative margin for flagging decisions FP32 may take differently


@contextlib.contextmanager
def evaluated_in(dtype):
    """Evaluate the same definitions in another floating-point type inside the block (not
    thread-safe).  Tests use float32 to measure how far any float32 evaluation of the
    definition lands from FP64 for each output, the conditioning their tolerances allow for;
    results outside the block are FP64."""
    global DT
    old, DT = DT, dtype
    try:
        yield
    finally:
        DT = old


# ----------------------------------------------------------------------------- helpers
def _t(a) -> torch.Tensor:
    return torch.as_tensor(np.asarray(a, dtype=np.float64), dtype=DT)


def quat_to_rotmat(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrix of unit quaternions q = (w, x, y, z) (Hamilton convention), [N,3,3]."""
    w, x, y, z = q.unbind(-1)
    r00 = 1 - 2 * (y * y + z * z)
    r01 = 2 * (x * y - w * z)
    r02 = 2 * (x * z + w * y)
    r10 = 2 * (x * y + w * z)
    r11 = 1 - 2 * (x * x + z * z)
    r12 = 2 * (y * z - w * x)
    r20 = 2 * (x * z - w * y)
    r21 = 2 * (y * z + w * x)
    r22 = 1 - 2 * (x * x + y * y)
    return torch.stack([torch.stack([r00, r01, r02], -1),
                        torch.stack([r10, r11, r12], -1),
                        torch.stack([r20, r21, r22], -1)], -2)


def sh_basis(d: torch.Tensor, degree: int) -> torch.Tensor:
    """Real spherical harmonics of unit directions d [N,3], degrees 0..degree, [N,(deg+1)^2].

    Basis: for m > 0, sqrt(2) Re Y_l^m; for m < 0, sqrt(2) Im Y_l^|m|; Y_l^0 for
    m = 0, where Y_l^m are the complex orthonormal harmonics with the
    Condon-Shortley phase.  Order within a degree: m = -l .. l.
    """
    x, y, z = d.unbind(-1)
    pi = math.pi
    out = [torch.full_like(x, 0.5 / math.sqrt(pi))]
    if degree >= 1:
        k1 = math.sqrt(3.0 / (4.0 * pi))
        out += [-k1 * y, k1 * z, -k1 * x]
    if degree >= 2:
        k2a = 0.5 * math.sqrt(15.0 / pi)
        k2b = 0.25 * math.sqrt(5.0 / pi)
        k2c = 0.25 * math.sqrt(15.0 / pi)
        out += [k2a * x * y, -k2a * y * z, k2b * (2 * z * z - x * x - y * y),
                -k2a * x * z, k2c * (x * x - y * y)]
    if degree >= 3:
        k3a = math.sqrt(70.0 / pi) / 8.0
        k3b = 0.5 * math.sqrt(105.0 / pi)
        k3c = math.sqrt(42.0 / pi) / 8.0
        k3d = 0.25 * math.sqrt(7.0 / pi)
        k3e = 0.25 * math.sqrt(105.0 / pi)
        out += [-k3a * y * (3 * x * x - y * y),
                k3b * x * y * z,
                -k3c * y * (4 * z * z - x * x - y * y),
                k3d * z * (2 * z * z - 3 * x * x - 3 * y * y),
                -k3c * x * (4 * z * z - x * x - y * y),
                k3e * z * (x * x - y * y),
                -k3a * x * (x * x - 3 * y * y)]
    if degree > 3:
        raise ValueError("SH degree must be 0..3")
    return torch.stack(out, -1)


def camera_tensors(cam: dict):
    vm = _t(cam["viewmat"])
    K = _t([[cam["fx"], 0.0, cam["cx"]], [0.0, cam["fy"], cam["cy"]], [0.0, 0.0, 1.0]])
    return vm[:3, :3], vm[:3, 3], K


def param_tensors(g: dict, requires_grad: bool = False) -> dict:
    out = {k: _t(g[k]).requires_grad_(requires_grad) for k in ("xyz", "quat", "scale", "opacity", "sh")}
    return out


# ----------------------------------------------------------------------------- projection
def project(p: dict, cam: dict, sh_degree: int) -> dict:
    """Per-surfel, per-view quantities (differentiable w.r.t. the parameters in ``p``).

    The surfel is P(u,v) = x + s_u t_u u + s_v t_v v, with t_u, t_v the first
    two columns of the rotation of the normalised quaternion.  Its 3x3
    splat-to-pixel matrix is T = K [R s_u t_u, R s_v t_v, R x + t], so that
    (x z, y z, z)^T = T (u, v, 1)^T for the image point of P(u,v).
    """
    r_cw, t_cw, K = camera_tensors(cam)
    q = p["quat"] / p["quat"].norm(dim=-1, keepdim=True)
    rot = quat_to_rotmat(q)
    t_u, t_v = rot[..., 0], rot[..., 1]
    su, sv = p["scale"][:, 0:1], p["scale"][:, 1:2]
    U = (su * t_u) @ r_cw.T             # camera-frame tangent axes (scaled)
    V = (sv * t_v) @ r_cw.T
    pc = p["xyz"] @ r_cw.T + t_cw       # camera-frame centre
    Hc = torch.stack([U, V, pc], dim=-1)  # [N,3,3], columns act on (u, v, 1)
    T = K @ Hc
    z_c = pc[:, 2]
    # cull a surfel whose 3-sigma square has a corner at or behind the near plane
    z_min = z_c - 3.0 * (U[:, 2].abs() + V[:, 2].abs())
    culled = (z_min <= cam["near"]).detach()
    # camera-frame normal, flipped to face the camera
    n_cam = torch.linalg.cross(t_u, t_v) @ r_cw.T
    facing = ((n_cam * pc).sum(-1) > 0).detach()
    n_cam = torch.where(facing[:, None], -n_cam, n_cam)
    # view-dependent colour
    campos = -(r_cw.T @ t_cw)
    d = p["xyz"] - campos
    d = d / d.norm(dim=-1, keepdim=True)
    basis = sh_basis(d, sh_degree)                         # [N,K]
    rgb_raw = (basis[:, :, None] * p["sh"]).sum(1) + 0.5   # [N,3]
    rgb = rgb_raw.clamp(min=0.0)
    return dict(T=T, z_c=z_c, culled=culled, normal=n_cam, rgb=rgb, rgb_raw=rgb_raw,
                opacity=p["opacity"], cull_margin=(z_min - cam["near"]).detach())


def depth_order(z_c: torch.Tensor) -> torch.Tensor:
    """Front-to-back order: ascending centre depth, ties by ascending index.  The depth that
    decides the order is rounded to float32, the precision of the device's sort keys: an
    order is a discrete decision, so both sides take it in the same precision (two surfels
    whose depths round to the same float32 value are ordered by index on both sides)."""
    return torch.sort(z_c.detach().to(torch.float32), stable=True).indices


# ----------------------------------------------------------------------------- candidates
def candidate_mask(T: torch.Tensor, scale: torch.Tensor, cam: dict, xs: torch.Tensor,
                   ys: torch.Tensor) -> torch.Tensor:
    """Conservative candidate test [B,n]: False only where rho > 9 is certain.

    rho <= 9 needs either u^2 + v^2 <= 9, whose hit point lies within
    3 max(s_u, s_v) of the centre so the pixel ray passes that close to it, or
    |x - c|^2 <= 9 sigma_f^2.  Dropping the other candidates cannot change a
    result: they are skipped by the support test anyway.
    """
    with torch.no_grad():
        pc_x = (T[:, 0, 2] - cam["cx"] * T[:, 2, 2]) / cam["fx"]
        pc_y = (T[:, 1, 2] - cam["cy"] * T[:, 2, 2]) / cam["fy"]
        pc = torch.stack([pc_x, pc_y, T[:, 2, 2]], -1)               # camera-frame centre
        r = 3.0 * scale.max(dim=-1).values
        dx = (xs - cam["cx"]) / cam["fx"]
        dy = (ys - cam["cy"]) / cam["fy"]
        dirs = torch.stack([dx, dy, torch.ones_like(dx)], -1)
        dirs = dirs / dirs.norm(dim=-1, keepdim=True)                 # [B,3]
        proj = dirs @ pc.T                                            # [B,n]
        dist2 = (pc * pc).sum(-1)[None, :] - proj * proj
        near_ray = dist2 <= (r * r)[None, :] * (1 + 1e-6) + 1e-12
        cx = T[:, 0, 2] / T[:, 2, 2]
        cy = T[:, 1, 2] / T[:, 2, 2]
        fd2 = (xs[:, None] - cx[None, :]) ** 2 + (ys[:, None] - cy[None, :]) ** 2
        near_c = fd2 <= RHO_CUT * SIGMA_F2 * (1 + 1e-6)
        return near_ray | near_c


# ----------------------------------------------------------------------------- compositing
def front_to_back(rho, opacity):
    """Front-to-back compositing weights of Sec. 4.3 from each candidate's rho
    (columns already in depth order, rows are pixels): alpha = min(0.99, o exp(-rho/2)),
    a candidate with rho > 9 or alpha < 1/255 is skipped, and a pixel stops at the first
    candidate that would take its transmittance T (1 - alpha) below 1e-4 (that one is not
    blended).  Returns the weights w = alpha T_before of the blended candidates, the
    final transmittance and the decisions that a float32 evaluation may take the other
    way (the rho cut, the 1/255 floor, the stop)."""
    alpha_raw = opacity[None] * torch.exp(-0.5 * rho)
    alpha = alpha_raw.clamp(max=ALPHA_MAX)
    valid = ((rho <= RHO_CUT) & (alpha >= ALPHA_MIN)).detach()
    a = torch.where(valid, alpha, torch.zeros_like(alpha))
    one_minus = 1.0 - a
    t_incl = torch.cumprod(one_minus, dim=1)
    blended = (valid & (t_incl.detach() >= T_EPS))
    t_excl = torch.cat([torch.ones(rho.shape[0], 1, dtype=DT), t_incl[:, :-1]], dim=1)
    w = torch.where(blended, a * t_excl, torch.zeros_like(a))
    t_final = torch.where(blended, one_minus, torch.ones_like(a)).prod(1)
    with torch.no_grad():
        e = FRAGILE_REL
        a_at_cut = (opacity * math.exp(-0.5 * RHO_CUT)).clamp(max=ALPHA_MAX)
        f_cut = ((rho - RHO_CUT).abs() <= e * RHO_CUT) & (a_at_cut[None] >= ALPHA_MIN * (1 - e))
        f_amin = ((alpha_raw - ALPHA_MIN).abs() <= e * ALPHA_MIN) & (rho <= RHO_CUT * (1 + e))
        f_stop = valid & ((t_incl - T_EPS).abs() <= e * T_EPS)
    return dict(w=w, t_final=t_final, blended=blended, alpha_raw=alpha_raw, n_blended=blended.sum(1),
                at_edge=f_cut | f_amin | f_stop)


def composite(T, z_c, normal, rgb, opacity, xs, ys, rgb_raw=None):
    """Front-to-back compositing of the candidates (columns, already in depth order)
    for the pixel centres (xs, ys) (rows).  Returns per-pixel outputs and the
    per-candidate blending weights."""
    B = xs.shape[0]
    n = T.shape[0]
    if n == 0:
        z = torch.zeros(B, dtype=DT)
        return dict(rgb=torch.zeros(B, 3, dtype=DT), alpha=z, depth=z.clone(), depth2=z.clone(),
                    normal=torch.zeros(B, 3, dtype=DT), t_final=torch.ones(B, dtype=DT),
                    n_blended=torch.zeros(B, dtype=torch.int64),
                    fragile=torch.zeros(B, dtype=torch.bool),
                    fragile_grad=torch.zeros(B, dtype=torch.bool), w=torch.zeros(B, 0, dtype=DT),
                    z=torch.zeros(B, 0, dtype=DT))
    # homogeneous pixel planes h_x = (-1, 0, x), h_y = (0, -1, y) pulled back to (u, v, 1)
    row0, row1, row2 = T[:, 0, :], T[:, 1, :], T[:, 2, :]
    h_u = -row0[None] + xs[:, None, None] * row2[None]   # [B,n,3]
    h_v = -row1[None] + ys[:, None, None] * row2[None]
    cr = torch.linalg.cross(h_u, h_v)
    degenerate = (cr[..., 2] == 0).detach()
    w_h = torch.where(degenerate, torch.ones_like(cr[..., 2]), cr[..., 2])
    u = cr[..., 0] / w_h
    v = cr[..., 1] / w_h
    rho3 = torch.where(degenerate, torch.full_like(u, math.inf), u * u + v * v)
    cx = row0[:, 2] / row2[:, 2]
    cy = row1[:, 2] / row2[:, 2]
    rho2 = ((xs[:, None] - cx[None]) ** 2 + (ys[:, None] - cy[None]) ** 2) / SIGMA_F2
    rho = torch.minimum(rho3, rho2)
    use_hit = (rho3 <= rho2).detach()
    z_hit = row2[None, :, 0] * u + row2[None, :, 1] * v + row2[None, :, 2]
    z = torch.where(use_hit, z_hit, z_c[None].expand(B, n))
    fb = front_to_back(rho, opacity)
    w, blended, alpha_raw = fb["w"], fb["blended"], fb["alpha_raw"]
    out = dict(
        rgb=w @ rgb, alpha=w.sum(1), depth=(w * z).sum(1), depth2=(w * z * z).sum(1), normal=w @ normal,
        t_final=fb["t_final"], n_blended=fb["n_blended"], w=w, z=z)
    # decisions that a float32 evaluation may take the other way (besides those of the
    # compositing): the surfel/filter switch, and for gradients the clamp
    with torch.no_grad():
        e = FRAGILE_REL
        f_branch = blended & ((rho3 - rho2).abs() <= e * torch.maximum(rho3.clamp(max=1e30), rho2))
        at_edge = fb["at_edge"] | f_branch
        fragile = at_edge.any(1)
        f_clamp = blended & ((alpha_raw - ALPHA_MAX).abs() <= e)
        f_grad = f_clamp
        if rgb_raw is not None:
            g_col = (rgb_raw.abs() <= e).any(-1)
            f_grad = f_grad | (blended & g_col[None])
        out["fragile"] = fragile
        out["fragile_grad"] = fragile | f_grad.any(1)
        out["at_edge"] = at_edge  # [B, n]: the candidate itself is at a fragile threshold
    return out


# ----------------------------------------------------------------------------- render
def pixel_centres(cam: dict, pixels: Optional[np.ndarray]):
    W, H = cam["width"], cam["height"]
    if pixels is None:
        pixels = np.arange(W * H)
    pixels = np.asarray(pixels, np.int64)
    xs = _t(pixels % W + 0.5)
    ys = _t(pixels // W + 0.5)
    return pixels, xs, ys


def render(g: dict, cam: dict, pixels: Optional[np.ndarray] = None, d_out: Optional[dict] = None,
           prefilter: bool = True, chunk: int = 256, pair_powers=()) -> dict:
    """Render one view at the given flat pixel indices (row-major, default all).

    Returns numpy FP64 arrays: rgb [P,3], alpha [P], depth [P], depth2 [P]
    (sum of w z^2, for the depth distortion), normal [P,3], t_final [P],
    n_blended [P], fragile [P], fragile_grad [P], and score [N] (max blending
    weight of each surfel over these pixels), with score_firm [N] (the same max
    over the pixels that are not fragile) and at_edge [N] (the surfel is itself
    at a fragile threshold at some pixel).  A score is certain in float32 where
    the surfel is not at_edge and its max is reached at a firm pixel (score ==
    score_firm); elsewhere a float32 evaluation may differ.  If ``d_out`` holds cotangents
    (rgb, alpha, depth, normal, optionally depth2) for these pixels, also
    returns ``grads``: d(sum <d_out, out>)/d(xyz, quat, scale, opacity, sh).
    For every p in ``pair_powers`` it also returns ``distortion_pairs_<p>`` [P]:
    the depth distortion of Eq. 3 by brute force over each pixel's blended
    pairs, sum_{i,j} w_i w_j |z_i - z_j|^p (p = 1 is the form 2DGS prints,
    p = 2 the squared reading; a diagnostic, not differentiated).
    """
    need_grad = d_out is not None
    params = param_tensors(g, requires_grad=need_grad)
    N = params["xyz"].shape[0]
    pixels, xs_all, ys_all = pixel_centres(cam, pixels)
    P = len(pixels)
    proj = project(params, cam, g["sh_degree"])
    alive = torch.nonzero(~proj["culled"]).flatten()
    order = alive[depth_order(proj["z_c"][alive])]          # front-to-back candidate list
    keys = ("T", "z_c", "normal", "rgb", "opacity")
    base = {k: proj[k].detach() for k in keys}
    acc = {k: torch.zeros_like(base[k]) for k in keys} if need_grad else None
    res = dict(rgb=np.zeros((P, 3)), alpha=np.zeros(P), depth=np.zeros(P), depth2=np.zeros(P), normal=np.zeros((P, 3)),
               t_final=np.ones(P), n_blended=np.zeros(P, np.int64), fragile=np.zeros(P, bool),
               fragile_grad=np.zeros(P, bool))
    for pw in pair_powers:
        res[f"distortion_pairs_{pw}"] = np.zeros(P)
    score = torch.zeros(N, dtype=DT)
    score_firm = torch.zeros(N, dtype=DT)        # max weight over the pixels that are not fragile
    at_edge = torch.zeros(N, dtype=torch.bool)   # the surfel is itself at a fragile threshold somewhere
    if need_grad:
        dts = {k: _t(d_out[k]) for k in ("rgb", "alpha", "depth", "normal")}
        dts["depth2"] = _t(d_out["depth2"]) if "depth2" in d_out else torch.zeros(P, dtype=DT)
    scale_d = params["scale"].detach()
    rgb_raw = proj["rgb_raw"].detach()
    for s in range(0, P, chunk):
        e = min(P, s + chunk)
        xs, ys = xs_all[s:e], ys_all[s:e]
        cols = order
        if prefilter and len(order) > 0:
            T_o, s_o = base["T"][order], scale_d[order]
            hit = torch.zeros(len(order), dtype=torch.bool)
            for r0 in range(0, e - s, 32):  # rows in small groups to bound memory
                hit |= candidate_mask(T_o, s_o, cam, xs[r0:r0 + 32], ys[r0:r0 + 32]).any(0)
            cols = order[hit]
        sub = {k: base[k][cols].clone().requires_grad_(need_grad) for k in keys}
        out = composite(sub["T"], sub["z_c"], sub["normal"], sub["rgb"], sub["opacity"], xs, ys,
                        rgb_raw=rgb_raw[cols])
        for k in ("rgb", "alpha", "depth", "depth2", "normal", "t_final", "n_blended", "fragile", "fragile_grad"):
            res[k][s:e] = out[k].detach().numpy()
        if len(cols):
            w_d = out["w"].detach()
            score[cols] = torch.maximum(score[cols], w_d.max(0).values)
            firm = ~out["fragile"]
            if firm.any():
                score_firm[cols] = torch.maximum(score_firm[cols], w_d[firm].max(0).values)
            at_edge[cols] |= out["at_edge"].any(0)
        for pw in pair_powers:
            w_d, z_d = out["w"].detach(), out["z"].detach()
            for b in range(e - s):
                nz = torch.nonzero(w_d[b]).flatten()
                wb, zb = w_d[b, nz], z_d[b, nz]
                res[f"distortion_pairs_{pw}"][s + b] = float(
                    (wb[:, None] * wb[None, :] * (zb[:, None] - zb[None, :]).abs() ** pw).sum())
        if need_grad and len(cols):
            loss = ((out["rgb"] * dts["rgb"][s:e]).sum() + (out["alpha"] * dts["alpha"][s:e]).sum()
                    + (out["depth"] * dts["depth"][s:e]).sum() + (out["normal"] * dts["normal"][s:e]).sum()
                    + (out["depth2"] * dts["depth2"][s:e]).sum())
            gs = torch.autograd.grad(loss, [sub[k] for k in keys], allow_unused=True)
            for k, gk in zip(keys, gs):
                if gk is not None:
                    acc[k].index_add_(0, cols, gk)
    res["score"] = score.numpy()
    res["score_firm"] = score_firm.numpy()
    res["at_edge"] = at_edge.numpy()
    res["cull_margin"] = proj["cull_margin"].numpy()
    if need_grad:
        torch.autograd.backward([proj[k] for k in keys], [acc[k] for k in keys])
        res["grads"] = {k: (params[k].grad.numpy() if params[k].grad is not None
                            else np.zeros(params[k].shape)) for k in params}
    return res


def render_views(g: dict, cams: list, d_outs: Optional[list] = None, pixels: Optional[list] = None,
                 prefilter: bool = True) -> list:
    """``render`` over several views; gradients (if requested) are per view."""
    out = []
    for i, cam in enumerate(cams):
        out.append(render(g, cam, None if pixels is None else pixels[i],
                          None if d_outs is None else d_outs[i], prefilter=prefilter))
    return out


# ----------------------------------------------------------------------------- paper's additions
def background_loss(alpha: np.ndarray, mask: np.ndarray) -> float:
    """L_b = (1 / (h w)) sum A (1 - M) over one view (Eq. 1); alpha and mask are [h,w]."""
    a = np.asarray(alpha, np.float64)
    m = np.asarray(mask, np.float64)
    return float(np.sum(a * (1.0 - m)) / a.size)


def background_loss_grad(mask: np.ndarray, gamma: float) -> np.ndarray:
    """d(gamma L_b)/dA = gamma (1 - M) / (h w) (Eq. 1 weighted as in Eq. 3)."""
    m = np.asarray(mask, np.float64)
    return gamma * (1.0 - m) / m.size


def masked_l1(rgb: np.ndarray, target: np.ndarray, mask: np.ndarray, weight: float = 1.0):
    """L1 part of the photometric loss of Eq. 2 on the masked images of one view.

    rgb (the rendering R) and target (the image I) are [h*w, 3], mask M is [h*w]
    and multiplies every colour channel.  Returns the mean over the 3 h w values
    of |I M - R M| and d(weight L1)/dR = weight sign(R M - I M) M / (3 h w), which
    is 0 where the two masked values are equal (the subgradient taken at the kink).
    """
    r = np.asarray(rgb, np.float64).reshape(-1, 3)
    t = np.asarray(target, np.float64).reshape(-1, 3)
    m = np.asarray(mask, np.float64).reshape(-1, 1)
    diff = r * m - t * m
    loss = float(np.abs(diff).sum() / diff.size)
    grad = weight * np.sign(diff) * m / diff.size
    return loss, grad


def contribution_score(g: dict, cams: list, prefilter: bool = True) -> np.ndarray:
    """Max blending weight of every surfel over all pixels of all views (Sec. 4.3)."""
    score = np.zeros(len(g["opacity"]))
    for cam in cams:
        score = np.maximum(score, render(g, cam, prefilter=prefilter)["score"])
    return score


def keep_set(score: np.ndarray, tau: float, borderline: float = 1e-6):
    """Keep-set {score > tau} and the indices whose score lies within ``borderline`` of tau."""
    s = np.asarray(score, np.float64)
    keep = s > tau
    near = np.nonzero(np.abs(s - tau) <= borderline)[0]
    return keep, near


def prune(g: dict, keep: np.ndarray) -> dict:
    """Keep the surfels flagged in ``keep``, in their original order."""
    out = {k: np.asarray(g[k])[keep] for k in ("xyz", "quat", "scale", "opacity", "sh")}
    out["sh_degree"] = g["sh_degree"]
    return out


def adam_step(params: dict, grads: dict, m: dict, v: dict, lr, step: int,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15):
    """One Adam update in FP64 (Kingma & Ba, 2015, Algorithm 1), the optimiser of
    the 2DGS training whose schedule Sec. 5.1 keeps.  For every element:
    biased moments m and v, their bias-corrected values, then the parameter step.
    Returns new (params, m, v) dicts; the inputs are not modified.  ``lr`` is a
    number or a dict with one learning rate per array."""
    keys = ("xyz", "quat", "scale", "opacity", "sh")
    new_p, new_m, new_v = {}, {}, {}
    for k in keys:
        rate = float(lr[k]) if isinstance(lr, dict) else float(lr)
        g = np.asarray(grads[k], np.float64)
        mk = beta1 * np.asarray(m[k], np.float64) + (1.0 - beta1) * g
        vk = beta2 * np.asarray(v[k], np.float64) + (1.0 - beta2) * g * g
        m_hat = mk / (1.0 - beta1 ** step)
        v_hat = vk / (1.0 - beta2 ** step)
        new_p[k] = np.asarray(params[k], np.float64) - rate * m_hat / (np.sqrt(v_hat) + eps)
        new_m[k] = mk
        new_v[k] = vk
    return new_p, new_m, new_v


# ----------------------------------------------------------------------------- photometric metrics and D-SSIM
# SSIM as the 3DGS photometric loss (the L_c that Eq. 2 masks) and the evaluation of Sec. 5 use
# it: windowed statistics under an 11x11 Gaussian window of sigma 1.5 (zero outside the
# image), stabilising constants C1 = 0.01^2, C2 = 0.03^2 for intensities in [0, 1].
SSIM_RADIUS = 5
SSIM_SIGMA = 1.5
SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2


def ssim_window() -> np.ndarray:
    """The normalised 1-D Gaussian of the separable SSIM window (11 taps)."""
    x = np.arange(-SSIM_RADIUS, SSIM_RADIUS + 1, dtype=np.float64)
    w = np.exp(-x * x / (2.0 * SSIM_SIGMA ** 2))
    return w / w.sum()


def ssim_blur(x: torch.Tensor) -> torch.Tensor:
    """Windowed mean of every channel of an [h, w, c] FP64 image, zero outside the image."""
    g = torch.tensor(ssim_window(), dtype=torch.float64)
    k = (g[:, None] * g[None, :])[None, None]                       # [1,1,11,11]
    planes = x.permute(2, 0, 1).unsqueeze(1)                         # [c,1,h,w]
    out = torch.nn.functional.conv2d(planes, k, padding=SSIM_RADIUS)
    return out.squeeze(1).permute(1, 2, 0)


def ssim_map(x1: torch.Tensor, x2: torch.Tensor) -> torch.Tensor:
    """Per-pixel, per-channel SSIM of two [h, w, 3] images: luminance, contrast and structure
    terms from the windowed means, variances and covariance."""
    mu1, mu2 = ssim_blur(x1), ssim_blur(x2)
    s11 = ssim_blur(x1 * x1) - mu1 * mu1
    s22 = ssim_blur(x2 * x2) - mu2 * mu2
    s12 = ssim_blur(x1 * x2) - mu1 * mu2
    return ((2 * mu1 * mu2 + SSIM_C1) * (2 * s12 + SSIM_C2)) / \
        ((mu1 * mu1 + mu2 * mu2 + SSIM_C1) * (s11 + s22 + SSIM_C2))


def masked_ssim(rgb: np.ndarray, target: np.ndarray, mask: np.ndarray, weight: float = 0.0):
    """SSIM of one view with both images masked first (Eq. 2 masks the inputs of L_c; Sec. 5
    masks the inputs of the evaluation SSIM).  rgb, target [h, w, 3], mask [h, w] in {0, 1}.
    Returns (mean over all 3 h w values, mean over the values of mask pixels, gradient of
    weight (1 - mean over all) with respect to rgb)."""
    m = torch.tensor(np.asarray(mask, np.float64))[..., None]
    r = torch.tensor(np.asarray(rgb, np.float64), requires_grad=True)
    t = torch.tensor(np.asarray(target, np.float64))
    s = ssim_map(t * m, r * m)
    s_all = s.mean()
    n_m = float(m.sum()) * 3.0
    s_masked = float((s * m).sum().detach()) / n_m if n_m > 0 else float("nan")
    (weight * (1.0 - s_all)).backward()
    return float(s_all.detach()), s_masked, r.grad.numpy()


def masked_psnr(rgb: np.ndarray, target: np.ndarray, mask: np.ndarray, max_i: float = 1.0) -> float:
    """PSNR = 20 log10(MAX_I / sqrt(MSE)) with the masked MSE of Sec. 5: the squared masked
    differences summed over the image and divided by the number of mask values (3 per pixel)."""
    m = np.asarray(mask, np.float64)[..., None]
    d = (np.asarray(target, np.float64) - np.asarray(rgb, np.float64)) * m
    n = 3.0 * float(np.asarray(mask, np.float64).sum())
    if n == 0:
        return float("nan")
    mse = float((d * d).sum()) / n
    return float("inf") if mse == 0 else 20.0 * np.log10(max_i / np.sqrt(mse))


# ----------------------------------------------------------------------------- 2DGS regularisers of Eq. 3
# Eq. 3 adds the depth distortion L_d and the normal consistency L_n of 2DGS.  Both are
# functions of the composited planes of one view: A (alpha), D = sum w z (depth),
# Q = sum w z^2 (depth2) and N_r = sum w n (normal).

def depth_distortion(alpha, depth, depth2, weight: float = 1.0):
    """Per pixel sum_{i,j} w_i w_j (z_i - z_j)^2 over the blended entries, which equals
    2 (A Q - D^2); the loss is its mean over the view's pixels.  Returns (loss, gradients of
    weight * loss with respect to alpha, depth, depth2), numpy FP64 [h w]."""
    a = torch.tensor(np.asarray(alpha, np.float64), requires_grad=True)
    d = torch.tensor(np.asarray(depth, np.float64), requires_grad=True)
    q = torch.tensor(np.asarray(depth2, np.float64), requires_grad=True)
    loss = (2.0 * (a * q - d * d)).mean()
    (weight * loss).backward()
    return float(loss.detach()), a.grad.numpy(), d.grad.numpy(), q.grad.numpy()


def normal_consistency(alpha, depth, normal, cam: dict, weight: float = 1.0, a_min: float = 0.5):
    """Per pixel sum_i w_i (1 - n_i . N) = A - N . N_r, with N the unit normal of the surface of
    expected depth D / A: the camera-frame points P = (D / A) ((x - cx) / fx, (y - cy) / fy, 1)
    at the pixel centres, N = normalize((P[x+1] - P[x-1]) x (P[y+1] - P[y-1])) turned towards the
    camera.  A pixel counts when it and its four neighbours lie inside the image and have
    A > a_min; the loss is the sum over those pixels divided by h w.  Returns (loss, gradients of
    weight * loss with respect to alpha [h w], depth [h w], normal [h w, 3])."""
    W, H = cam["width"], cam["height"]
    a = torch.tensor(np.asarray(alpha, np.float64).reshape(H, W), requires_grad=True)
    d = torch.tensor(np.asarray(depth, np.float64).reshape(H, W), requires_grad=True)
    nr = torch.tensor(np.asarray(normal, np.float64).reshape(H, W, 3), requires_grad=True)
    ok = (a.detach() > a_min)
    xs = (torch.arange(W, dtype=DT) + 0.5 - cam["cx"]) / cam["fx"]
    ys = (torch.arange(H, dtype=DT) + 0.5 - cam["cy"]) / cam["fy"]
    ray = torch.stack([xs[None, :].expand(H, W), ys[:, None].expand(H, W), torch.ones(H, W, dtype=DT)], -1)
    z = torch.where(ok, d / torch.where(ok, a, torch.ones_like(a)), torch.zeros_like(d))
    P = z[..., None] * ray
    dx = P[1:-1, 2:] - P[1:-1, :-2]
    dy = P[2:, 1:-1] - P[:-2, 1:-1]
    c = torch.linalg.cross(dx, dy)
    valid = (ok[1:-1, 1:-1] & ok[1:-1, 2:] & ok[1:-1, :-2] & ok[2:, 1:-1] & ok[:-2, 1:-1])
    norm = torch.where(valid, c.norm(dim=-1), torch.ones_like(c[..., 0]))
    N = c / norm[..., None]
    facing = ((N * P[1:-1, 1:-1]).sum(-1) > 0).detach()
    N = torch.where(facing[..., None], -N, N)
    term = a[1:-1, 1:-1] - (N * nr[1:-1, 1:-1]).sum(-1)
    loss = torch.where(valid, term, torch.zeros_like(term)).sum() / (H * W)
    (weight * loss).backward()
    return (float(loss.detach()), a.grad.numpy().reshape(-1), d.grad.numpy().reshape(-1),
            nr.grad.numpy().reshape(-1, 3))


# ----------------------------------------------------------------------------- 3DGS variant (Appendix B)
# Appendix B runs the same pruning record in 3DGS: 3D Gaussians splatted with the EWA
# projection of their covariance.  Same skip (rho > 9, alpha < 1/255), clamp, stop rule,
# depth order and contribution score as the 2DGS path; rho is the Mahalanobis distance
# under the projected covariance dilated by the 3DGS screen-space low-pass (0.3 px^2).
EWA_DILATION = 0.3


def project_ewa(g: dict, cam: dict) -> dict:
    """Per-Gaussian EWA projection: camera-frame mean t, 3D covariance R diag(s^2) R^T,
    image covariance J W Sigma W^T J^T + 0.3 I (J the Jacobian of the pinhole projection
    at t, W the world-to-camera rotation), its inverse (the conic), centre pixel, colour
    and centre depth.  Scales are [N,3]."""
    r_cw, t_cw, K = camera_tensors(cam)
    xyz, quat, scale = _t(g["xyz"]), _t(g["quat"]), _t(g["scale"])
    rot = quat_to_rotmat(quat / quat.norm(dim=-1, keepdim=True))
    sig3 = rot @ torch.diag_embed(scale * scale) @ rot.transpose(1, 2)
    t = xyz @ r_cw.T + t_cw
    tx, ty, tz = t[:, 0], t[:, 1], t[:, 2]
    fx, fy = cam["fx"], cam["fy"]
    zero = torch.zeros_like(tz)
    J = torch.stack([torch.stack([fx / tz, zero, -fx * tx / (tz * tz)], -1),
                     torch.stack([zero, fy / tz, -fy * ty / (tz * tz)], -1)], 1)     # [N,2,3]
    Tm = J @ r_cw
    cov2 = Tm @ sig3 @ Tm.transpose(1, 2) + EWA_DILATION * torch.eye(2, dtype=DT)
    conic = torch.linalg.inv(cov2)
    centre = torch.stack([fx * tx / tz + cam["cx"], fy * ty / tz + cam["cy"]], -1)
    campos = -(r_cw.T @ t_cw)
    d = xyz - campos
    d = d / d.norm(dim=-1, keepdim=True)
    rgb = ((sh_basis(d, g["sh_degree"])[:, :, None] * _t(g["sh"])).sum(1) + 0.5).clamp(min=0.0)
    return dict(conic=conic, cov2=cov2, centre=centre, z=tz, rgb=rgb, opacity=_t(g["opacity"]),
                culled=tz <= cam["near"])


def render_3d(g: dict, cam: dict, pixels: Optional[np.ndarray] = None, chunk: int = 256) -> dict:
    """Forward of the 3DGS variant at the given flat pixel indices (default all): per pixel,
    the non-culled Gaussians in ascending centre depth (ties by index), rho = d^T conic d
    with d = x - centre, alpha = min(0.99, o exp(-rho/2)), skipped if rho > 9 or
    alpha < 1/255, stopped at the first candidate with T (1 - alpha) < 1e-4 (not blended).
    Returns numpy rgb [P,3], alpha [P], depth [P] (sum w z), t_final [P], n_blended [P],
    fragile [P] and score [N] (max blending weight over these pixels)."""
    pr = project_ewa(g, cam)
    N = pr["z"].shape[0]
    alive = torch.nonzero(~pr["culled"]).flatten()
    order = alive[depth_order(pr["z"][alive])]
    pixels, xs_all, ys_all = pixel_centres(cam, pixels)
    P = len(pixels)
    res = dict(rgb=np.zeros((P, 3)), alpha=np.zeros(P), depth=np.zeros(P), t_final=np.ones(P),
               n_blended=np.zeros(P, np.int64), fragile=np.zeros(P, bool))
    score = torch.zeros(N, dtype=DT)
    C, ctr = pr["conic"][order], pr["centre"][order]
    o, z, rgb = pr["opacity"][order], pr["z"][order], pr["rgb"][order]
    for s in range(0, P, chunk):
        e = min(P, s + chunk)
        dx = xs_all[s:e, None] - ctr[None, :, 0]
        dy = ys_all[s:e, None] - ctr[None, :, 1]
        rho = C[None, :, 0, 0] * dx * dx + 2.0 * C[None, :, 0, 1] * dx * dy + C[None, :, 1, 1] * dy * dy
        fb = front_to_back(rho, o)
        w = fb["w"]
        res["rgb"][s:e] = (w @ rgb).numpy()
        res["alpha"][s:e] = w.sum(1).numpy()
        res["depth"][s:e] = (w @ z).numpy()
        res["t_final"][s:e] = fb["t_final"].numpy()
        res["n_blended"][s:e] = fb["n_blended"].numpy()
        if len(order):
            score[order] = torch.maximum(score[order], w.max(0).values)
        res["fragile"][s:e] = fb["at_edge"].any(1).numpy()
    res["score"] = score.numpy()
    return res


def contribution_score_3d(g: dict, cams: list) -> np.ndarray:
    """Max blending weight of every 3D Gaussian over all pixels of all views (Appendix B)."""
    s = np.zeros(len(np.asarray(g["opacity"])))
    for cam in cams:
        s = np.maximum(s, render_3d(g, cam)["score"])
    return s
