"""PyTorch binding of libocgs: argument marshalling only.

Every function here validates tensors, passes their device pointers and the
current CUDA stream to the C ABI of ``include/ocgs.h`` and returns torch
tensors.  All arithmetic of the method runs in the library's CUDA kernels;
nothing here computes a rasterizer result, and nothing falls back to the CPU.

Parameter layout (float32, CUDA, contiguous): xyz [N,3], quat [N,4] (w,x,y,z),
scale [N,2], opacity [N], sh [N,(deg+1)^2,3].  Cameras are dicts with a
4x4 world->camera ``viewmat`` (OpenCV axes), ``fx, fy, cx, cy``, ``width``,
``height`` and ``near``.  Images of several views are concatenated in view
order: rgb [P,3], alpha [P], depth [P], normal [P,3].
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib

PARAM_KEYS = ("xyz", "quat", "scale", "opacity", "sh")


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _check_param(name: str, t: torch.Tensor, shape_tail, device) -> None:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    if tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected [N,{','.join(map(str, shape_tail))}]")


def sh_degree_of(sh: torch.Tensor) -> int:
    k = sh.shape[1]
    deg = int(round(k ** 0.5)) - 1
    if (deg + 1) ** 2 != k or not 0 <= deg <= 3:
        raise ValueError(f"sh must be [N,(deg+1)^2,3] with deg 0..3, got {tuple(sh.shape)}")
    return deg


def gaussians_struct(g: dict, device) -> _lib.Gaussians:
    n = g["xyz"].shape[0]
    deg = sh_degree_of(g["sh"])
    for key, tail in (("xyz", (3,)), ("quat", (4,)), ("scale", (2,)), ("opacity", ()),
                      ("sh", ((deg + 1) ** 2, 3))):
        _check_param(key, g[key], tail, device)
        if g[key].shape[0] != n:
            raise ValueError(f"{key} has {g[key].shape[0]} rows, expected {n}")
    return _lib.Gaussians(_ptr(g["xyz"]), _ptr(g["quat"]), _ptr(g["scale"]), _ptr(g["opacity"]),
                          _ptr(g["sh"]), n, deg, 0)


def gaussians3d_struct(g: dict, device) -> _lib.Gaussians3d:
    """3D Gaussians (the 3DGS variant): scale [N,3]."""
    n = g["xyz"].shape[0]
    deg = sh_degree_of(g["sh"])
    for key, tail in (("xyz", (3,)), ("quat", (4,)), ("scale", (3,)), ("opacity", ()),
                      ("sh", ((deg + 1) ** 2, 3))):
        _check_param(key, g[key], tail, device)
        if g[key].shape[0] != n:
            raise ValueError(f"{key} has {g[key].shape[0]} rows, expected {n}")
    return _lib.Gaussians3d(_ptr(g["xyz"]), _ptr(g["quat"]), _ptr(g["scale"]), _ptr(g["opacity"]),
                            _ptr(g["sh"]), n, deg, 0)


def camera_array(cameras: Sequence[dict]):
    arr = (_lib.Camera * len(cameras))()
    for i, cam in enumerate(cameras):
        vm = np.asarray(cam["viewmat"], np.float64).reshape(16)
        c = arr[i]
        for k in range(16):
            c.viewmat[k] = float(vm[k])
        c.fx, c.fy, c.cx, c.cy = float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"])
        c.width, c.height = int(cam["width"]), int(cam["height"])
        c.near_plane = float(cam.get("near", 0.2))
    return arr


def n_pixels(cameras: Sequence[dict]) -> int:
    return int(sum(int(c["width"]) * int(c["height"]) for c in cameras))


def pixel_offsets(cameras: Sequence[dict]) -> list:
    off = [0]
    for c in cameras:
        off.append(off[-1] + int(c["width"]) * int(c["height"]))
    return off


class ForwardState:
    """Opaque forward state of one ``render`` call (owned by its Rasterizer)."""

    def __init__(self, rast: "Rasterizer", handle: C.c_void_p, n: int, deg: int, cameras):
        self._rast = rast
        self.handle = handle
        self.n = n
        self.sh_degree = deg
        self.cameras = list(cameras)

    def info(self) -> dict:
        """Pairs K, pixels P, tiles, views and E (pairs both passes evaluate). Synchronises."""
        inf = _lib.StateInfo()
        self._rast._call("ocgs_state_query", self._rast._ctx, self.handle, C.byref(inf))
        return {k: getattr(inf, k) for k, _ in _lib.StateInfo._fields_}

    def release(self) -> None:
        if self.handle:
            self._rast._call("ocgs_state_release", self._rast._ctx, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class ContributionGraph:
    """The pruning sweep captured as one CUDA graph (see ocgs_contribution_graph_create)."""

    def __init__(self, rast: "Rasterizer", handle: C.c_void_p, score: torch.Tensor, keep_alive):
        self._rast = rast
        self.handle = handle
        self.score = score
        self._keep = keep_alive  # parameter tensors the graph reads

    def launch(self) -> torch.Tensor:
        self._rast._bind_stream()
        self._rast._call("ocgs_graph_launch", self._rast._ctx, self.handle)
        return self.score

    def close(self) -> None:
        if self.handle:
            self._rast._call("ocgs_graph_destroy", self._rast._ctx, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# share of the depth order binned in the first pass of a persistent render
FRONT_FRACTION = 0.1


class Rasterizer:
    """One libocgs context on one CUDA device."""

    def __init__(self, device=None, tile=(16, 16), persistent: bool = False, pixels_per_thread: int = 2,
                 front_fraction: float = FRONT_FRACTION, batch: int = 32):
        self.lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device) \
            if not isinstance(device, torch.device) else device
        ctx = C.c_void_p()
        st = self.lib.ocgs_create(C.byref(ctx), self.device.index, None)
        if st != _lib.OK:
            raise _lib.OcgsError(st, "ocgs_create failed (is a CUDA device present?)")
        self._ctx = ctx
        self.set_options(tile=tile, persistent=persistent, pixels_per_thread=pixels_per_thread,
                         front_fraction=front_fraction, batch=batch)

    # -- plumbing
    def _call(self, name: str, *args) -> int:
        st = getattr(self.lib, name)(*args)
        if st != _lib.OK:
            raise _lib.OcgsError(st, self.lib.ocgs_last_error(self._ctx).decode())
        return st

    def _bind_stream(self) -> None:
        s = torch.cuda.current_stream(self.device).cuda_stream
        self.lib.ocgs_set_stream(self._ctx, C.c_void_p(s))

    def close(self) -> None:
        if getattr(self, "_ctx", None):
            self.lib.ocgs_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, tile=(16, 16), persistent: bool = False, pixels_per_thread: int = 2,
                    front_fraction: float = FRONT_FRACTION, batch: int = 32) -> None:
        """Launch options (see ocgs_options); none changes a result.  ``front_fraction``: share
        of the depth order binned in the first of two passes (persistent renders; 0 = one pass);
        ``batch``: Gaussians a warp stages in shared memory at a time (16, 32 or 64)."""
        o = _lib.Options(int(tile[0]), int(tile[1]), int(bool(persistent)), int(pixels_per_thread),
                         float(front_fraction), int(batch))
        self._call("ocgs_set_options", self._ctx, C.byref(o))
        self.tile = (int(tile[0]), int(tile[1]))
        self.persistent = bool(persistent)
        self.pixels_per_thread = int(pixels_per_thread)
        self.front_fraction = float(front_fraction)
        self.batch = int(batch)

    def set_coverage(self, rect: bool) -> None:
        """Tile coverage of the binning (see ocgs_set_coverage): False, the default, keeps the
        pairs whose support reaches the tile; True bins every tile of each record's screen
        rectangle with no support test, which must render the same bits, only slower."""
        self._call("ocgs_set_coverage", self._ctx, int(bool(rect)))

    def options(self) -> dict:
        """The context's launch options, as ``set_options`` takes them."""
        return dict(tile=self.tile, persistent=self.persistent, pixels_per_thread=self.pixels_per_thread,
                    front_fraction=self.front_fraction, batch=self.batch)

    def autotune(self, gaussians: dict, cameras: Sequence[dict], cache_path: Optional[str] = None) -> dict:
        """Time the launch-option candidates on this workload's training render and backward and keep
        the fastest (see ocgs_autotune); returns the chosen options and their time."""
        self._bind_stream()
        gs = gaussians_struct(gaussians, self.device)
        res = _lib.TuneResult()
        self._call("ocgs_autotune", self._ctx, C.byref(gs), camera_array(cameras), len(cameras),
                   None if cache_path is None else str(cache_path).encode(), C.byref(res))
        b = res.best
        self.tile = (b.tile_w, b.tile_h)
        self.persistent = bool(b.persistent)
        self.pixels_per_thread = b.pixels_per_thread
        self.front_fraction = float(b.front_fraction)
        self.batch = int(b.batch)
        return {"tile": self.tile, "pixels_per_thread": b.pixels_per_thread, "persistent": bool(b.persistent),
                "front_fraction": self.front_fraction, "batch": self.batch,
                "ms": res.best_ms, "n_tried": res.n_tried, "from_cache": bool(res.from_cache)}

    def stats(self) -> dict:
        s = _lib.Stats()
        self._call("ocgs_get_stats", self._ctx, C.byref(s))
        return {k: getattr(s, k) for k, _ in _lib.Stats._fields_}

    def sync(self) -> None:
        self._call("ocgs_sync", self._ctx)

    def profile(self, enable: bool) -> None:
        """Start (reset) or stop the library's per-stage CUDA-event timers."""
        self._call("ocgs_profile_enable", self._ctx, int(bool(enable)))

    def profile_read(self) -> dict:
        """Summed device milliseconds and instance counts per stage (synchronises)."""
        p = _lib.Profile()
        self._call("ocgs_profile_read", self._ctx, C.byref(p))
        return {name: (p.ms[i], p.launches[i]) for i, name in enumerate(_lib.STAGES)}

    def kernel_launches(self) -> int:
        """Kernels launched by libocgs in this process so far."""
        return int(self.lib.ocgs_kernel_launches())

    # -- the method
    def render(self, gaussians: dict, cameras: Sequence[dict], score: Optional[torch.Tensor] = None,
               keep_state: bool = True, out: Optional[dict] = None, depth2: bool = False):
        """Forward rasterization of all ``cameras`` in one batched pass.

        Returns ({rgb, alpha, depth, normal[, depth2]}, ForwardState or None).
        ``depth2`` adds the plane Q = sum w z^2 (for the depth distortion).  When
        ``score`` [N] is given it is max-accumulated with each Gaussian's
        largest blending weight."""
        self._bind_stream()
        gs = gaussians_struct(gaussians, self.device)
        cams = camera_array(cameras)
        P = n_pixels(cameras)
        f32 = dict(dtype=torch.float32, device=self.device)
        if out is None:
            out = dict(rgb=torch.empty(P, 3, **f32), alpha=torch.empty(P, **f32),
                       depth=torch.empty(P, **f32), normal=torch.empty(P, 3, **f32))
        if depth2 and out.get("depth2") is None:
            out["depth2"] = torch.empty(P, **f32)
        img = _lib.Image(_ptr(out["rgb"]), _ptr(out["alpha"]), _ptr(out["depth"]), _ptr(out["normal"]),
                         _ptr(out.get("depth2")))
        if score is not None:
            _check_param("score", score, (), self.device)
        handle = C.c_void_p()
        st = self.lib.ocgs_render(self._ctx, C.byref(gs), cams, len(cameras), C.byref(img), _ptr(score),
                                  C.byref(handle) if keep_state else None)
        if st != _lib.OK:
            msg = self.lib.ocgs_last_error(self._ctx).decode()
            if handle:
                self.lib.ocgs_state_release(self._ctx, handle)
            raise _lib.OcgsError(st, msg)
        state = ForwardState(self, handle, gs.n, gs.sh_degree, cameras) if keep_state else None
        return out, state

    def render_backward(self, state: ForwardState, gaussians: dict, d_out: dict,
                        grads: Optional[dict] = None) -> dict:
        """Gradients of sum <d_out, out> w.r.t. the parameters (added into ``grads``)."""
        self._bind_stream()
        gs = gaussians_struct(gaussians, self.device)
        if grads is None:
            grads = {k: torch.zeros_like(gaussians[k]) for k in PARAM_KEYS}
        img = _lib.Image(_ptr(d_out.get("rgb")), _ptr(d_out.get("alpha")), _ptr(d_out.get("depth")),
                         _ptr(d_out.get("normal")), _ptr(d_out.get("depth2")))
        for k, v in d_out.items():
            if v is not None and (not v.is_cuda or v.dtype != torch.float32 or not v.is_contiguous()):
                raise ValueError(f"d_out[{k}] must be a contiguous float32 CUDA tensor")
        go = _lib.GaussiansOut(*[_ptr(grads[k]) for k in PARAM_KEYS])
        self._call("ocgs_render_backward", self._ctx, state.handle, C.byref(gs), C.byref(img), C.byref(go))
        return grads

    def background_loss(self, alpha: torch.Tensor, mask: torch.Tensor, cameras: Sequence[dict],
                        gamma: float = 0.5, d_alpha: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Per-view L_b (Eq. 1) as a float64 tensor; adds gamma dL_b/dA into ``d_alpha``."""
        self._bind_stream()
        if mask.dtype != torch.uint8 or not mask.is_cuda or not mask.is_contiguous():
            raise ValueError("mask must be a contiguous uint8 CUDA tensor")
        if not alpha.is_cuda or alpha.dtype != torch.float32 or not alpha.is_contiguous():
            raise ValueError("alpha must be a contiguous float32 CUDA tensor")
        P = n_pixels(cameras)
        if alpha.numel() != P or mask.numel() != P:
            raise ValueError(f"alpha and mask must hold {P} pixels")
        loss = torch.empty(len(cameras), dtype=torch.float64, device=self.device)
        self._call("ocgs_background_loss", self._ctx, _ptr(alpha), _ptr(mask), camera_array(cameras),
                   len(cameras), float(gamma), _ptr(loss), _ptr(d_alpha))
        return loss

    def masked_l1(self, rgb: torch.Tensor, target: torch.Tensor, mask: torch.Tensor, cameras: Sequence[dict],
                  weight: float = 1.0, d_rgb: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Per-view masked L1 of Eq. 2 (float64 tensor); adds weight * dL/dR into ``d_rgb``."""
        self._bind_stream()
        P = n_pixels(cameras)
        for name, t in (("rgb", rgb), ("target", target)):
            if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != 3 * P:
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of {P}x3 values")
        if mask.dtype != torch.uint8 or not mask.is_cuda or not mask.is_contiguous() or mask.numel() != P:
            raise ValueError(f"mask must be a contiguous uint8 CUDA tensor of {P} values")
        loss = torch.empty(len(cameras), dtype=torch.float64, device=self.device)
        self._call("ocgs_masked_l1", self._ctx, _ptr(rgb), _ptr(target), _ptr(mask), camera_array(cameras),
                   len(cameras), float(weight), _ptr(loss), _ptr(d_rgb))
        return loss

    def _check_images(self, rgb, target, mask, cameras, d_rgb=None):
        P = n_pixels(cameras)
        for name, t in (("rgb", rgb), ("target", target)) + ((("d_rgb", d_rgb),) if d_rgb is not None else ()):
            if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != 3 * P:
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of {P}x3 values")
        if mask.dtype != torch.uint8 or not mask.is_cuda or not mask.is_contiguous() or mask.numel() != P:
            raise ValueError(f"mask must be a contiguous uint8 CUDA tensor of {P} values")

    def ssim(self, rgb: torch.Tensor, target: torch.Tensor, mask: torch.Tensor, cameras: Sequence[dict],
             weight: float = 0.0, d_rgb: Optional[torch.Tensor] = None):
        """Per-view SSIM of the masked images: (mean over all values, mean over mask values), both
        float64 tensors; adds weight * d(1 - SSIM)/dR into ``d_rgb`` (the D-SSIM term of Eq. 2)."""
        self._bind_stream()
        self._check_images(rgb, target, mask, cameras, d_rgb)
        s_all = torch.empty(len(cameras), dtype=torch.float64, device=self.device)
        s_m = torch.empty(len(cameras), dtype=torch.float64, device=self.device)
        self._call("ocgs_ssim", self._ctx, _ptr(rgb), _ptr(target), _ptr(mask), camera_array(cameras), len(cameras),
                   float(weight), _ptr(s_all), _ptr(s_m), _ptr(d_rgb))
        return s_all, s_m

    def masked_psnr(self, rgb: torch.Tensor, target: torch.Tensor, mask: torch.Tensor, cameras: Sequence[dict],
                    max_i: float = 1.0) -> torch.Tensor:
        """Per-view masked PSNR of Sec. 5 (float64 tensor)."""
        self._bind_stream()
        self._check_images(rgb, target, mask, cameras)
        out = torch.empty(len(cameras), dtype=torch.float64, device=self.device)
        self._call("ocgs_masked_psnr", self._ctx, _ptr(rgb), _ptr(target), _ptr(mask), camera_array(cameras),
                   len(cameras), float(max_i), _ptr(out))
        return out

    def _check_planes(self, cameras, **planes):
        P = n_pixels(cameras)
        for name, (t, ch) in planes.items():
            if t is None:
                continue
            if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != ch * P:
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of {P}x{ch} values")

    def depth_distortion(self, alpha, depth, depth2, cameras: Sequence[dict], weight: float = 1.0,
                         grads: Optional[dict] = None) -> torch.Tensor:
        """Per-view 2DGS depth distortion (Eq. 3) from the alpha, depth and depth2 planes; with
        ``grads`` = {alpha, depth, depth2} adds weight * d loss / d plane into them."""
        self._bind_stream()
        g = grads or {}
        self._check_planes(cameras, alpha=(alpha, 1), depth=(depth, 1), depth2=(depth2, 1),
                           d_alpha=(g.get("alpha"), 1), d_depth=(g.get("depth"), 1), d_depth2=(g.get("depth2"), 1))
        loss = torch.empty(len(cameras), dtype=torch.float64, device=self.device)
        self._call("ocgs_depth_distortion", self._ctx, _ptr(alpha), _ptr(depth), _ptr(depth2), camera_array(cameras),
                   len(cameras), float(weight), _ptr(loss), _ptr(g.get("alpha")), _ptr(g.get("depth")),
                   _ptr(g.get("depth2")))
        return loss

    def normal_consistency(self, alpha, depth, normal, cameras: Sequence[dict], weight: float = 1.0,
                           a_min: float = 0.5, grads: Optional[dict] = None) -> torch.Tensor:
        """Per-view 2DGS normal consistency (Eq. 3) from the alpha, depth and normal planes; with
        ``grads`` = {alpha, depth, normal} adds weight * d loss / d plane into them."""
        self._bind_stream()
        g = grads or {}
        self._check_planes(cameras, alpha=(alpha, 1), depth=(depth, 1), normal=(normal, 3),
                           d_alpha=(g.get("alpha"), 1), d_depth=(g.get("depth"), 1), d_normal=(g.get("normal"), 3))
        loss = torch.empty(len(cameras), dtype=torch.float64, device=self.device)
        self._call("ocgs_normal_consistency", self._ctx, _ptr(alpha), _ptr(depth), _ptr(normal),
                   camera_array(cameras), len(cameras), float(weight), float(a_min), _ptr(loss),
                   _ptr(g.get("alpha")), _ptr(g.get("depth")), _ptr(g.get("normal")))
        return loss

    def render_3d(self, gaussians: dict, cameras: Sequence[dict], score: Optional[torch.Tensor] = None) -> dict:
        """Forward of the 3DGS variant (Appendix B): {rgb, alpha, depth} of all ``cameras``;
        ``score`` [N] is max-accumulated as in ``render``."""
        self._bind_stream()
        gs = gaussians3d_struct(gaussians, self.device)
        P = n_pixels(cameras)
        f32 = dict(dtype=torch.float32, device=self.device)
        out = dict(rgb=torch.empty(P, 3, **f32), alpha=torch.empty(P, **f32), depth=torch.empty(P, **f32),
                   normal=torch.empty(P, 3, **f32))
        if score is not None:
            _check_param("score", score, (), self.device)
        img = _lib.Image(_ptr(out["rgb"]), _ptr(out["alpha"]), _ptr(out["depth"]), _ptr(out["normal"]), None)
        self._call("ocgs_render_3d", self._ctx, C.byref(gs), camera_array(cameras), len(cameras), C.byref(img),
                   _ptr(score))
        del out["normal"]
        return out

    def accumulate_contribution_3d(self, gaussians: dict, cameras: Sequence[dict],
                                   score: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Pruning record of the 3DGS variant: max blending weight of every 3D Gaussian over all views."""
        self._bind_stream()
        gs = gaussians3d_struct(gaussians, self.device)
        if score is None:
            score = torch.zeros(gs.n, dtype=torch.float32, device=self.device)
        _check_param("score", score, (), self.device)
        self._call("ocgs_accumulate_contribution_3d", self._ctx, C.byref(gs), camera_array(cameras), len(cameras),
                   _ptr(score))
        return score

    def accumulate_contribution(self, gaussians: dict, cameras: Sequence[dict],
                                score: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Pruning sweep (Sec. 4.3): max blending weight of every Gaussian over all views."""
        self._bind_stream()
        gs = gaussians_struct(gaussians, self.device)
        if score is None:
            score = torch.zeros(gs.n, dtype=torch.float32, device=self.device)
        _check_param("score", score, (), self.device)
        self._call("ocgs_accumulate_contribution", self._ctx, C.byref(gs), camera_array(cameras),
                   len(cameras), _ptr(score))
        return score

    def contribution_graph(self, gaussians: dict, cameras: Sequence[dict], score: Optional[torch.Tensor] = None,
                           headroom: float = 1.25) -> ContributionGraph:
        """Capture the pruning sweep over ``cameras`` once; ``.launch()`` replays it."""
        self._bind_stream()
        gs = gaussians_struct(gaussians, self.device)
        if score is None:
            score = torch.zeros(gs.n, dtype=torch.float32, device=self.device)
        _check_param("score", score, (), self.device)
        handle = C.c_void_p()
        self._call("ocgs_contribution_graph_create", self._ctx, C.byref(gs), camera_array(cameras), len(cameras),
                   _ptr(score), float(headroom), C.byref(handle))
        return ContributionGraph(self, handle, score, [gaussians[k] for k in PARAM_KEYS])

    def prune(self, gaussians: dict, score: torch.Tensor, threshold: float, borderline_cap: int = 4096):
        """Keep {score > threshold}; returns (kept parameters, borderline indices)."""
        self._bind_stream()
        gs = gaussians_struct(gaussians, self.device)
        _check_param("score", score, (), self.device)
        out = {k: torch.empty_like(gaussians[k]) for k in PARAM_KEYS}
        go = _lib.GaussiansOut(*[_ptr(out[k]) for k in PARAM_KEYS])
        border = torch.empty(max(1, borderline_cap), dtype=torch.int64, device=self.device)
        n_kept = C.c_int64()
        n_border = C.c_int64()
        self._call("ocgs_prune", self._ctx, _ptr(score), float(threshold), C.byref(gs), C.byref(go),
                   C.byref(n_kept), _ptr(border), int(borderline_cap), C.byref(n_border))
        kept = {k: v[: n_kept.value] for k, v in out.items()}
        return kept, border[: min(n_border.value, borderline_cap)], n_border.value


    def adam_step(self, params: dict, grads: dict, m: dict, v: dict, lr, step: int,
                  beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15):
        """One fused Adam update (in place) of ``params`` and the moments ``m``, ``v``.

        ``lr`` is one learning rate or a dict with one per parameter array."""
        self._bind_stream()
        gs = gaussians_struct(grads, self.device)
        for name, d in (("params", params), ("m", m), ("v", v)):
            for k in PARAM_KEYS:
                if d[k].shape != grads[k].shape or d[k].dtype != torch.float32 or not d[k].is_contiguous() \
                        or d[k].device != self.device:
                    raise ValueError(f"{name}[{k}] must be a contiguous float32 {tuple(grads[k].shape)} on {self.device}")
        outs = [_lib.GaussiansOut(*[_ptr(d[k]) for k in PARAM_KEYS]) for d in (params, m, v)]
        rates = [float(lr[k]) for k in PARAM_KEYS] if isinstance(lr, dict) else [float(lr)] * 5
        cfg = _lib.AdamConfig((C.c_double * 5)(*rates), float(beta1), float(beta2), float(eps), int(step))
        self._call("ocgs_adam_step", self._ctx, C.byref(gs), C.byref(outs[0]), C.byref(outs[1]),
                   C.byref(outs[2]), C.byref(cfg))


class RenderFunction(torch.autograd.Function):
    """Differentiable render of a list of views through libocgs: outputs (rgb, alpha, depth,
    normal) of ``Rasterizer.render``, gradients from ``Rasterizer.render_backward``.

    * Cotangents of unused outputs reach the backward as None (they are not materialised as
      zeros), so a loss on colour and opacity alone runs the backward without the depth and
      normal terms.
    * The parameters are kept with ``save_for_backward``: changing one in place between the
      forward and the backward raises torch's version-counter error instead of differentiating
      at another point than the one rendered.
    * The first backward releases the forward state; a second backward through the same render
      (``retain_graph=True``) raises RuntimeError."""

    @staticmethod
    def forward(ctx, rast: Rasterizer, cameras, xyz, quat, scale, opacity, sh):
        g = dict(xyz=xyz.detach(), quat=quat.detach(), scale=scale.detach(), opacity=opacity.detach(),
                 sh=sh.detach())
        out, state = rast.render(g, cameras)
        ctx.rast = rast
        ctx.state = state
        ctx.save_for_backward(xyz, quat, scale, opacity, sh)
        ctx.set_materialize_grads(False)
        return out["rgb"], out["alpha"], out["depth"], out["normal"]

    @staticmethod
    def backward(ctx, g_rgb, g_alpha, g_depth, g_normal):
        if ctx.state is None or not ctx.state.handle:
            raise RuntimeError("RenderFunction: the forward state of this render was released by an earlier "
                               "backward; render again to differentiate again")
        params = ctx.saved_tensors  # raises if a parameter was modified in place after the forward
        g = {k: p.detach() for k, p in zip(PARAM_KEYS, params)}
        d_out = {k: v.contiguous() for k, v in
                 (("rgb", g_rgb), ("alpha", g_alpha), ("depth", g_depth), ("normal", g_normal)) if v is not None}
        state, ctx.state = ctx.state, None
        try:
            if not d_out:
                return (None,) * (2 + len(PARAM_KEYS))
            grads = ctx.rast.render_backward(state, g, d_out)
        finally:
            state.release()
        return (None, None) + tuple(grads[k] for k in PARAM_KEYS)


def render(rast: Rasterizer, gaussians: dict, cameras: Sequence[dict]):
    """Differentiable (rgb, alpha, depth, normal) of ``cameras``."""
    return RenderFunction.apply(rast, list(cameras), *[gaussians[k] for k in PARAM_KEYS])
