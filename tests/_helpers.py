"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch

KEYS = ("xyz", "quat", "scale", "opacity", "sh")
OUT_KEYS = ("rgb", "alpha", "depth", "normal")
FWD_TOL = 1e-4   # max abs error, FP32 device vs FP64 oracle
GRAD_TOL = 1e-3  # relative error per element (see grad_bar)
GRAD_FLOOR = 1e-2  # floor of the relative error, as a share of the group's largest entry
# allowance in units of a float32 evaluation's distance from FP64 (see grad_bar): one float32
# evaluation is a single sample of the rounding error of an ill-conditioned element, and the
# kernels' evaluation order differs from the oracle's (measured up to 3.8x on config 4)
GRAD_COND = 10.0


def to_device(g: dict, dev) -> dict:
    return {k: torch.tensor(np.asarray(g[k], np.float32), device=dev) for k in KEYS}


def gpu_at(out: dict, pixels: np.ndarray, offset: int = 0) -> dict:
    idx = torch.as_tensor(pixels + offset, device=out["alpha"].device)
    return {k: out[k][idx].double().cpu().numpy() for k in OUT_KEYS}


def forward_errors(gpu: dict, ref: dict, mask: np.ndarray) -> dict:
    return {k: float(np.abs(gpu[k] - ref[k])[mask].max()) if mask.any() else 0.0 for k in OUT_KEYS}


def oracle_adjoint(g_np: dict, cam: dict, d_out: dict, pixels=None) -> tuple:
    """The oracle's adjoint of sum <d_out, out> in FP64, and the same definition evaluated in
    float32 (the yardstick of each element's float32 conditioning)."""
    import oracle
    ref = oracle.render(g_np, cam, pixels=pixels, d_out=d_out)["grads"]
    with oracle.evaluated_in(torch.float32):
        ref32 = oracle.render(g_np, cam, pixels=pixels, d_out=d_out)["grads"]
    return ref, ref32


def _np(x) -> np.ndarray:
    return np.asarray(x.double().cpu().numpy() if isinstance(x, torch.Tensor) else x, np.float64).reshape(-1)


def grad_bar(ref: np.ndarray, ref32=None) -> np.ndarray:
    """Per-element bound on |g - g_ref|: GRAD_TOL relative to the element, with a floor at
    GRAD_FLOOR of the group's largest entry (elements the sum cancels to nearly zero are judged
    against the group's scale), or GRAD_COND times the distance of a float32 evaluation of the
    same definition from FP64 where that is larger (an element that float32 arithmetic itself
    cannot resolve to GRAD_TOL)."""
    b = _np(ref)
    bar = GRAD_TOL * np.maximum(np.abs(b), max(GRAD_FLOOR * np.abs(b).max(), 1e-30))
    if ref32 is not None:
        bar = np.maximum(bar, GRAD_COND * np.abs(_np(ref32) - b))
    return bar


def grad_errors(gpu: dict, ref: dict, ref32: dict = None) -> dict:
    """Per parameter group, max over elements of |g - g_ref| / grad_bar: 1 is at the bar."""
    errs = {}
    for k in KEYS:
        a, b = _np(gpu[k]), _np(ref[k])
        errs[k] = float((np.abs(a - b) / grad_bar(b, None if ref32 is None else ref32[k])).max()) if b.size else 0.0
    return errs


def worst_element(gpu: dict, ref: dict, key: str, ref32: dict = None) -> tuple:
    """(index, gpu value, reference value, float32 evaluation) of the element that sets
    grad_errors[key]."""
    a, b = _np(gpu[key]), _np(ref[key])
    r32 = None if ref32 is None else _np(ref32[key])
    i = int(np.argmax(np.abs(a - b) / grad_bar(b, r32)))
    return i, float(a[i]), float(b[i]), None if r32 is None else float(r32[i])


def add_grads(tot: dict, g: dict) -> dict:
    return {k: tot.get(k, 0.0) + np.asarray(g[k], np.float64) for k in KEYS}


def masked(v: np.ndarray, ok: np.ndarray) -> np.ndarray:
    return np.where(ok.reshape((-1,) + (1,) * (v.ndim - 1)), v, 0.0)
