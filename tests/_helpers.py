"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch

KEYS = ("xyz", "quat", "scale", "opacity", "sh")
OUT_KEYS = ("rgb", "alpha", "depth", "normal")
FWD_TOL = 1e-4   # max abs error, FP32 device vs FP64 oracle
GRAD_TOL = 1e-3  # relative error (inf-norm per parameter group)


def to_device(g: dict, dev) -> dict:
    return {k: torch.tensor(np.asarray(g[k], np.float32), device=dev) for k in KEYS}


def gpu_at(out: dict, pixels: np.ndarray, offset: int = 0) -> dict:
    idx = torch.as_tensor(pixels + offset, device=out["alpha"].device)
    return {k: out[k][idx].double().cpu().numpy() for k in OUT_KEYS}


def forward_errors(gpu: dict, ref: dict, mask: np.ndarray) -> dict:
    return {k: float(np.abs(gpu[k] - ref[k])[mask].max()) if mask.any() else 0.0 for k in OUT_KEYS}


def grad_errors(gpu: dict, ref: dict) -> dict:
    errs = {}
    for k in KEYS:
        a = gpu[k].double().cpu().numpy()
        b = ref[k]
        errs[k] = float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))
    return errs


def masked(v: np.ndarray, ok: np.ndarray) -> np.ndarray:
    return np.where(ok.reshape((-1,) + (1,) * (v.ndim - 1)), v, 0.0)
