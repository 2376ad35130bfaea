"""Shared helpers for the parity tests (comparison rule and device plumbing)."""
from __future__ import annotations

import numpy as np

# Per-point acceptance rule for FP64 results against the oracle:
#   |gpu - ref| <= RTOL * |ref| + ATOL
RTOL = 1e-12
ATOL = 1e-14


def parity_report(gpu: np.ndarray, ref: np.ndarray, rtol: float = RTOL, atol: float = ATOL) -> dict:
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    err = np.abs(gpu - ref)
    allowed = rtol * np.abs(ref) + atol
    bad = ~(err <= allowed)            # NaN counts as bad
    worst = int(np.argmax(np.where(np.isfinite(err), err / allowed, np.inf)))
    return {
        "n": int(gpu.size),
        "bad": int(bad.sum()),
        "max_abs": float(np.nanmax(err)) if err.size else 0.0,
        "max_ratio": float(np.nanmax(err / allowed)) if err.size else 0.0,
        "worst_index": np.unravel_index(worst, gpu.shape) if gpu.size else None,
    }


def assert_parity(gpu, ref, rtol: float = RTOL, atol: float = ATOL, what: str = "") -> dict:
    rep = parity_report(gpu, ref, rtol, atol)
    assert rep["bad"] == 0, f"{what}: {rep['bad']} of {rep['n']} points outside tolerance; {rep}"
    return rep


def to_dev(arr: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr)).to("cuda")


def padded_dev(arr: np.ndarray, pitch: int, fill: float = float("nan")):
    """Device copy whose last axis is padded to `pitch` (returns the strided view)."""
    import torch
    shape = arr.shape[:-1] + (pitch,)
    buf = torch.full(shape, fill, dtype=torch.float64, device="cuda")
    buf[..., : arr.shape[-1]] = torch.from_numpy(np.ascontiguousarray(arr)).to("cuda")
    return buf[..., : arr.shape[-1]]
