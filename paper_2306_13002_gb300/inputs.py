"""Seeded synthetic inputs shared by the tests, the benchmark and the CPU oracle runs.

This module holds no arithmetic of the stencil method itself: it only draws numbers.
Every value is a pure function of (seed, counter), so any slab of a large field can be
regenerated independently and both sides of a comparison see bit-identical inputs.

Generator: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used in counter mode: output number i (i = 0, 1, ...) of stream
`seed` is mix(seed + (i + 1) * 0x9E3779B97F4A7C15 mod 2^64) with the published mixing
constants. A uniform double in [0, 1) is the top 53 bits times 2^-53, scaled to [lo, hi)
as lo + (hi - lo) * u.

Field recipes (the workloads of the compressible-flow RHS and the 25-point star stencil):
  * RHS conserved variables U[5][nz+2h][ny+2h][nx+2h], components c = 0..4 =
    (rho, m_x, m_y, m_z, E); rho and E uniform in [0.5, 1.5), momenta uniform in
    [-0.5, 0.5). The counter is the flat C-order index over the whole (c, k, j, i) array.
  * Stencil u and a, each [nz+2h][ny+2h][nx+2h], uniform in [0, 1). u uses counters
    0 .. V-1 and a uses V .. 2V-1 (V = extended volume), from the same seed.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
MIX1 = np.uint64(0xBF58476D1CE4E5B9)
MIX2 = np.uint64(0x94D049BB133111EB)
TWO_M53 = float(2.0 ** -53)

SEED_RHS_SMALL = 13002      # 32^3 interior, halo 2
SEED_RHS_LARGE = 13003      # 128^3 / 256^3
SEED_STENCIL = 13004        # 384^3, halo 4
SEED_BATCH = 13005          # 64 uneven grids
SEED_VARIANTS = 13006       # rewriter variant sampling
SEED_HUGE = 13007           # 512^3 RHS / 768^3 stencil

_CHUNK = 1 << 23


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Counter-mode SplitMix64 outputs (uint64) for the given counters."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (counters.astype(np.uint64) + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * MIX1
        z = (z ^ (z >> np.uint64(27))) * MIX2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, start: int, count: int, lo: float, hi: float, out: np.ndarray | None = None) -> np.ndarray:
    """Uniform doubles in [lo, hi) for counters start .. start+count-1 (chunked, bounded memory;
    large requests are split across threads, which changes no value)."""
    if out is None:
        out = np.empty(count, dtype=np.float64)
    scale = float(hi) - float(lo)

    def chunk(s):
        n = min(_CHUNK, count - s)
        z = splitmix64(seed, np.arange(start + s, start + s + n, dtype=np.uint64))
        u = (z >> np.uint64(11)).astype(np.float64) * TWO_M53
        out[s:s + n] = lo + scale * u

    starts = range(0, count, _CHUNK)
    if count > 4 * _CHUNK:
        import concurrent.futures as cf
        import os
        with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(chunk, starts))
    else:
        for s in starts:
            chunk(s)
    return out


RHS_RANGES = ((0.5, 1.5), (-0.5, 0.5), (-0.5, 0.5), (-0.5, 0.5), (0.5, 1.5))


def rhs_field(nx: int, ny: int | None = None, nz: int | None = None, halo: int = 2,
              seed: int = SEED_RHS_SMALL) -> np.ndarray:
    """Conserved variables U, shape (5, nz+2h, ny+2h, nx+2h), C order, float64."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    X, Y, Z = nx + 2 * halo, ny + 2 * halo, nz + 2 * halo
    vol = X * Y * Z
    U = np.empty((5, Z, Y, X), dtype=np.float64)
    flat = U.reshape(5, vol)
    for c, (lo, hi) in enumerate(RHS_RANGES):
        uniform(seed, c * vol, vol, lo, hi, out=flat[c])
    return U


def stencil_fields(nx: int, ny: int | None = None, nz: int | None = None, halo: int = 4,
                   seed: int = SEED_STENCIL) -> tuple[np.ndarray, np.ndarray]:
    """(u, a), each shape (nz+2h, ny+2h, nx+2h), uniform in [0, 1)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    shape = (nz + 2 * halo, ny + 2 * halo, nx + 2 * halo)
    vol = shape[0] * shape[1] * shape[2]
    u = uniform(seed, 0, vol, 0.0, 1.0).reshape(shape)
    a = uniform(seed, vol, vol, 0.0, 1.0).reshape(shape)
    return u, a


SEED_BLOCK = 13008          # block-assembly body


def block_fields(nx: int, ny: int | None = None, nz: int | None = None, halo: int = 1,
                 seed: int = SEED_BLOCK) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(A, B, G) for the block-assembly body: A, B (25, Z, Y, X) uniform in [-1, 1), G (Z, Y, X)
    uniform in [0.5, 1.5); counters A: 0.., B: 25V.., G: 50V.. (V = extended volume)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    shape = (nz + 2 * halo, ny + 2 * halo, nx + 2 * halo)
    vol = shape[0] * shape[1] * shape[2]
    A = uniform(seed, 0, 25 * vol, -1.0, 1.0).reshape((25,) + shape)
    B = uniform(seed, 25 * vol, 25 * vol, -1.0, 1.0).reshape((25,) + shape)
    G = uniform(seed, 50 * vol, vol, 0.5, 1.5).reshape(shape)
    return A, B, G


def batch_sides(n_grids: int, seed: int = SEED_BATCH, lo: int = 16, hi: int = 160) -> np.ndarray:
    """Grid sides (n_grids, 3) as (nx, ny, nz), each round(exp(U(ln lo, ln hi))) clamped to [lo, hi].

    Rounding is numpy's round-half-even.
    """
    u = uniform(seed, 0, 3 * n_grids, np.log(lo), np.log(hi))
    s = np.clip(np.rint(np.exp(u)), lo, hi).astype(np.int64)
    return s.reshape(n_grids, 3)


def pad_rows(arr: np.ndarray, pitch: int) -> np.ndarray:
    """Copy an array into one whose last axis is padded to `pitch` elements (NaN padding).

    Returns a view of the padded buffer with the original shape; `.base` holds the buffer.
    """
    X = arr.shape[-1]
    if pitch < X:
        raise ValueError("pitch smaller than row length")
    buf = np.full(arr.shape[:-1] + (pitch,), np.nan, dtype=arr.dtype)
    buf[..., :X] = arr
    return buf[..., :X]
