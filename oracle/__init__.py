"""CPU oracle (TEST INFRASTRUCTURE ONLY).

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import
this package. The CUDA library never imports, links or calls it, and it imports nothing
from the CUDA library; the two share only the seeded input generator.

Contents:
  * `rhs`, `stencil`: the as-written FP64 loop nests of `acs_oracle.c` (built with gcc,
    -O2 -ffp-contract=off, OpenMP over k), through ctypes.
  * `exact`: exact-rational (fractions.Fraction) evaluation of the same definitions, the
    arbiter for any disagreement and the brute-force pin on tiny grids.
  * `exact.saturated_*`: the saturated form's regrouping written over Fractions, to check
    that it is an exact identity of the as-written form (Table I rules preserve value).
  * `variant`: compiles an edited copy of the oracle source, for tests that plant a
    mistake in the oracle and check that the pins catch it.

Parity pins: every function here is pinned by tests that do not re-type its formula
(closed forms of linear/quadratic/cubic/quartic fields, invariants, symmetries, a
library routine for the pure second difference, brute force in exact rationals).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "acs_oracle.c")
_LIB = os.path.join(_HERE, "_acs_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def _compile(src: str, out: str) -> None:
    tmp = out + f".tmp{os.getpid()}"
    r = subprocess.run(["gcc", *CFLAGS, "-fopenmp", src, "-o", tmp], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(["gcc", *CFLAGS, src, "-o", tmp], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available). Returns the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        _compile(_SRC, _LIB)
    return _LIB


def _strides(arr: np.ndarray) -> tuple[int, ...]:
    if arr.dtype != np.float64:
        raise TypeError("oracle works on float64 arrays")
    if arr.strides[-1] != 8:
        raise ValueError("x must be the unit-stride axis")
    return tuple(s // 8 for s in arr.strides)


class Oracle:
    """The oracle loop nests from one compiled copy of `acs_oracle.c`."""

    def __init__(self, libpath: str):
        lib = ctypes.CDLL(libpath)
        i64, dbl, i32, p = ctypes.c_longlong, ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        lib.oracle_rhs.argtypes = [p, p, i32, i32, i32, i32, i64, i64, i64, i64, i64, i64,
                                   dbl, dbl, dbl, dbl, dbl, i32, i32, i32]
        lib.oracle_rhs.restype = None
        lib.oracle_stencil.argtypes = [p, p, p, i32, i32, i32, i32, i64, i64, i64, i64, p, i32, i32, i32]
        lib.oracle_stencil.restype = None
        lib.oracle_block.argtypes = [p, p, p, p, i32, i32, i32, i32, i64, i64, i64, i64, i64, i64, p, i32, i32, i32]
        lib.oracle_block.restype = None
        lib.oracle_has_openmp.restype = i32
        self.lib = lib

    def has_openmp(self) -> bool:
        return bool(self.lib.oracle_has_openmp())

    def rhs(self, U: np.ndarray, gamma: float = 1.4, eps: float = 0.25, h=(1.0, 1.0, 1.0), halo: int = 2,
            k_range: tuple[int, int] | None = None, threads: int = 1, out: np.ndarray | None = None) -> np.ndarray:
        """As-written RHS. U: (5, nz+2h, ny+2h, nx+2h) float64 (any row/plane pitch).

        Returns R: (5, nz, ny, nx); planes outside `k_range` are left as NaN. With `out` (a
        C-contiguous float64 array of that shape, reused across calls) R is written there instead
        of a new NaN-filled array, and planes outside `k_range` keep what `out` held.
        """
        if U.ndim != 4 or U.shape[0] != 5:
            raise ValueError("U must be (5, Z, Y, X)")
        if halo < 2:
            raise ValueError("the RHS needs a halo of at least 2")
        nz, ny, nx = (s - 2 * halo for s in U.shape[1:])
        sc, sz, sy, _ = _strides(U)
        if out is None:
            R = np.full((5, nz, ny, nx), np.nan)
        else:
            if out.shape != (5, nz, ny, nx) or out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"]:
                raise ValueError("out must be a C-contiguous float64 array of shape (5, nz, ny, nx)")
            R = out
        k0, k1 = (0, nz) if k_range is None else k_range
        self.lib.oracle_rhs(U.ctypes.data, R.ctypes.data, nx, ny, nz, halo, sy, sz, sc,
                            nx, nx * ny, nx * ny * nz, float(gamma), float(eps),
                            float(h[0]), float(h[1]), float(h[2]), int(k0), int(k1), int(threads))
        return R

    def stencil(self, u: np.ndarray, a: np.ndarray, c: np.ndarray | None = None, halo: int = 4,
                k_range: tuple[int, int] | None = None, threads: int = 1) -> np.ndarray:
        """As-written 25-point star stencil. u, a: (nz+2h, ny+2h, nx+2h). Returns (nz, ny, nx)."""
        if u.shape != a.shape or u.ndim != 3:
            raise ValueError("u and a must be 3D arrays of the same shape")
        if halo < 4:
            raise ValueError("the star stencil needs a halo of at least 4")
        c = taylor_coeffs() if c is None else np.ascontiguousarray(c, dtype=np.float64).reshape(3, 4)
        nz, ny, nx = (s - 2 * halo for s in u.shape)
        uz, uy, _ = _strides(u)
        az, ay, _ = _strides(a)
        if (az, ay) != (uz, uy):
            raise ValueError("u and a must share strides")
        out = np.full((nz, ny, nx), np.nan)
        k0, k1 = (0, nz) if k_range is None else k_range
        self.lib.oracle_stencil(u.ctypes.data, a.ctypes.data, out.ctypes.data, nx, ny, nz, halo, uy, uz,
                                nx, nx * ny, c.ctypes.data, int(k0), int(k1), int(threads))
        return out


    def block(self, A: np.ndarray, B: np.ndarray, G: np.ndarray, prm=(0.01, 1.5, 2.0, 0.75, 0.5), halo: int = 1,
              k_range: tuple[int, int] | None = None, threads: int = 1) -> np.ndarray:
        """Block-assembly body. A, B: (25, Z, Y, X); G: (Z, Y, X) with the same strides per component.
        Returns out: (75, nz, ny, nx)."""
        if A.shape != B.shape or A.ndim != 4 or A.shape[0] != 25 or G.shape != A.shape[1:]:
            raise ValueError("A, B must be (25, Z, Y, X) and G (Z, Y, X)")
        if halo < 1:
            raise ValueError("the block body needs a halo of at least 1")
        sc, sz, sy, _ = _strides(A)
        if _strides(B) != (sc, sz, sy, 1) or _strides(G) != (sz, sy, 1):
            raise ValueError("A, B and G must share strides")
        nz, ny, nx = (s - 2 * halo for s in A.shape[1:])
        out = np.full((75, nz, ny, nx), np.nan)
        k0, k1 = (0, nz) if k_range is None else k_range
        pr = np.ascontiguousarray(prm, dtype=np.float64)
        self.lib.oracle_block(A.ctypes.data, B.ctypes.data, G.ctypes.data, out.ctypes.data, nx, ny, nz, halo, sy, sz,
                              sc, nx, nx * ny, nx * ny * nz, pr.ctypes.data, int(k0), int(k1), int(threads))
        return out


def default() -> Oracle:
    global _lib
    with _lock:
        if _lib is None:
            _lib = Oracle(build())
    return _lib


def variant(src_text: str, workdir: str) -> Oracle:
    """Compile a modified copy of the oracle source (used by tests that plant mistakes)."""
    src = os.path.join(workdir, "oracle_variant.c")
    with open(src, "w") as f:
        f.write(src_text)
    lib = os.path.join(workdir, "oracle_variant.so")
    _compile(src, lib)
    return Oracle(lib)


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def has_openmp() -> bool:
    return default().has_openmp()


def rhs(U, gamma=1.4, eps=0.25, h=(1.0, 1.0, 1.0), halo=2, k_range=None, threads=1, out=None):
    """As-written RHS through the default oracle build (see `Oracle.rhs`)."""
    return default().rhs(U, gamma, eps, h, halo, k_range, threads, out)


def block(A, B, G, prm=(0.01, 1.5, 2.0, 0.75, 0.5), halo=1, k_range=None, threads=1):
    """Block-assembly body through the default oracle build (see `Oracle.block`)."""
    return default().block(A, B, G, prm, halo, k_range, threads)


def stencil(u, a, c=None, halo=4, k_range=None, threads=1):
    """As-written star stencil through the default oracle build (see `Oracle.stencil`)."""
    return default().stencil(u, a, c, halo, k_range, threads)


TAYLOR8 = (8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0)


def taylor_coeffs() -> np.ndarray:
    """c[3][4]: the 8th-order central second-derivative weights (h = 1) on every axis."""
    return np.array([TAYLOR8] * 3, dtype=np.float64)


