"""Thin ctypes binding of `libacs.so` (argument marshalling only).

The functions carry the C-ABI names of `include/acs.h`. They accept torch CUDA tensors
(or any object with `data_ptr()`, `stride()`, `shape`), build the `acs_grid` from the
tensors' own strides, call the library on the given stream and raise `AcsError` on a
non-OK status. Every step of the computation runs in the CUDA library; if it is missing,
loading fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libacs.so")

ACS_OK = 0
STATUS_NAMES = {
    0: "ACS_OK", 1: "ACS_ERR_INVALID", 2: "ACS_ERR_ALIGN", 3: "ACS_ERR_CUDA", 4: "ACS_ERR_UNSUPPORTED",
    5: "ACS_ERR_TIMEOUT", 6: "ACS_ERR_NOMODEL", 7: "ACS_ERR_ALIAS", 8: "ACS_ERR_WORKSPACE",
}

TAYLOR8 = (8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0)


class AcsError(RuntimeError):
    def __init__(self, status: int, func: str, detail: str):
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{func}: {self.name}: {detail}")


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("halo", ctypes.c_int),
                ("in_sy", ctypes.c_longlong), ("in_sz", ctypes.c_longlong), ("in_sc", ctypes.c_longlong),
                ("out_sy", ctypes.c_longlong), ("out_sz", ctypes.c_longlong), ("out_sc", ctypes.c_longlong)]


class RhsParams(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("eps", ctypes.c_double), ("h", ctypes.c_double * 3)]


class Tile(ctypes.Structure):
    _fields_ = [("bx", ctypes.c_int), ("by", ctypes.c_int), ("kchunk", ctypes.c_int), ("flags", ctypes.c_int)]


class BatchItem(ctypes.Structure):
    _fields_ = [("in0", ctypes.c_void_p), ("in1", ctypes.c_void_p), ("out", ctypes.c_void_p), ("g", Grid)]


class BatchPlan(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int), ("tile", Tile), ("total_units", ctypes.c_longlong),
                ("ws", ctypes.c_void_p), ("ws_bytes", ctypes.c_size_t)]


KIND_RHS, KIND_STENCIL = 0, 1
TILE_BALANCED = 1  # acs_tile.flags: one block per resident slot, equal (column, plane) shares
TILE_TMA = 2       # acs_tile.flags: planes staged by TMA tensor copies (single-grid saturated kernels)
VARIANT_NFEAT = 20
SCOPE_ITERATION, SCOPE_MARCH = 0, 1   # acs_scope


class VariantInfo(ctypes.Structure):
    _fields_ = [("feats", ctypes.c_float * VARIANT_NFEAT), ("cost", ctypes.c_double), ("enodes", ctypes.c_int),
                ("eclasses", ctypes.c_int), ("iterations", ctypes.c_int), ("scope", ctypes.c_int),
                ("block_x", ctypes.c_int), ("block_y", ctypes.c_int), ("flags", ctypes.c_int),
                ("src_bytes", ctypes.c_longlong), ("dag_bytes", ctypes.c_longlong)]


class RankerModel(ctypes.Structure):
    _fields_ = [("n_feats", ctypes.c_int), ("hidden", ctypes.c_int), ("params", ctypes.c_void_p)]

_lock = threading.Lock()
_lib = None

FORMS = {"as_written": 0, "cse": 1, "cse_sat": 2, "cse_bulk": 3, "accsat": 4, "saturated": 5}

EXPORTS = ("acs_rhs_plain", "acs_rhs_saturated", "acs_rhs_form", "acs_stencil_plain", "acs_stencil_saturated",
           "acs_batch_workspace_bytes", "acs_batch_prepare", "acs_batch_launch", "acs_batch_run_static",
           "acs_autotune_rhs",
           "acs_autotune_stencil", "acs_autotune_batch", "acs_tune_cache_save", "acs_tune_cache_load",
           "acs_tune_cache_clear", "acs_tune_cache_size", "acs_variant_generate", "acs_variant_feature_name",
           "acs_variant_build", "acs_variant_launch", "acs_variant_free", "acs_ranker_param_count",
           "acs_ranker_workspace_bytes", "acs_ranker_train", "acs_variant_rank", "acs_status_string",
           "acs_last_error", "acs_abi_version", "acs_block_form", "acs_rhs_host_workspace_bytes",
           "acs_rhs_saturated_host", "acs_wait_timeouts", "acs_wait_selftest", "acs_ranker_gradient",
           "acs_ranker_save", "acs_ranker_load", "acs_fp64_rate_probe", "acs_rcp_selftest")


def lib() -> ctypes.CDLL:
    """Load libacs.so (built by `build.build()` / `__graft_entry__.build()`)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                                   "(run paper_2306_13002_gb300.build.build())")
            L = ctypes.CDLL(LIB_PATH)
            p, st = ctypes.c_void_p, ctypes.c_int
            L.acs_rhs_plain.argtypes = [p, p, ctypes.POINTER(Grid), ctypes.POINTER(RhsParams), p]
            L.acs_rhs_saturated.argtypes = [p, p, ctypes.POINTER(Grid), ctypes.POINTER(RhsParams),
                                            ctypes.POINTER(Tile), p, p]
            L.acs_rhs_form.argtypes = [p, p, ctypes.POINTER(Grid), ctypes.POINTER(RhsParams), st,
                                       ctypes.POINTER(Tile), p]
            L.acs_stencil_plain.argtypes = [p, p, p, ctypes.POINTER(Grid), ctypes.POINTER(ctypes.c_double), p]
            L.acs_stencil_saturated.argtypes = [p, p, p, ctypes.POINTER(Grid), ctypes.POINTER(ctypes.c_double),
                                                ctypes.POINTER(Tile), p]
            for f in ("acs_rhs_plain", "acs_rhs_saturated", "acs_rhs_form", "acs_stencil_plain",
                      "acs_stencil_saturated"):
                getattr(L, f).restype = st
            T, G = ctypes.POINTER(Tile), ctypes.POINTER(Grid)
            f32p = ctypes.POINTER(ctypes.c_float)
            L.acs_batch_workspace_bytes.argtypes = [st]
            L.acs_batch_workspace_bytes.restype = ctypes.c_size_t
            L.acs_batch_prepare.argtypes = [ctypes.POINTER(BatchItem), st, st, T, p, ctypes.c_size_t,
                                            ctypes.POINTER(BatchPlan), p]
            L.acs_batch_launch.argtypes = [ctypes.POINTER(BatchPlan), p, p]
            L.acs_batch_run_static.argtypes = [ctypes.POINTER(BatchItem), st, st, T, p, p]
            L.acs_autotune_rhs.argtypes = [p, p, G, ctypes.POINTER(RhsParams), T, f32p, p]
            L.acs_autotune_stencil.argtypes = [p, p, p, G, ctypes.POINTER(ctypes.c_double), T, f32p, p]
            L.acs_autotune_batch.argtypes = [ctypes.POINTER(BatchItem), st, st, p, p, ctypes.c_size_t, T, f32p, p]
            L.acs_tune_cache_save.argtypes = [ctypes.c_char_p]
            L.acs_tune_cache_load.argtypes = [ctypes.c_char_p]
            L.acs_tune_cache_clear.restype = None
            L.acs_tune_cache_size.restype = st
            for f in ("acs_batch_prepare", "acs_batch_launch", "acs_batch_run_static", "acs_autotune_rhs", "acs_autotune_stencil",
                      "acs_autotune_batch", "acs_tune_cache_save", "acs_tune_cache_load"):
                getattr(L, f).restype = st
            L.acs_variant_generate.argtypes = [ctypes.c_ulonglong, st, st, ctypes.c_char_p, ctypes.c_size_t,
                                               ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(VariantInfo)]
            L.acs_variant_feature_name.argtypes = [st]
            L.acs_variant_feature_name.restype = ctypes.c_char_p
            L.acs_variant_build.argtypes = [ctypes.c_char_p, ctypes.POINTER(VariantInfo), ctypes.POINTER(ctypes.c_void_p),
                                            ctypes.POINTER(ctypes.c_int)]
            L.acs_variant_launch.argtypes = [p, p, p, G, ctypes.POINTER(RhsParams), p]
            L.acs_variant_free.argtypes = [p]
            L.acs_variant_free.restype = None
            L.acs_ranker_param_count.argtypes = [st, st]
            L.acs_ranker_param_count.restype = ctypes.c_size_t
            L.acs_ranker_workspace_bytes.argtypes = [st, st, st]
            L.acs_ranker_workspace_bytes.restype = ctypes.c_size_t
            L.acs_ranker_train.argtypes = [p, p, st, st, st, st, ctypes.c_float, ctypes.c_float, ctypes.c_ulonglong,
                                           p, p, ctypes.c_size_t, p]
            L.acs_variant_rank.argtypes = [p, st, st, ctypes.POINTER(RankerModel), p, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_float), p]
            for f in ("acs_variant_generate", "acs_variant_build", "acs_variant_launch", "acs_ranker_train",
                      "acs_variant_rank"):
                getattr(L, f).restype = st
            L.acs_block_form.argtypes = [p, p, p, p, G, ctypes.POINTER(ctypes.c_double), st, p]
            L.acs_block_form.restype = st
            L.acs_rhs_host_workspace_bytes.argtypes = [G, st]
            L.acs_rhs_host_workspace_bytes.restype = ctypes.c_size_t
            L.acs_rhs_saturated_host.argtypes = [p, p, G, ctypes.POINTER(RhsParams), T, st, p, ctypes.c_size_t, p]
            L.acs_rhs_saturated_host.restype = st
            L.acs_status_string.argtypes = [st]
            L.acs_status_string.restype = ctypes.c_char_p
            L.acs_last_error.restype = ctypes.c_char_p
            L.acs_abi_version.restype = ctypes.c_int
            L.acs_wait_timeouts.argtypes = [ctypes.POINTER(ctypes.c_uint)]
            L.acs_wait_timeouts.restype = st
            L.acs_wait_selftest.argtypes = [ctypes.POINTER(ctypes.c_uint), ctypes.c_void_p]
            L.acs_wait_selftest.restype = st
            L.acs_ranker_gradient.argtypes = [p, p, st, st, st, p, ctypes.c_float, p, p, ctypes.c_size_t, p]
            L.acs_ranker_save.argtypes = [ctypes.c_char_p, ctypes.POINTER(RankerModel)]
            L.acs_ranker_load.argtypes = [ctypes.c_char_p, p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]
            L.acs_fp64_rate_probe.argtypes = [p, st, st, st, ctypes.POINTER(ctypes.c_longlong), p]
            L.acs_rcp_selftest.argtypes = [p, p, ctypes.c_longlong, p]
            for f in ("acs_ranker_gradient", "acs_ranker_save", "acs_ranker_load", "acs_fp64_rate_probe",
                      "acs_rcp_selftest"):
                getattr(L, f).restype = st
            _lib = L
    return _lib


def _check(status: int, func: str) -> None:
    if status != ACS_OK:
        raise AcsError(status, func, lib().acs_last_error().decode())


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream or None
        except Exception:  # pragma: no cover
            return None
    if isinstance(stream, int):
        return stream or None
    return getattr(stream, "cuda_stream", None) or None


def _tile(tile) -> ctypes.POINTER(Tile) | None:
    if tile is None:
        return None
    if isinstance(tile, Tile):
        return ctypes.byref(tile)
    bx, by, kchunk, flags = (tuple(tile) + (0, 0, 0, 0))[:4]
    return ctypes.byref(Tile(int(bx), int(by), int(kchunk), int(flags)))


def _on_device(*tensors) -> None:
    """The device entry points take device memory: refuse host tensors before any launch."""
    for t in tensors:
        if t is not None and not t.is_cuda:
            raise ValueError("device entry points take CUDA tensors; got a tensor on " + str(t.device))


def grid_for(inp, out, halo: int, ncomp: int, host: bool = False) -> Grid:
    """acs_grid from an input (halo-extended) and an output tensor's shapes and strides; both on
    the GPU, or both on the host for the host-streamed entry point (host=True)."""
    if host:
        if inp.is_cuda or out.is_cuda:
            raise ValueError("the host-streamed entry point takes host (CPU) tensors")
    else:
        _on_device(inp, out)
    if ncomp == 5:
        _, Z, Y, X = inp.shape
        isc, isz, isy, isx = inp.stride()
        osc, osz, osy, osx = out.stride()
        onz, ony, onx = out.shape[1:]
    else:
        Z, Y, X = inp.shape
        isz, isy, isx = inp.stride()
        osz, osy, osx = out.stride()
        isc = osc = 0
        onz, ony, onx = out.shape
    if isx != 1 or osx != 1:
        raise ValueError("x must be the unit-stride axis of input and output")
    nx, ny, nz = X - 2 * halo, Y - 2 * halo, Z - 2 * halo
    if (onx, ony, onz) != (nx, ny, nz):
        raise ValueError(f"output shape {(onz, ony, onx)} does not match the interior {(nz, ny, nx)}")
    return Grid(nx, ny, nz, halo, isy, isz, isc, osy, osz, osc)


def _params(gamma, eps, h) -> RhsParams:
    return RhsParams(float(gamma), float(eps), (ctypes.c_double * 3)(*[float(v) for v in h]))


def acs_rhs_plain(U, R, gamma: float = 1.4, eps: float = 0.25, h=(1.0, 1.0, 1.0), halo: int = 2,
                  stream=None) -> None:
    g = grid_for(U, R, halo, 5)
    pr = _params(gamma, eps, h)
    _check(lib().acs_rhs_plain(U.data_ptr(), R.data_ptr(), ctypes.byref(g), ctypes.byref(pr),
                               _stream_ptr(stream)), "acs_rhs_plain")


def acs_rhs_saturated(U, R, gamma: float = 1.4, eps: float = 0.25, h=(1.0, 1.0, 1.0), halo: int = 2,
                      tile=None, variant=None, stream=None) -> None:
    """Saturated RHS; `variant` None for the library's kernel, or a march-scope `Variant`."""
    g = grid_for(U, R, halo, 5)
    pr = _params(gamma, eps, h)
    vh = variant.handle if variant is not None else None
    if variant is not None and not vh:
        raise ValueError("variant has been closed")
    _check(lib().acs_rhs_saturated(U.data_ptr(), R.data_ptr(), ctypes.byref(g), ctypes.byref(pr), _tile(tile), vh,
                                   _stream_ptr(stream)), "acs_rhs_saturated")


def acs_rhs_form(U, R, form, gamma: float = 1.4, eps: float = 0.25, h=(1.0, 1.0, 1.0), halo: int = 2,
                 tile=None, stream=None) -> None:
    """RHS in one code version; `form` is an acs_form value or a name from FORMS."""
    f = FORMS[form] if isinstance(form, str) else int(form)
    g = grid_for(U, R, halo, 5)
    pr = _params(gamma, eps, h)
    _check(lib().acs_rhs_form(U.data_ptr(), R.data_ptr(), ctypes.byref(g), ctypes.byref(pr), f, _tile(tile),
                              _stream_ptr(stream)), "acs_rhs_form")


def _coef(c) -> ctypes.Array:
    if c is None:
        vals = list(TAYLOR8) * 3
    else:
        vals = [float(v) for row in c for v in (row if hasattr(row, "__len__") else [row])]
    if len(vals) != 12:
        raise ValueError("stencil coefficients must be 3 x 4")
    return (ctypes.c_double * 12)(*vals)


def acs_stencil_plain(u, a, out, c=None, halo: int = 4, stream=None) -> None:
    g = grid_for(u, out, halo, 1)
    _on_device(a)
    if tuple(a.stride()) != tuple(u.stride()) or tuple(a.shape) != tuple(u.shape):
        raise ValueError("u and a must have the same shape and strides")
    _check(lib().acs_stencil_plain(u.data_ptr(), a.data_ptr(), out.data_ptr(), ctypes.byref(g), _coef(c),
                                   _stream_ptr(stream)), "acs_stencil_plain")


def acs_stencil_saturated(u, a, out, c=None, halo: int = 4, tile=None, stream=None) -> None:
    g = grid_for(u, out, halo, 1)
    _on_device(a)
    if tuple(a.stride()) != tuple(u.stride()) or tuple(a.shape) != tuple(u.shape):
        raise ValueError("u and a must have the same shape and strides")
    _check(lib().acs_stencil_saturated(u.data_ptr(), a.data_ptr(), out.data_ptr(), ctypes.byref(g), _coef(c),
                                       _tile(tile), _stream_ptr(stream)), "acs_stencil_saturated")


def acs_wait_timeouts() -> int:
    """Bounded device-side waits that ran out on the current device (0 in normal operation);
    synchronous, call it after the work has completed."""
    n = ctypes.c_uint(0)
    _check(lib().acs_wait_timeouts(ctypes.byref(n)), "acs_wait_timeouts")
    return int(n.value)


def acs_wait_selftest(stream=None) -> int:
    """Run the bounded-wait path once (32 waits on an mbarrier phase nothing completes, about
    one second); returns how many waits ran out (32 when the path works)."""
    n = ctypes.c_uint(0)
    _check(lib().acs_wait_selftest(ctypes.byref(n), _stream_ptr(stream)), "acs_wait_selftest")
    return int(n.value)


def acs_status_string(status: int) -> str:
    return lib().acs_status_string(int(status)).decode()


def acs_abi_version() -> int:
    return int(lib().acs_abi_version())


# ------------------------------------------------------------------ batch and autotune

def acs_batch_workspace_bytes(n: int) -> int:
    return int(lib().acs_batch_workspace_bytes(int(n)))


def batch_items(kind: int, grids, halo: int | None = None):
    """ctypes array of acs_batch_item from (in0, in1, out) tensor triples (in1 None for the RHS)."""
    halo = (2 if kind == KIND_RHS else 4) if halo is None else halo
    arr = (BatchItem * len(grids))()
    for q, (in0, in1, out) in enumerate(grids):
        g = grid_for(in0, out, halo, 5 if kind == KIND_RHS else 1)
        _on_device(in1)
        arr[q] = BatchItem(in0.data_ptr(), in1.data_ptr() if in1 is not None else None, out.data_ptr(), g)
    return arr


def _batch_params(kind: int, params):
    """(void* for the C call, object to keep alive during the call)."""
    if kind == KIND_RHS:
        if params is None:
            params = {}
        pr = params if isinstance(params, RhsParams) else _params(
            params.get("gamma", 1.4), params.get("eps", 0.25), params.get("h", (1.0, 1.0, 1.0)))
        return ctypes.cast(ctypes.pointer(pr), ctypes.c_void_p), pr
    c = _coef(params)
    return ctypes.cast(c, ctypes.c_void_p), c


def acs_batch_prepare(kind: int, grids, ws, tile=None, halo: int | None = None, stream=None) -> BatchPlan:
    """Validate and upload a batch; `ws` is a device tensor of >= acs_batch_workspace_bytes(n) bytes."""
    _on_device(ws)
    items = batch_items(kind, grids, halo)
    plan = BatchPlan()
    nbytes = ws.numel() * ws.element_size()
    _check(lib().acs_batch_prepare(items, len(grids), kind, _tile(tile), ws.data_ptr(), nbytes, ctypes.byref(plan),
                                   _stream_ptr(stream)), "acs_batch_prepare")
    plan._keep = (items, ws, grids)
    return plan


def acs_batch_launch(plan: BatchPlan, params=None, stream=None) -> None:
    ptr, keep = _batch_params(plan.kind, params)
    _check(lib().acs_batch_launch(ctypes.byref(plan), ptr, _stream_ptr(stream)), "acs_batch_launch")
    del keep


BATCH_STATIC_MAX = 256


def acs_batch_run_static(kind: int, grids, params=None, tile=None, halo: int | None = None, stream=None) -> None:
    """Run a batch with the library's fixed device scratch: no workspace, no allocation.

    For callers that cannot allocate device memory when they run a batch (a fixed budget
    handed out by their own allocator, or a loop that cannot accept an allocation's
    synchronisation). At most BATCH_STATIC_MAX grids; calls share the scratch, so calls
    whose kernels overlap on the GPU race. Every call synchronises the stream (it uploads
    the unit table), so it cannot run inside a CUDA-graph capture; use acs_batch_prepare and
    acs_batch_launch for a graph.
    """
    items = batch_items(kind, grids, halo)
    ptr, keep = _batch_params(kind, params)
    _check(lib().acs_batch_run_static(items, len(grids), kind, _tile(tile), ptr, _stream_ptr(stream)),
           "acs_batch_run_static")
    del keep


def acs_autotune_rhs(U, R, gamma=1.4, eps=0.25, h=(1.0, 1.0, 1.0), halo=2, stream=None):
    g = grid_for(U, R, halo, 5)
    pr = _params(gamma, eps, h)
    t, ms = Tile(), ctypes.c_float()
    _check(lib().acs_autotune_rhs(U.data_ptr(), R.data_ptr(), ctypes.byref(g), ctypes.byref(pr), ctypes.byref(t),
                                  ctypes.byref(ms), _stream_ptr(stream)), "acs_autotune_rhs")
    return (t.bx, t.by, t.kchunk, t.flags), ms.value


def acs_autotune_stencil(u, a, out, c=None, halo=4, stream=None):
    g = grid_for(u, out, halo, 1)
    t, ms = Tile(), ctypes.c_float()
    _check(lib().acs_autotune_stencil(u.data_ptr(), a.data_ptr(), out.data_ptr(), ctypes.byref(g), _coef(c),
                                      ctypes.byref(t), ctypes.byref(ms), _stream_ptr(stream)), "acs_autotune_stencil")
    return (t.bx, t.by, t.kchunk, t.flags), ms.value


def acs_autotune_batch(kind: int, grids, ws, params=None, halo=None, stream=None):
    _on_device(ws)
    items = batch_items(kind, grids, halo)
    ptr, keep = _batch_params(kind, params)
    t, ms = Tile(), ctypes.c_float()
    nbytes = ws.numel() * ws.element_size()
    _check(lib().acs_autotune_batch(items, len(grids), kind, ptr, ws.data_ptr(), nbytes, ctypes.byref(t),
                                    ctypes.byref(ms), _stream_ptr(stream)), "acs_autotune_batch")
    del keep
    return (t.bx, t.by, t.kchunk, t.flags), ms.value


def acs_tune_cache_save(path: str) -> None:
    _check(lib().acs_tune_cache_save(path.encode()), "acs_tune_cache_save")


def acs_tune_cache_load(path: str) -> None:
    _check(lib().acs_tune_cache_load(path.encode()), "acs_tune_cache_load")


def acs_tune_cache_clear() -> None:
    lib().acs_tune_cache_clear()


def acs_tune_cache_size() -> int:
    return int(lib().acs_tune_cache_size())


# ------------------------------------------------------------------ rewriter and ranker

def acs_variant_feature_names() -> list[str]:
    return [lib().acs_variant_feature_name(i).decode() for i in range(VARIANT_NFEAT)]


def acs_variant_generate(seed: int, index: int, scope: int = SCOPE_ITERATION):
    """(cuda_source, dag_text, VariantInfo) of rewriter variant `index` in `scope` (host only)."""
    info = VariantInfo()
    _check(lib().acs_variant_generate(int(seed), int(index), int(scope), None, 0, None, 0, ctypes.byref(info)),
           "acs_variant_generate")
    src = ctypes.create_string_buffer(int(info.src_bytes))
    dag = ctypes.create_string_buffer(int(info.dag_bytes))
    _check(lib().acs_variant_generate(int(seed), int(index), int(scope), src, len(src), dag, len(dag),
                                      ctypes.byref(info)), "acs_variant_generate")
    return src.value.decode(), dag.value.decode(), info


class Variant:
    """A compiled, loaded rewriter variant (freed with close())."""

    def __init__(self, src: str, info: VariantInfo):
        h, regs = ctypes.c_void_p(), ctypes.c_int()
        _check(lib().acs_variant_build(src.encode(), ctypes.byref(info), ctypes.byref(h), ctypes.byref(regs)),
               "acs_variant_build")
        self.handle, self.regs = h, regs.value
        self.scope, self.block = int(info.scope), (int(info.block_x), int(info.block_y))
        self.flags = int(info.flags)

    def launch(self, U, R, gamma=1.4, eps=0.25, h=(1.0, 1.0, 1.0), halo=2, stream=None):
        g = grid_for(U, R, halo, 5)
        pr = _params(gamma, eps, h)
        _check(lib().acs_variant_launch(self.handle, U.data_ptr(), R.data_ptr(), ctypes.byref(g), ctypes.byref(pr),
                                        _stream_ptr(stream)), "acs_variant_launch")

    def close(self):
        if self.handle:
            lib().acs_variant_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def acs_ranker_param_count(n_feats: int, hidden: int) -> int:
    return int(lib().acs_ranker_param_count(int(n_feats), int(hidden)))


def acs_ranker_workspace_bytes(n: int, n_feats: int, hidden: int) -> int:
    return int(lib().acs_ranker_workspace_bytes(int(n), int(n_feats), int(hidden)))


def acs_ranker_train(feats, times_ms, params, ws, hidden=64, epochs=3000, lr=3e-3, seed=13006, fast_weight=0.0,
                     stream=None):
    """Train the MLP on device tensors feats (n x F float32) and times_ms (n float32)."""
    _on_device(feats, times_ms, params, ws)
    n, F = feats.shape
    _check(lib().acs_ranker_train(feats.data_ptr(), times_ms.data_ptr(), int(n), int(F), int(hidden), int(epochs),
                                  float(lr), float(fast_weight), int(seed), params.data_ptr(), ws.data_ptr(),
                                  ws.numel() * ws.element_size(), _stream_ptr(stream)), "acs_ranker_train")


def acs_variant_rank(feats, params=None, hidden=64, scores_dev=None, stream=None):
    """(order fastest-first, scores) for device feats; params None = the paper's analytical cost."""
    import torch
    _on_device(feats, params, scores_dev)
    n, F = feats.shape
    if scores_dev is None:
        scores_dev = torch.empty(n, dtype=torch.float32, device=feats.device)
    order = (ctypes.c_int * n)()
    score = (ctypes.c_float * n)()
    model = RankerModel(int(F), int(hidden), params.data_ptr()) if params is not None else None
    _check(lib().acs_variant_rank(feats.data_ptr(), int(n), int(F), ctypes.byref(model) if model else None,
                                  scores_dev.data_ptr(), order, score, _stream_ptr(stream)), "acs_variant_rank")
    return list(order), list(score)


def acs_ranker_gradient(feats, times_ms, params, grad, ws, hidden=64, fast_weight=0.0, stream=None) -> None:
    """Loss gradient at `params` (no update) into the device tensor `grad` (P floats)."""
    _on_device(feats, times_ms, params, grad, ws)
    n, F = feats.shape
    _check(lib().acs_ranker_gradient(feats.data_ptr(), times_ms.data_ptr(), int(n), int(F), int(hidden),
                                     params.data_ptr(), float(fast_weight), grad.data_ptr(), ws.data_ptr(),
                                     ws.numel() * ws.element_size(), _stream_ptr(stream)), "acs_ranker_gradient")


def acs_ranker_save(path: str, params, n_feats: int, hidden: int = 64) -> None:
    _on_device(params)
    model = RankerModel(int(n_feats), int(hidden), params.data_ptr())
    _check(lib().acs_ranker_save(str(path).encode(), ctypes.byref(model)), "acs_ranker_save")


def acs_ranker_load(path: str, device="cuda"):
    """(params device tensor, n_feats, hidden) from a model file written by acs_ranker_save."""
    import torch
    F, H = ctypes.c_int(), ctypes.c_int()
    _check(lib().acs_ranker_load(str(path).encode(), None, 0, ctypes.byref(F), ctypes.byref(H)), "acs_ranker_load")
    params = torch.empty(acs_ranker_param_count(F.value, H.value), dtype=torch.float32, device=device)
    _check(lib().acs_ranker_load(str(path).encode(), params.data_ptr(), params.numel(), None, None),
           "acs_ranker_load")
    return params, F.value, H.value


def acs_fp64_rate_probe(sink, blocks: int, threads: int, iters: int, stream=None) -> int:
    """Launch the FP64-pipe probe (asynchronous); returns the FP64 operations it issues."""
    _on_device(sink)
    if sink.numel() < blocks * threads:
        raise ValueError("sink holds fewer than blocks x threads doubles")
    ops = ctypes.c_longlong()
    _check(lib().acs_fp64_rate_probe(sink.data_ptr(), int(blocks), int(threads), int(iters), ctypes.byref(ops),
                                     _stream_ptr(stream)), "acs_fp64_rate_probe")
    return int(ops.value)


def acs_rcp_selftest(x, y, stream=None) -> None:
    """y = the saturated RHS's reciprocal of x (device float64 tensors of equal size)."""
    _on_device(x, y)
    if x.numel() != y.numel() or not x.is_contiguous() or not y.is_contiguous():
        raise ValueError("x and y must be contiguous and of equal size")
    _check(lib().acs_rcp_selftest(x.data_ptr(), y.data_ptr(), int(x.numel()), _stream_ptr(stream)),
           "acs_rcp_selftest")


BLOCK_PRM = (0.01, 1.5, 2.0, 0.75, 0.5)


def acs_block_form(A, B, G, out, form, prm=BLOCK_PRM, halo: int = 1, stream=None) -> None:
    """Block-assembly body; A, B (25, Z, Y, X), G (Z, Y, X), out (75, nz, ny, nx) device tensors."""
    f = FORMS[form] if isinstance(form, str) else int(form)
    _on_device(A, B, G, out)
    _, Z, Y, X = A.shape
    isc, isz, isy, isx = A.stride()
    if tuple(B.stride()) != (isc, isz, isy, isx) or tuple(G.stride()) != (isz, isy, isx) or isx != 1:
        raise ValueError("A, B and G must share strides (x unit stride)")
    osc, osz, osy, osx = out.stride()
    nx, ny, nz = X - 2 * halo, Y - 2 * halo, Z - 2 * halo
    if tuple(out.shape) != (75, nz, ny, nx) or osx != 1:
        raise ValueError("out must be (75, nz, ny, nx) with unit x stride")
    g = Grid(nx, ny, nz, halo, isy, isz, isc, osy, osz, osc)
    pr = (ctypes.c_double * 5)(*[float(v) for v in prm])
    _check(lib().acs_block_form(A.data_ptr(), B.data_ptr(), G.data_ptr(), out.data_ptr(), ctypes.byref(g), pr, f,
                                _stream_ptr(stream)), "acs_block_form")


def acs_rhs_host_workspace_bytes(U_host, R_host, halo: int = 2, slab: int = 0) -> int:
    g = grid_for(U_host, R_host, halo, 5, host=True)
    return int(lib().acs_rhs_host_workspace_bytes(ctypes.byref(g), int(slab)))


def acs_rhs_saturated_host(U_host, R_host, ws, gamma=1.4, eps=0.25, h=(1.0, 1.0, 1.0), halo=2, tile=None, slab=0,
                           stream=None) -> None:
    """Saturated RHS on host (CPU, ideally pinned) tensors, streamed in z-slabs through `ws` (device)."""
    g = grid_for(U_host, R_host, halo, 5, host=True)
    _on_device(ws)
    pr = _params(gamma, eps, h)
    _check(lib().acs_rhs_saturated_host(U_host.data_ptr(), R_host.data_ptr(), ctypes.byref(g), ctypes.byref(pr),
                                        _tile(tile), int(slab), ws.data_ptr(), ws.numel() * ws.element_size(),
                                        _stream_ptr(stream)), "acs_rhs_saturated_host")
