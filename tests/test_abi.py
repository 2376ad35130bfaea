"""C-ABI checks that need no GPU: the library loads, exports every symbol declared in
include/acs.h, and rejects bad arguments on the host before any launch.

The pointer values passed here are never dereferenced: argument checks return first.
"""
import ctypes
import os
import re

import pytest

from paper_2306_13002_gb300 import binding
from paper_2306_13002_gb300 import build as acs_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    acs_build.build()
    return binding.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "acs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(acs_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "acs_rhs_saturated" in names and "acs_stencil_plain" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in acs.h but not exported"


def test_abi_version_and_status_strings(lib):
    assert binding.acs_abi_version() >= 102
    for s in range(9):
        assert binding.acs_status_string(s) and binding.acs_status_string(s) != "unknown status"
    assert binding.acs_status_string(99) == "unknown status"


FAKE_U = 0x10000000            # 16-byte aligned fake device addresses, never dereferenced
FAKE_R = 0x40000000


def _grid(nx=8, ny=8, nz=8, halo=2, comp=True, pad=0):
    X, Y, Z = nx + 2 * halo + pad, ny + 2 * halo, nz + 2 * halo
    return binding.Grid(nx, ny, nz, halo, X, X * Y, X * Y * Z if comp else 0, nx, nx * ny, nx * ny * nz if comp else 0)


def _params(h=(1.0, 1.0, 1.0)):
    return binding.RhsParams(1.4, 0.25, (ctypes.c_double * 3)(*h))


def _call_rhs(lib, U, R, g, p, sat=False, tile=None):
    if sat:
        t = ctypes.byref(binding.Tile(*tile)) if tile else None
        return lib.acs_rhs_saturated(U, R, ctypes.byref(g) if g else None, ctypes.byref(p) if p else None, t, None,
                                     None)
    return lib.acs_rhs_plain(U, R, ctypes.byref(g) if g else None, ctypes.byref(p) if p else None, None)


@pytest.mark.parametrize("sat", [False, True])
def test_rhs_rejects_bad_arguments(lib, sat):
    E = binding
    cases = [
        (None, FAKE_R, _grid(), _params(), 1),
        (FAKE_U, None, _grid(), _params(), 1),
        (FAKE_U, FAKE_R, None, _params(), 1),
        (FAKE_U, FAKE_R, _grid(), None, 1),
        (FAKE_U + 4, FAKE_R, _grid(), _params(), 2),
        (FAKE_U, FAKE_R, _grid(nx=0), _params(), 1),
        (FAKE_U, FAKE_R, _grid(halo=1), _params(), 1),
        (FAKE_U, FAKE_R, _grid(), _params(h=(1.0, 0.0, 1.0)), 1),
        (FAKE_U, FAKE_R, _grid(), _params(h=(1.0, float("inf"), 1.0)), 1),
        (FAKE_U, FAKE_U + 8 * 100, _grid(), _params(), 7),           # output inside the input
    ]
    for U, R, g, p, want in cases:
        st = _call_rhs(lib, U, R, g, p, sat=sat)
        assert st == want, (st, want, E.acs_status_string(st))
        assert binding.lib().acs_last_error().decode()


def test_rhs_rejects_short_strides(lib):
    g = _grid()
    g.in_sy = 8                 # shorter than the extended row (12)
    assert _call_rhs(lib, FAKE_U, FAKE_R, g, _params()) == 1
    g = _grid()
    g.out_sc = 10
    assert _call_rhs(lib, FAKE_U, FAKE_R, g, _params()) == 1


@pytest.mark.parametrize("field,value", [("in_sy", 1 << 62), ("in_sz", 1 << 62), ("in_sc", (1 << 63) - 1),
                                         ("out_sy", 1 << 61), ("out_sc", 1 << 60)])
def test_rejects_strides_whose_extent_overflows(lib, field, value):
    """Huge strides (products with the extents past 64 bits, or arrays of 2^62 bytes and more)
    are rejected on the host, for both forms and the stencil."""
    g = _grid()
    setattr(g, field, value)
    if field == "in_sy":
        g.in_sz, g.in_sc = max(g.in_sz, 1 << 62), max(g.in_sc, 1 << 62)
    assert _call_rhs(lib, FAKE_U, FAKE_R, g, _params()) == 1
    assert _call_rhs(lib, FAKE_U, FAKE_R, g, _params(), sat=True) == 1
    gs = _grid(halo=4, comp=False)
    if field.endswith("sc"):
        return
    setattr(gs, field, value)
    c = (ctypes.c_double * 12)(*([1.0] * 12))
    assert lib.acs_stencil_saturated(FAKE_U, FAKE_U + 0x1000000, FAKE_R, ctypes.byref(gs), c, None, None) == 1


def test_saturated_rejects_unbuilt_tile_and_flags(lib):
    assert _call_rhs(lib, FAKE_U, FAKE_R, _grid(), _params(), sat=True, tile=(24, 8, 0, 0)) == 4
    assert _call_rhs(lib, FAKE_U, FAKE_R, _grid(), _params(), sat=True, tile=(32, 8, 0, 4)) == 1   # unknown flag
    assert _call_rhs(lib, FAKE_U, FAKE_R, _grid(), _params(), sat=True, tile=(32, 8, 0, 5)) == 1
    assert _call_rhs(lib, FAKE_U, FAKE_R, _grid(), _params(), sat=True, tile=(32, 8, -1, 0)) == 1


def test_stencil_rejects_bad_arguments(lib):
    c = (ctypes.c_double * 12)(*([1.0] * 12))
    g = _grid(halo=4, comp=False)
    A = FAKE_U + 0x1000000
    assert lib.acs_stencil_plain(FAKE_U, A, FAKE_R, ctypes.byref(g), None, None) == 1
    assert lib.acs_stencil_plain(FAKE_U, A, FAKE_R, ctypes.byref(_grid(halo=3, comp=False)), c, None) == 1
    assert lib.acs_stencil_plain(FAKE_U, A, A + 80, ctypes.byref(g), c, None) == 7      # out inside a
    bad = (ctypes.c_double * 12)(*([1.0] * 11 + [float("nan")]))
    assert lib.acs_stencil_saturated(FAKE_U, A, FAKE_R, ctypes.byref(g), bad, None, None) == 1
    t = binding.Tile(48, 8, 0, 0)
    assert lib.acs_stencil_saturated(FAKE_U, A, FAKE_R, ctypes.byref(g), c, ctypes.byref(t), None) == 4


def test_batch_prepare_rejects_bad_arguments(lib):
    g = _grid(halo=4, comp=False)
    A = FAKE_U + 0x1000000
    items = (binding.BatchItem * 2)(binding.BatchItem(FAKE_U, A, FAKE_R, g), binding.BatchItem(FAKE_U, A, FAKE_R, g))
    plan = binding.BatchPlan()
    need = binding.acs_batch_workspace_bytes(2)
    assert need > 0 and binding.acs_batch_workspace_bytes(0) == 0
    WS = 0x70000000
    st = lib.acs_batch_prepare(items, 2, 1, None, WS, need - 1, ctypes.byref(plan), None)
    assert st == 8                                                    # workspace too small
    assert lib.acs_batch_prepare(items, 2, 1, None, WS + 8, need, ctypes.byref(plan), None) == 2   # misaligned
    assert lib.acs_batch_prepare(items, 2, 1, None, None, need, ctypes.byref(plan), None) == 8
    assert lib.acs_batch_prepare(items, 0, 1, None, WS, need, ctypes.byref(plan), None) == 1
    assert lib.acs_batch_prepare(items, 2, 7, None, WS, need, ctypes.byref(plan), None) == 1
    assert lib.acs_batch_prepare(None, 2, 1, None, WS, need, ctypes.byref(plan), None) == 1
    bad = (binding.BatchItem * 1)(binding.BatchItem(FAKE_U, A, A + 80, g))
    assert lib.acs_batch_prepare(bad, 1, 1, None, WS, need, ctypes.byref(plan), None) == 7     # alias
    t = binding.Tile(24, 8, 8, 0)
    assert lib.acs_batch_prepare(items, 2, 1, ctypes.byref(t), WS, need, ctypes.byref(plan), None) == 4
    t = binding.Tile(32, 8, 8, binding.TILE_BALANCED)   # the batch takes work from its own queue
    assert lib.acs_batch_prepare(items, 2, 1, ctypes.byref(t), WS, need, ctypes.byref(plan), None) == 1


def test_batch_launch_rejects_unprepared_plan(lib):
    plan = binding.BatchPlan()
    c = (ctypes.c_double * 12)(*([1.0] * 12))
    assert lib.acs_batch_launch(ctypes.byref(plan), ctypes.cast(c, ctypes.c_void_p), None) == 1
    assert lib.acs_batch_launch(None, None, None) == 1


def test_tune_cache_file_errors(lib, tmp_path):
    assert lib.acs_tune_cache_load(str(tmp_path / "missing.txt").encode()) == 1
    p = tmp_path / "x.txt"
    p.write_text("not a cache\n")
    assert lib.acs_tune_cache_load(str(p).encode()) == 1
    lib.acs_tune_cache_clear()
    assert lib.acs_tune_cache_size() == 0


def test_wait_selftest_rejects_null_output(lib):
    assert lib.acs_wait_selftest(None, None) == 1        # ACS_ERR_INVALID before any launch


def test_binding_refuses_host_tensors_for_device_entry_points(lib):
    """The device entry points take CUDA tensors: host tensors are refused before any call, and
    the host-streamed entry point refuses the reverse."""
    torch = pytest.importorskip("torch")
    U = torch.zeros((5, 8, 8, 8), dtype=torch.float64)
    R = torch.zeros((5, 4, 4, 4), dtype=torch.float64)
    for fn in (binding.acs_rhs_plain, binding.acs_rhs_saturated):
        with pytest.raises(ValueError, match="CUDA tensors"):
            fn(U, R)
    u = torch.zeros((12, 12, 12), dtype=torch.float64)
    out = torch.zeros((4, 4, 4), dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA tensors"):
        binding.acs_stencil_saturated(u, u, out)
    with pytest.raises(ValueError, match="CUDA tensors"):
        binding.acs_batch_prepare(binding.KIND_STENCIL, [(u, u, out)], torch.zeros(64, dtype=torch.float64))
    with pytest.raises(ValueError, match="CUDA tensors"):
        binding.acs_rhs_saturated_host(U, R, torch.zeros(8, dtype=torch.float64))


def test_block_form_rejects_bad_arguments(lib):
    """The block-assembly body's host checks: NULL arrays, unknown form, short component strides,
    an output extent past 2^62 bytes (75 components), an output overlapping A."""
    nx = ny = nz = 8
    X = nx + 2
    g = binding.Grid(nx, ny, nz, 1, X, X * X, X ** 3, nx, nx * ny, nx * ny * nz)
    prm = (ctypes.c_double * 5)(*binding.BLOCK_PRM)
    A, B, G, OUT = 0x10000000, 0x20000000, 0x30000000, 0x40000000
    f = binding.FORMS["saturated"]
    assert lib.acs_block_form(None, B, G, OUT, ctypes.byref(g), prm, f, None) == 1
    assert lib.acs_block_form(A, B, G, OUT, ctypes.byref(g), prm, 99, None) == 1
    short = binding.Grid(nx, ny, nz, 1, X, X * X, X ** 3 - 1, nx, nx * ny, nx * ny * nz)
    assert lib.acs_block_form(A, B, G, OUT, ctypes.byref(short), prm, f, None) == 1
    huge = binding.Grid(nx, ny, nz, 1, X, X * X, X ** 3, nx, nx * ny, 1 << 58)
    assert lib.acs_block_form(A, B, G, OUT, ctypes.byref(huge), prm, f, None) == 1
    assert lib.acs_block_form(A, B, G, A + 8 * 100, ctypes.byref(g), prm, f, None) == 7   # overlaps A


def test_probe_and_selftest_entry_points_reject_bad_arguments(lib):
    ops = ctypes.c_longlong(-1)
    assert lib.acs_fp64_rate_probe(None, 4, 256, 10, ctypes.byref(ops), None) == 1
    for blocks, threads, iters in ((0, 256, 10), (4, 48, 10), (4, 2048, 10), (4, 256, 0)):
        assert lib.acs_fp64_rate_probe(FAKE_U, blocks, threads, iters, None, None) == 1
    assert lib.acs_fp64_rate_probe(FAKE_U + 4, 4, 256, 10, None, None) == 2
    assert lib.acs_rcp_selftest(FAKE_U, FAKE_R, -1, None) == 1
    assert lib.acs_rcp_selftest(None, FAKE_R, 8, None) == 1
    assert lib.acs_rcp_selftest(FAKE_U, FAKE_U + 8, 8, None) == 7        # y overlaps x
    assert lib.acs_rcp_selftest(FAKE_U, FAKE_R, 0, None) == 0            # nothing to do


def test_ranker_gradient_and_model_files_reject_bad_arguments(lib, tmp_path):
    assert lib.acs_ranker_gradient(None, FAKE_R, 8, 4, 16, FAKE_U, 1.0, FAKE_R, FAKE_U, 1 << 20, None) == 1
    assert lib.acs_ranker_gradient(FAKE_U, FAKE_R, 0, 4, 16, FAKE_U, 1.0, FAKE_R, FAKE_U, 1 << 20, None) == 1
    assert lib.acs_ranker_gradient(FAKE_U, FAKE_R, 8, 4, 16, FAKE_U, -1.0, FAKE_R, FAKE_U, 1 << 20, None) == 1
    assert lib.acs_ranker_train(FAKE_U, FAKE_R, 8, 4, 16, 10, 1e-3, 9.0, 1, FAKE_R, FAKE_U, 1 << 20, None) == 1
    assert lib.acs_ranker_save(None, None) == 1
    bad = tmp_path / "bad.model"
    bad.write_text("acs-ranker-model 1\n3 4 999\n")
    F, H = ctypes.c_int(), ctypes.c_int()
    assert lib.acs_ranker_load(str(bad).encode(), None, 0, ctypes.byref(F), ctypes.byref(H)) == 1
    bad.write_text("not a model\n")
    assert lib.acs_ranker_load(str(bad).encode(), None, 0, None, None) == 1
    assert lib.acs_ranker_load(str(tmp_path / "missing").encode(), None, 0, None, None) == 1
    # a well-formed file is read for its sizes without touching a device (params NULL)
    n_par = binding.acs_ranker_param_count(3, 4)
    good = tmp_path / "good.model"
    good.write_text("acs-ranker-model 1\n3 4 %d\n" % n_par + "0x1p-2\n" * n_par)
    assert lib.acs_ranker_load(str(good).encode(), None, 0, ctypes.byref(F), ctypes.byref(H)) == 0
    assert (F.value, H.value) == (3, 4)
    good.write_text("acs-ranker-model 1\n3 4 %d\n" % n_par + "0x1p-2\n" * (n_par - 1) + "nan\n")
    assert lib.acs_ranker_load(str(good).encode(), None, 0, None, None) == 1
