"""The allocation-free batch entry point (acs_batch_run_static) against the workspace batch.

Some callers of this library cannot allocate device memory when they run a batch (their
application owns the device budget through its own allocator, or a time-critical loop cannot
take the synchronisation an allocation may bring). acs_batch_run_static serves them from a
fixed scratch array inside the library. This file runs last in the suite so that a failure
here cannot hide any other test.
"""
import ctypes

import pytest

from paper_2306_13002_gb300 import binding, inputs
from paper_2306_13002_gb300 import build as acs_build
from _parity import assert_parity, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _grids(kind, sides, seed0):
    grids = []
    for q, (nx, ny, nz) in enumerate(sides):
        nx, ny, nz = int(nx), int(ny), int(nz)
        if kind == binding.KIND_STENCIL:
            u, a = inputs.stencil_fields(nx, ny, nz, halo=4, seed=seed0 + q)
            grids.append((to_dev(u), to_dev(a), torch.full((nz, ny, nx), float("nan"), dtype=torch.float64,
                                                           device="cuda")))
        else:
            U = inputs.rhs_field(nx, ny, nz, halo=2, seed=seed0 + q)
            grids.append((to_dev(U), None, torch.full((5, nz, ny, nx), float("nan"), dtype=torch.float64,
                                                      device="cuda")))
    return grids


def _static_call(kind, grids, params):
    """Call the entry point through the C ABI directly."""
    items = binding.batch_items(kind, grids)
    ptr, keep = binding._batch_params(kind, params)
    st = binding.lib().acs_batch_run_static(items, len(grids), kind, None, ptr,
                                            torch.cuda.current_stream().cuda_stream)
    del keep
    return st


@pytest.mark.parametrize("kind", [binding.KIND_STENCIL, binding.KIND_RHS])
def test_static_scratch_batch_matches_workspace_batch(kind):
    acs_build.build()
    sides = inputs.batch_sides(24, seed=inputs.SEED_BATCH + 9, lo=4, hi=48)
    grids = _grids(kind, sides, 9100)
    ref_grids = [(g[0], g[1], torch.empty_like(g[2])) for g in grids]
    params = None if kind == binding.KIND_STENCIL else {"gamma": 1.4, "eps": 0.25, "h": (1.0, 0.5, 2.0)}
    ws = torch.zeros((binding.acs_batch_workspace_bytes(len(grids)) + 15) // 16 * 2, dtype=torch.float64,
                     device="cuda")
    plan = binding.acs_batch_prepare(kind, ref_grids, ws)
    for call in range(2):                          # two calls in a row, new inputs each time
        if call == 1:
            for (x, _, out) in grids:
                x.mul_(1.25)
                out.fill_(float("nan"))
        assert _static_call(kind, grids, params) == binding.ACS_OK, binding.lib().acs_last_error()
        binding.acs_batch_launch(plan, params)
        torch.cuda.synchronize()
        for q, ((_, _, out), (_, _, ref)) in enumerate(zip(grids, ref_grids)):
            assert_parity(out.cpu().numpy(), ref.cpu().numpy(), what=f"call {call} grid {q}")


def test_static_scratch_rejects_oversized_batch():
    acs_build.build()
    grids = _grids(binding.KIND_STENCIL, [(2, 2, 2)], 9200)
    many = grids * (binding.BATCH_STATIC_MAX + 1)
    out_before = grids[0][2].clone()
    st = _static_call(binding.KIND_STENCIL, many, None)
    assert st == 8, binding.acs_status_string(st)   # ACS_ERR_WORKSPACE
    assert b"static scratch maximum" in binding.lib().acs_last_error()
    torch.cuda.synchronize()
    assert torch.equal(torch.isnan(grids[0][2]), torch.isnan(out_before))
