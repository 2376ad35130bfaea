"""GPU tests of the batched persistent launch, its CUDA-graph capture and the autotuner."""
import os

import numpy as np
import pytest

import oracle
from paper_2306_13002_gb300 import binding, inputs
from _parity import assert_parity, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _stencil_batch(sides, seed0):
    grids, host = [], []
    for q, (nx, ny, nz) in enumerate(sides):
        u, a = inputs.stencil_fields(int(nx), int(ny), int(nz), halo=4, seed=seed0 + q)
        out = torch.full((int(nz), int(ny), int(nx)), float("nan"), dtype=torch.float64, device="cuda")
        grids.append((to_dev(u), to_dev(a), out))
        host.append((u, a))
    return grids, host


def _ws(n):
    nbytes = binding.acs_batch_workspace_bytes(n)
    return torch.zeros((nbytes + 15) // 16 * 2, dtype=torch.float64, device="cuda")


def test_stencil_batch_64_uneven_grids_matches_oracle():
    """64 grids, sides log-uniform in [16, 160] per axis, one persistent launch."""
    sides = inputs.batch_sides(64, seed=inputs.SEED_BATCH)
    grids, host = _stencil_batch(sides, 7000)
    ws = _ws(len(grids))
    plan = binding.acs_batch_prepare(binding.KIND_STENCIL, grids, ws)
    binding.acs_batch_launch(plan)
    torch.cuda.synchronize()
    for (u, a), (_, _, out) in zip(host, grids):
        assert_parity(out.cpu().numpy(), oracle.stencil(u, a, threads=8), what=f"batch grid {u.shape}")


@pytest.mark.parametrize("tile", [None, (32, 4, 4), (16, 16, 32), (64, 8, 8)])
def test_stencil_batch_tiles(tile):
    sides = [(5, 3, 2), (40, 17, 9), (1, 1, 1), (33, 70, 12), (64, 8, 30)]
    grids, host = _stencil_batch(sides, 7100)
    plan = binding.acs_batch_prepare(binding.KIND_STENCIL, grids, _ws(len(grids)), tile=tile)
    binding.acs_batch_launch(plan)
    torch.cuda.synchronize()
    for (u, a), (_, _, out) in zip(host, grids):
        assert_parity(out.cpu().numpy(), oracle.stencil(u, a), what=f"batch {tile} grid {u.shape}")


@pytest.mark.parametrize("h", [(1.0, 0.5, 2.0), (0.37, 0.37, 0.37)])   # three scales / folded into the fluxes
@pytest.mark.parametrize("tile", [None, (16, 8, 4), (32, 16, 8)])
def test_rhs_batch_matches_oracle(tile, h):
    rng = np.random.default_rng(11)
    sides = rng.integers(1, 60, size=(10, 3))
    grids, host = [], []
    for q, (nx, ny, nz) in enumerate(sides):
        U = inputs.rhs_field(int(nx), int(ny), int(nz), halo=2, seed=7200 + q)
        R = torch.full((5, int(nz), int(ny), int(nx)), float("nan"), dtype=torch.float64, device="cuda")
        grids.append((to_dev(U), None, R))
        host.append(U)
    params = {"gamma": 1.4, "eps": 0.25, "h": h}
    plan = binding.acs_batch_prepare(binding.KIND_RHS, grids, _ws(len(grids)), tile=tile)
    binding.acs_batch_launch(plan, params)
    torch.cuda.synchronize()
    for U, (_, _, R) in zip(host, grids):
        assert_parity(R.cpu().numpy(), oracle.rhs(U, h=h), what=f"rhs batch {U.shape} h={h}")


def _guided_units(sides, bx, by, kchunk, per_sm):
    """Unit count of a batch plan: grids largest first; the last grids whose units (in chunks
    of kchunk // 4) fit in two waves of resident blocks take the short chunks."""
    waves = 2 * torch.cuda.get_device_properties(0).multi_processor_count * per_sm
    order = sorted(range(len(sides)), key=lambda q: -int(np.prod(sides[q])))   # stable, largest first
    tail_kc = max(1, kchunk // 4)

    def units(q, kc):
        nx, ny, nz = (int(v) for v in sides[q])
        return -(-nx // bx) * -(-ny // by) * -(-nz // kc)

    kcs = {q: kchunk for q in order}
    acc = 0
    for q in reversed(order):
        acc += units(q, tail_kc)
        if acc > waves:
            break
        kcs[q] = tail_kc
    return sum(units(q, kcs[q]) for q in order)


def test_rhs_batch_guided_chunks_head_and_tail():
    """Twelve 64^3 grids (units of 16 planes, the queue's head) and twenty small grids (the
    tail, units of 4 planes): parity with the oracle and the plan's unit count."""
    sides = [(64, 64, 64)] * 12 + [(int(a), int(b), int(c)) for a, b, c in
                                   inputs.batch_sides(20, seed=inputs.SEED_BATCH + 20, lo=8, hi=40)]
    grids, host = [], []
    for q, (nx, ny, nz) in enumerate(sides):
        U = inputs.rhs_field(nx, ny, nz, halo=2, seed=7700 + q)
        grids.append((to_dev(U), None, torch.full((5, nz, ny, nx), float("nan"), dtype=torch.float64,
                                                  device="cuda")))
        host.append(U)
    plan = binding.acs_batch_prepare(binding.KIND_RHS, grids, _ws(len(grids)), tile=(16, 16, 16))
    assert plan.total_units == _guided_units(sides, 16, 16, 16, per_sm=2)
    assert plan.total_units > 12 * 16 * 4            # some grids keep 16-plane units
    binding.acs_batch_launch(plan)
    torch.cuda.synchronize()
    for U, (_, _, R) in zip(host, grids):
        assert_parity(R.cpu().numpy(), oracle.rhs(U, threads=8), what=f"rhs guided batch {U.shape}")


def test_batch_in_cuda_graph_replays():
    """Capture acs_batch_launch once; replay after changing the inputs in place."""
    sides = inputs.batch_sides(12, seed=inputs.SEED_BATCH + 1)
    grids, host = _stencil_batch(sides, 7300)
    ws = _ws(len(grids))
    plan = binding.acs_batch_prepare(binding.KIND_STENCIL, grids, ws)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        binding.acs_batch_launch(plan, stream=s)            # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        binding.acs_batch_launch(plan, stream=torch.cuda.current_stream())
    for rep in range(3):
        for q, (u_d, a_d, out) in enumerate(grids):
            u_new = host[q][0] * (1.0 + 0.5 * rep)
            u_d.copy_(torch.from_numpy(u_new))
            out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for q, (u_d, a_d, out) in enumerate(grids):
            u_new = host[q][0] * (1.0 + 0.5 * rep)
            assert_parity(out.cpu().numpy(), oracle.stencil(u_new, host[q][1]), what=f"replay {rep} grid {q}")


def test_batch_workspace_errors():
    grids, _ = _stencil_batch([(8, 8, 8), (9, 9, 9)], 7400)
    small = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.AcsError) as ei:
        binding.acs_batch_prepare(binding.KIND_STENCIL, grids, small)
    assert ei.value.name == "ACS_ERR_WORKSPACE"
    ws = _ws(2)
    mis = ws.view(torch.uint8)[8:]
    with pytest.raises(binding.AcsError) as ei:
        binding.acs_batch_prepare(binding.KIND_STENCIL, grids, mis)
    assert ei.value.name == "ACS_ERR_ALIGN"
    with pytest.raises(binding.AcsError) as ei:
        binding.acs_batch_prepare(binding.KIND_STENCIL, grids, ws, tile=(48, 8, 8))
    assert ei.value.name == "ACS_ERR_UNSUPPORTED"


def test_autotune_single_grid_and_cache_roundtrip(tmp_path):
    binding.acs_tune_cache_clear()
    u, a = inputs.stencil_fields(64, 48, 40, seed=7500)
    ud, ad = to_dev(u), to_dev(a)
    out = torch.empty((40, 48, 64), dtype=torch.float64, device="cuda")
    tile, ms = binding.acs_autotune_stencil(ud, ad, out)
    assert tile[0] in (16, 32, 64) and tile[1] in (4, 8, 16) and ms > 0
    assert tile[2] >= 1 or tile[3] & binding.TILE_BALANCED
    U = inputs.rhs_field(40, 36, 30, halo=2, seed=7501)
    Ud = to_dev(U)
    R = torch.empty((5, 30, 36, 40), dtype=torch.float64, device="cuda")
    rtile, rms = binding.acs_autotune_rhs(Ud, R)
    assert rtile[0] in (16, 32, 64) and rms > 0
    assert binding.acs_tune_cache_size() == 2
    # a NULL-tile call now runs with the tuned shape; results still match the oracle
    out.fill_(float("nan"))
    binding.acs_stencil_saturated(ud, ad, out)
    R.fill_(float("nan"))
    binding.acs_rhs_saturated(Ud, R)
    torch.cuda.synchronize()
    assert_parity(out.cpu().numpy(), oracle.stencil(u, a), what="tuned stencil")
    assert_parity(R.cpu().numpy(), oracle.rhs(U), what="tuned rhs")
    path = str(tmp_path / "tune.txt")
    binding.acs_tune_cache_save(path)
    binding.acs_tune_cache_clear()
    assert binding.acs_tune_cache_size() == 0
    binding.acs_tune_cache_load(path)
    assert binding.acs_tune_cache_size() == 2
    with open(path) as f:
        assert f.readline().startswith("acs-tune-cache 2")
    # version-1 files (no flags column) still load
    v1 = tmp_path / "v1.txt"
    v1.write_text("acs-tune-cache 1\n32 8 16 1.0 1:8x8x8;\n")
    binding.acs_tune_cache_load(str(v1))
    assert binding.acs_tune_cache_size() == 3
    for text in ("acs-tune-cache 1\n48 8 8 1.0 1:8x8x8;\n",          # unbuilt tile
                 "acs-tune-cache 2\n32 8 0 1 1.0 3:8x8x8;\n",        # balanced schedule for a batch
                 "acs-tune-cache 2\n32 8 8 1 1.0 1:8x8x8;\n",        # balanced with a z-chunk
                 "acs-tune-cache 2\n32 8 8 4 1.0 1:8x8x8;\n",        # unknown flag
                 "acs-tune-cache 2\n32 8 8 2 1.0 2:8x8x8;\n",        # TMA staging for a batch
                 "acs-tune-cache 3\n"):
        bad = tmp_path / "bad.txt"
        bad.write_text(text)
        with pytest.raises(binding.AcsError):
            binding.acs_tune_cache_load(str(bad))
    binding.acs_tune_cache_clear()


def test_autotune_batch_picks_a_working_tile():
    sides = inputs.batch_sides(16, seed=inputs.SEED_BATCH + 2)
    grids, host = _stencil_batch(sides, 7600)
    ws = _ws(len(grids))
    tile, ms = binding.acs_autotune_batch(binding.KIND_STENCIL, grids, ws)
    assert ms > 0
    plan = binding.acs_batch_prepare(binding.KIND_STENCIL, grids, ws, tile=tile)
    for (_, _, out) in grids:
        out.fill_(float("nan"))
    binding.acs_batch_launch(plan)
    torch.cuda.synchronize()
    for (u, a), (_, _, out) in zip(host, grids):
        assert_parity(out.cpu().numpy(), oracle.stencil(u, a), what=f"tuned batch {u.shape}")
    binding.acs_tune_cache_clear()


def _padded(arr, pitch):
    """Device view of `arr` whose rows sit in a buffer of row pitch `pitch` (elements)."""
    v = inputs.pad_rows(arr, pitch)
    return torch.from_numpy(v.base).cuda()[..., :arr.shape[-1]]


@pytest.mark.parametrize("tile", [(16, 8, 8, binding.TILE_TMA), (32, 8, 16, binding.TILE_TMA),
                                  (16, 16, 4, binding.TILE_TMA)])
def test_stencil_batch_tma_mixed_layouts(tile):
    """A star-stencil batch with TMA staging: grids of even row pitch are copied by tensor
    copies, the odd-pitch ones element-wise, a padded one (odd side, even pitch) by tensor
    copies; every grid matches the oracle, its halo is untouched and no bounded wait ran out.
    The same plan replayed from a CUDA graph gives the same bits."""
    sides = [(40, 17, 9), (33, 70, 12), (64, 8, 30), (20, 20, 20), (5, 3, 2), (16, 24, 7), (31, 9, 15)]
    grids, host = [], []
    for q, (nx, ny, nz) in enumerate(sides):
        u, a = inputs.stencil_fields(nx, ny, nz, halo=4, seed=7400 + q)
        out = torch.full((nz + 2, ny, nx), float("nan"), dtype=torch.float64, device="cuda")
        if q == len(sides) - 1:                     # odd side, rows padded to an even pitch
            ud, ad = _padded(u, nx + 9), _padded(a, nx + 9)
        else:
            ud, ad = to_dev(u), to_dev(a)
        grids.append((ud, ad, out[1:-1]))
        host.append((u, a, out))
    plan = binding.acs_batch_prepare(binding.KIND_STENCIL, grids, _ws(len(grids)), tile=tile)
    binding.acs_batch_launch(plan)
    torch.cuda.synchronize()
    first = []
    for (u, a, out) in host:
        o = out.cpu().numpy()
        assert np.isnan(o[0]).all() and np.isnan(o[-1]).all()
        assert_parity(o[1:-1], oracle.stencil(u, a), what=f"TMA batch {tile} grid {u.shape}")
        first.append(o.copy())
    assert binding.acs_wait_timeouts() == 0
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        binding.acs_batch_launch(plan, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        binding.acs_batch_launch(plan, stream=torch.cuda.current_stream())
    for (_, _, out) in host:
        out[1:-1].fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    for (_, _, out), o in zip(host, first):
        assert np.array_equal(out.cpu().numpy()[1:-1], o[1:-1])
    assert binding.acs_wait_timeouts() == 0


def test_batch_tma_flag_rules():
    sides = [(8, 8, 4)]
    grids, _ = _stencil_batch(sides, 7500)
    U = to_dev(inputs.rhs_field(8, 8, 4, halo=2, seed=7501))
    R = torch.empty((5, 4, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.AcsError) as ei:            # RHS batches stage element-wise only
        binding.acs_batch_prepare(binding.KIND_RHS, [(U, None, R)], _ws(1), tile=(32, 8, 8, binding.TILE_TMA))
    assert ei.value.name == "ACS_ERR_UNSUPPORTED"
    with pytest.raises(binding.AcsError) as ei:            # balanced has no meaning in a batch
        binding.acs_batch_prepare(binding.KIND_STENCIL, grids, _ws(1), tile=(32, 8, 8, binding.TILE_BALANCED))
    assert ei.value.name == "ACS_ERR_INVALID"
    with pytest.raises(binding.AcsError):                  # the static entry point stages element-wise
        binding.acs_batch_run_static(binding.KIND_STENCIL, grids, tile=(32, 8, 8, binding.TILE_TMA))
