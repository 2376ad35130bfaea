"""GPU tests of rewriter variants (NVRTC-compiled) and the learned ranker."""
import numpy as np
import pytest

import oracle
from paper_2306_13002_gb300 import binding, inputs, ranker
from _mlp_ref import np_forward as _np_forward, np_grad as _np_grad, small_problem as _small_problem, unpack as _unpack
from _parity import assert_parity, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_compiled_variants_match_oracle():
    """Per-iteration variants from random rule orders, compiled at run time, all compute the
    as-written RHS."""
    vs = ranker.compile_all(ranker.generate(12, seed=inputs.SEED_VARIANTS, scope=binding.SCOPE_ITERATION))
    h = (1.0, 0.5, 2.0)
    U = inputs.rhs_field(37, 21, 13, halo=2, seed=8100)
    ref = oracle.rhs(U, h=h)
    Ud = to_dev(U)
    for v in vs:
        R = torch.full((5, 13, 21, 37), float("nan"), dtype=torch.float64, device="cuda")
        v["module"].launch(Ud, R, h=h)
        torch.cuda.synchronize()
        assert v["module"].regs > 0
        assert_parity(R.cpu().numpy(), ref, what=f"variant {v['index']}")
        v["module"].close()


# The march-scope variants the bench's ranker block ranks (seed and count as in bench.py).
N_BENCH_VARIANTS = 512


@pytest.fixture(scope="module")
def march_variants():
    vs = ranker.compile_all(ranker.distinct(ranker.generate(N_BENCH_VARIANTS, seed=inputs.SEED_VARIANTS)))
    yield vs
    for v in vs:
        v["module"].close()


def test_every_ranked_march_variant_matches_oracle_ragged(march_variants):
    """Every distinct march variant of the bench's study, on a ragged grid (tiles cut on x and y,
    z-chunks cut), anisotropic spacing: within the parity tolerance of the oracle, and its halo
    untouched."""
    h = (1.0, 0.5, 2.0)
    nx, ny, nz = 38, 21, 13                         # even nx: TMA-staged variants can copy the layout
    U = inputs.rhs_field(nx, ny, nz, halo=2, seed=8200)
    ref = oracle.rhs(U, h=h)
    Ud = to_dev(U)
    kinds = set()
    for v in march_variants:
        R = torch.full((5, nz + 2, ny, nx), float("nan"), dtype=torch.float64, device="cuda")
        binding.acs_rhs_saturated(Ud, R[:, 1:-1], h=h, variant=v["module"])
        torch.cuda.synchronize()
        out = R.cpu().numpy()
        assert np.isnan(out[:, 0]).all() and np.isnan(out[:, -1]).all(), v["index"]
        assert_parity(out[:, 1:-1], ref, what=f"march variant {v['index']}")
        kinds.add((v["block"], v["flags"]))
    assert binding.acs_wait_timeouts() == 0
    assert len(kinds) >= 12                          # tiles x stagings x schedules all exercised


def test_every_ranked_march_variant_matches_oracle_at_162(march_variants):
    """The NPB class C side: every distinct march variant of the bench's study against the oracle
    over the whole 162^3 field (compared on the GPU)."""
    n = 162
    U = inputs.rhs_field(n, halo=2, seed=inputs.SEED_RHS_LARGE)
    ref = torch.from_numpy(oracle.rhs(U)).cuda()
    Ud = to_dev(U)
    R = torch.empty((5, n, n, n), dtype=torch.float64, device="cuda")
    tol = 1e-12 * ref.abs() + 1e-14
    for v in march_variants:
        R.fill_(float("nan"))
        binding.acs_rhs_saturated(Ud, R, variant=v["module"])
        bad = int(((R - ref).abs() > tol).sum()) + int(torch.isnan(R).sum())
        assert bad == 0, (v["index"], bad)


def test_march_variant_layout_and_argument_checks(march_variants):
    tma = next(v for v in march_variants if v["flags"] & binding.TILE_TMA)
    plain = next(v for v in march_variants if not v["flags"] & binding.TILE_TMA)
    U = inputs.rhs_field(37, 20, 9, halo=2, seed=8300)          # odd row pitch: no TMA copy of it
    ref = oracle.rhs(U)
    Ud = to_dev(U)
    R = torch.full((5, 9, 20, 37), float("nan"), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.AcsError) as ei:
        binding.acs_rhs_saturated(Ud, R, variant=tma["module"])
    assert ei.value.name == "ACS_ERR_UNSUPPORTED"
    binding.acs_rhs_saturated(Ud, R, variant=plain["module"])
    torch.cuda.synchronize()
    assert_parity(R.cpu().numpy(), ref, what="element-wise staged march variant, odd pitch")
    # the tile must be the variant's own (kchunk free)
    bx, by = plain["block"]
    binding.acs_rhs_saturated(Ud, R, tile=(bx, by, 3, plain["flags"]), variant=plain["module"])
    with pytest.raises(binding.AcsError):
        binding.acs_rhs_saturated(Ud, R, tile=(bx, by, 0, plain["flags"] ^ binding.TILE_BALANCED),
                                  variant=plain["module"])
    # per-iteration variants are not saturated kernels
    src, _, info = binding.acs_variant_generate(inputs.SEED_VARIANTS, 3, binding.SCOPE_ITERATION)
    it = binding.Variant(src, info)
    with pytest.raises(binding.AcsError) as ei:
        binding.acs_rhs_saturated(Ud, R, variant=it)
    assert ei.value.name == "ACS_ERR_INVALID"
    it.close()


def test_variant_build_reports_compile_errors():
    info = binding.acs_variant_generate(1, 1, binding.SCOPE_ITERATION)[2]
    with pytest.raises(binding.AcsError) as ei:
        binding.Variant("this is not CUDA", info)
    assert ei.value.name in ("ACS_ERR_INVALID", "ACS_ERR_UNSUPPORTED")
    info.block_x = 48
    with pytest.raises(binding.AcsError):
        binding.Variant(binding.acs_variant_generate(1, 1, binding.SCOPE_ITERATION)[0], info)


def test_ranker_learns_a_synthetic_cost():
    """Times that are a smooth function of the features are ranked well on held-out rows."""
    rng = np.random.default_rng(21)
    n, F = 300, 16
    X = rng.uniform(0, 10, size=(n, F)).astype(np.float32)
    t = np.exp(0.08 * X[:, 1] + 0.15 * X[:, 4] - 0.05 * X[:, 3] + 0.02 * X[:, 1] * X[:, 4] / 10).astype(np.float32)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    tr, te = slice(0, 220), slice(220, n)
    params = torch.empty(binding.acs_ranker_param_count(F, 64), dtype=torch.float32, device="cuda")
    ws = torch.empty(binding.acs_ranker_workspace_bytes(220, F, 64) // 4 + 4, dtype=torch.float32, device="cuda")
    binding.acs_ranker_train(Xd[tr].contiguous(), td[tr].contiguous(), params, ws, epochs=1500, lr=3e-3, seed=5)
    order, pred = binding.acs_variant_rank(Xd[te].contiguous(), params)
    assert ranker.spearman(pred, t[te]) > 0.9
    assert sorted(order) == list(range(n - 220))
    assert all(pred[order[i]] <= pred[order[i + 1]] for i in range(len(order) - 1))
    # deterministic for a given seed
    params2 = torch.empty_like(params)
    binding.acs_ranker_train(Xd[tr].contiguous(), td[tr].contiguous(), params2, ws, epochs=1500, lr=3e-3, seed=5)
    torch.cuda.synchronize()
    assert torch.equal(params, params2)


def test_analytical_rank_orders_by_paper_cost():
    vs = ranker.generate(20, seed=inputs.SEED_VARIANTS)
    X = torch.from_numpy(np.stack([v["feats"] for v in vs])).cuda()
    order, score = binding.acs_variant_rank(X, None)
    costs = [v["cost"] for v in vs]
    assert [costs[i] for i in order] == sorted(costs)
    assert score == pytest.approx(costs)


def test_rank_rejects_mismatched_model():
    X = torch.zeros((4, 20), dtype=torch.float32, device="cuda")
    params = torch.zeros(binding.acs_ranker_param_count(8, 64), dtype=torch.float32, device="cuda")
    import ctypes
    model = binding.RankerModel(8, 64, params.data_ptr())
    order = (ctypes.c_int * 4)()
    sd = torch.empty(4, dtype=torch.float32, device="cuda")
    st = binding.lib().acs_variant_rank(X.data_ptr(), 4, 20, ctypes.byref(model), sd.data_ptr(), order, None, None)
    assert st == 6                                   # ACS_ERR_NOMODEL


def test_small_study_end_to_end():
    """The whole pipeline on 64 march variants at 64^3: distinct variants only, split without
    duplicates, every variant consistent with the library's saturated kernel, and the MLP's pick
    among the held-out variants within 15 % of the best of them (the bench reports the 256^3 study)."""
    res = ranker.study(n_variants=64, n=64, epochs=1500, reps=3, extra_splits=3, search_candidates=48)
    assert res["variants_distinct"] >= 56 and res["train"] + res["test"] == res["variants_distinct"]
    sp = res["splits"]
    assert sp["n"] == 3 and 0 <= sp["mlp_pick_within_5pct_of_best"] <= 3
    assert 1.0 <= sp["mlp_pick_over_best_mean"] <= sp["mlp_pick_over_best_worst"]
    assert 1.0 <= sp["mlp_top3_measured_over_best_worst"] <= sp["mlp_pick_over_best_worst"]
    assert 1.0 <= res["mlp_top3_measured_over_best"] <= res["mlp_pick_over_best"]
    se = res["search"]   # the model ranks 48 further variants, compiles its shortlist, times the first 8
    assert se["candidates"] == 48 and 1 <= se["timed"] <= 8 and se["timed"] <= se["shortlist"] <= se["distinct_new"]
    assert se["best_ms"] == pytest.approx(min(se["timed_ms"]), abs=1e-4) and se["best_index"] >= 64
    assert se["max_err_over_tol_vs_saturated"] <= 2.0
    assert res["max_err_over_tol_vs_saturated"] <= 2.0
    assert res["best_test_ms"] > 0
    assert res["mlp_pick_over_best"] <= 1.15, res
    assert res["spearman_mlp_test"] > 0.5, res


# ------------------------------------------------------------------ numerical reference of the MLP

FW = 1.0   # the loss weighting the study uses


def _train(X, T, H, epochs, lr=1e-2, seed=3):
    n, F = X.shape
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    params = torch.empty(binding.acs_ranker_param_count(F, H), dtype=torch.float32, device="cuda")
    ws = torch.empty(binding.acs_ranker_workspace_bytes(n, F, H) // 4 + 4, dtype=torch.float32, device="cuda")
    binding.acs_ranker_train(Xd, Td, params, ws, hidden=H, epochs=epochs, lr=lr, seed=seed, fast_weight=FW)
    torch.cuda.synchronize()
    return params, Xd, Td, ws


def test_forward_gradient_and_adam_match_float64_reference():
    """acs_variant_rank (forward), acs_ranker_gradient and two Adam epochs of acs_ranker_train
    against the float64 reference above, at FP32 tolerances: forward 1e-5 relative, gradient
    1e-4 of the largest component, updates 1e-3 of the step size."""
    X, T, H = _small_problem()
    n, F = X.shape
    lr = 1e-2
    p0, Xd, Td, ws = _train(X, T, H, epochs=0, lr=lr)
    P0 = _unpack(p0.cpu().numpy(), F, H)
    # the initial model: statistics of the training set
    assert np.allclose(P0["mu"], X.astype(np.float64).mean(0), rtol=1e-6, atol=1e-6)
    assert np.isclose(P0["tmu"], np.log(T.astype(np.float64)).mean(), rtol=1e-6)
    # forward: predicted ms = exp(y tsd + tmu)
    _, pred = binding.acs_variant_rank(Xd, p0, hidden=H)
    y = _np_forward(P0, X.astype(np.float64))[3]
    ref_ms = np.exp(y * P0["tsd"] + P0["tmu"])
    assert np.allclose(pred, ref_ms, rtol=1e-5)
    # gradient at p0
    g0 = torch.empty_like(p0)
    binding.acs_ranker_gradient(Xd, Td, p0, g0, ws, hidden=H, fast_weight=FW)
    g0n = g0.cpu().numpy().astype(np.float64)
    gref = _np_grad(P0, X.astype(np.float64), T.astype(np.float64), FW)
    assert np.abs(gref).max() > 1e-3
    assert np.allclose(g0n, gref, rtol=1e-3, atol=1e-4 * np.abs(gref).max())
    # one Adam epoch: m = (1-b1) g, v = (1-b2) g^2, bias-corrected step lr * g / (|g| + 1e-8)
    b1, b2, e8 = 0.9, 0.999, 1e-8
    p1, _, _, _ = _train(X, T, H, epochs=1, lr=lr)
    p1n = p1.cpu().numpy().astype(np.float64)
    flat0 = p0.cpu().numpy().astype(np.float64)
    m = (1 - b1) * g0n
    v = (1 - b2) * g0n ** 2
    exp1 = flat0 - lr * (m / (1 - b1)) / (np.sqrt(v / (1 - b2)) + e8)
    assert np.allclose(p1n, exp1, rtol=0, atol=1e-3 * lr)
    assert np.abs(p1n - flat0).max() > 0.5 * lr          # the step happened
    assert np.array_equal(p1n[:2 * F + 2], flat0[:2 * F + 2])   # statistics are not trained
    # second epoch: the moments carry over, bias correction with step 2
    g1 = torch.empty_like(p1)
    binding.acs_ranker_gradient(Xd, Td, p1, g1, ws, hidden=H, fast_weight=FW)
    g1n = g1.cpu().numpy().astype(np.float64)
    assert np.allclose(g1n, _np_grad(_unpack(p1n, F, H), X.astype(np.float64), T.astype(np.float64), FW),
                       rtol=1e-3, atol=1e-4 * np.abs(gref).max())
    m = b1 * m + (1 - b1) * g1n
    v = b2 * v + (1 - b2) * g1n ** 2
    exp2 = p1n - lr * (m / (1 - b1 ** 2)) / (np.sqrt(v / (1 - b2 ** 2)) + e8)
    p2, _, _, _ = _train(X, T, H, epochs=2, lr=lr)
    assert np.allclose(p2.cpu().numpy().astype(np.float64), exp2, rtol=0, atol=2e-3 * lr)


def test_model_save_and_load_round_trip(tmp_path):
    X, T, H = _small_problem()
    n, F = X.shape
    p, Xd, _, _ = _train(X, T, H, epochs=20)
    path = tmp_path / "ranker.model"
    binding.acs_ranker_save(str(path), p, F, H)
    q, F2, H2 = binding.acs_ranker_load(str(path))
    assert (F2, H2) == (F, H)
    assert torch.equal(p, q)                                   # same bits
    assert binding.acs_variant_rank(Xd, q, hidden=H) == binding.acs_variant_rank(Xd, p, hidden=H)
    small = torch.empty(q.numel() - 1, dtype=torch.float32, device="cuda")
    assert binding.lib().acs_ranker_load(str(path).encode(), small.data_ptr(), small.numel(), None, None) == 8


@pytest.mark.parametrize("shape", [(1, 1, 1), (17, 1, 3), (2, 40, 1), (16, 16, 2), (33, 9, 1)])
def test_march_variants_on_degenerate_grids(shape, march_variants):
    """One of each staging x schedule among the bench's march variants, on grids of one plane,
    one row, one point: within the parity tolerance of the oracle (element-wise staged variants
    also where the pitch is odd; TMA variants where the layout allows them)."""
    nx, ny, nz = shape
    U = inputs.rhs_field(nx, ny, nz, halo=2, seed=8400 + nx + 7 * ny + 31 * nz)
    ref = oracle.rhs(U)
    Ud = to_dev(U)
    seen = set()
    for v in march_variants:
        key = v["flags"]
        if key in seen:
            continue
        if (v["flags"] & binding.TILE_TMA) and (nx + 4) % 2:
            continue                                  # odd pitch: TMA variants refuse it
        seen.add(key)
        R = torch.full((5, nz, ny, nx), float("nan"), dtype=torch.float64, device="cuda")
        binding.acs_rhs_saturated(Ud, R, variant=v["module"])
        torch.cuda.synchronize()
        assert_parity(R.cpu().numpy(), ref, what=f"march variant {v['index']} on {shape}")
    assert len(seen) >= (2 if (nx + 4) % 2 else 4)
    assert binding.acs_wait_timeouts() == 0
