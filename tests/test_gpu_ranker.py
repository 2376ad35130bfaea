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
    """Variants from random rule orders, compiled at run time, all compute the as-written RHS."""
    vs = ranker.compile_all(ranker.generate(12, seed=inputs.SEED_VARIANTS))
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


def test_variant_build_reports_compile_errors():
    with pytest.raises(binding.AcsError) as ei:
        binding.Variant("this is not CUDA", 32)
    assert ei.value.name in ("ACS_ERR_INVALID", "ACS_ERR_UNSUPPORTED")
    with pytest.raises(binding.AcsError):
        binding.Variant(binding.acs_variant_generate(1, 1)[0], 48)


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
    X = torch.zeros((4, 16), dtype=torch.float32, device="cuda")
    params = torch.zeros(binding.acs_ranker_param_count(8, 64), dtype=torch.float32, device="cuda")
    import ctypes
    model = binding.RankerModel(8, 64, params.data_ptr())
    order = (ctypes.c_int * 4)()
    sd = torch.empty(4, dtype=torch.float32, device="cuda")
    st = binding.lib().acs_variant_rank(X.data_ptr(), 4, 16, ctypes.byref(model), sd.data_ptr(), order, None, None)
    assert st == 6                                   # ACS_ERR_NOMODEL


def test_small_study_end_to_end():
    """The whole pipeline on 48 variants at 48^3: timings positive, ranks valid."""
    res = ranker.study(n_variants=48, n_train=36, n=48, epochs=800, reps=2)
    assert res["distinct_sources"] >= 40
    assert res["best_test_ms"] > 0 and res["mlp_pick_over_best"] >= 1.0
    assert res["variant1_vs_accsat_err_over_tol"] <= 1.0
    assert -1.0 <= res["spearman_mlp_test"] <= 1.0


# ------------------------------------------------------------------ numerical reference of the MLP

def _train(X, T, H, epochs, lr=1e-2, seed=3):
    n, F = X.shape
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    params = torch.empty(binding.acs_ranker_param_count(F, H), dtype=torch.float32, device="cuda")
    ws = torch.empty(binding.acs_ranker_workspace_bytes(n, F, H) // 4 + 4, dtype=torch.float32, device="cuda")
    binding.acs_ranker_train(Xd, Td, params, ws, hidden=H, epochs=epochs, lr=lr, seed=seed)
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
    binding.acs_ranker_gradient(Xd, Td, p0, g0, ws, hidden=H)
    g0n = g0.cpu().numpy().astype(np.float64)
    gref = _np_grad(P0, X.astype(np.float64), T.astype(np.float64))
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
    binding.acs_ranker_gradient(Xd, Td, p1, g1, ws, hidden=H)
    g1n = g1.cpu().numpy().astype(np.float64)
    assert np.allclose(g1n, _np_grad(_unpack(p1n, F, H), X.astype(np.float64), T.astype(np.float64)),
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
