"""GPU tests of rewriter variants (NVRTC-compiled) and the learned ranker."""
import numpy as np
import pytest

import oracle
from paper_2306_13002_gb300 import binding, inputs, ranker
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
