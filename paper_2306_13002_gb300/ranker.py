"""Rewriter variants and the learned ranker: generation, compilation, timing, training, ranking.

The pipeline the paper's extraction step stands for, with a learned cost in place of the
fixed one: the host rewriter (`acs_variant_generate`) produces N equivalent programs of the
RHS body from random rule orders; each is compiled with NVRTC and timed on the GPU; an FP32
MLP (`acs_ranker_train`, hand-written CUDA kernels) learns time from static features on a
training split; `acs_variant_rank` orders the held-out variants by the model and, for
comparison, by the paper's analytical cost (Sec. V-B).
"""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np

from . import binding, inputs


def spearman(a, b) -> float:
    """Spearman rank correlation with average ranks for ties."""
    def ranks(x):
        x = np.asarray(x, dtype=np.float64)
        order = np.argsort(x, kind="mergesort")
        r = np.empty(len(x))
        r[order] = np.arange(len(x), dtype=np.float64)
        for v in np.unique(x):                      # average ranks of ties
            idx = np.where(x == v)[0]
            if len(idx) > 1:
                r[idx] = r[idx].mean()
        return r
    ra, rb = ranks(a), ranks(b)
    ra -= ra.mean()
    rb -= rb.mean()
    den = np.sqrt((ra * ra).sum() * (rb * rb).sum())
    return float((ra * rb).sum() / den) if den > 0 else 0.0


def _one(seed: int, i: int, scope: int) -> dict:
    src, dag, info = binding.acs_variant_generate(seed, i, scope)
    return {"index": i, "src": src, "dag": dag, "info": info,
            "feats": np.array(info.feats[:], dtype=np.float32), "cost": info.cost,
            "block": (info.block_x, info.block_y), "flags": info.flags, "enodes": info.enodes,
            "iterations": info.iterations}


def generate(n: int, seed: int = inputs.SEED_VARIANTS, scope: int = binding.SCOPE_MARCH, start: int = 0,
             threads: int | None = None):
    """Host rewriter output for variants start..start+n-1 of `scope`: list of dicts (src, dag,
    feats, ...) in index order. Generation is host code with no shared state, run on `threads`
    threads (the library call releases the interpreter lock)."""
    threads = threads or min(16, os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(lambda i: _one(seed, i, scope), range(start, start + n)))


def distinct(variants):
    """The variants whose generated source is new (the first of each identical group): identical
    sources have identical features and run the same code, so they must not be split between the
    training and the test set."""
    seen, out = set(), []
    for v in variants:
        if v["src"] not in seen:
            seen.add(v["src"])
            out.append(v)
    return out


def compile_all(variants, threads: int | None = None):
    """NVRTC-compile every variant in parallel; fills v['module'] and the register feature."""
    threads = threads or min(16, os.cpu_count() or 4)

    def build(v):
        return binding.Variant(v["src"], v["info"])

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        mods = list(ex.map(build, variants))
    reg_idx = binding.acs_variant_feature_names().index("regs")
    for v, m in zip(variants, mods):
        v["module"] = m
        v["feats"][reg_idx] = float(m.regs)
    return variants


def time_all(variants, U, R, reps: int = 5, stream=None):
    """Mean CUDA-event time (ms) of each variant over `reps` launches after one warm-up."""
    import torch
    s = stream or torch.cuda.current_stream()
    for v in variants:
        m = v["module"]
        m.launch(U, R, stream=s)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(reps):
            m.launch(U, R, stream=s)
        b.record(s)
        b.synchronize()
        v["ms"] = a.elapsed_time(b) / reps
    return variants


def max_err_over_tol(R, ref, tol=None) -> float:
    """max |R - ref| / (1e-12 |ref| + 1e-14) over all points (<= 1: within the parity tolerance);
    `tol` may hold that denominator, precomputed once for many R."""
    if tol is None:
        tol = 1e-12 * ref.abs() + 1e-14
    return float((R - ref).abs_().div_(tol).max())


def search(params, hidden: int, start: int, count: int, U, R, regs_fill: float, known: set | None = None,
           seed: int = inputs.SEED_VARIANTS, shortlist: int = 64, timed: int = 8, reps: int = 3) -> dict:
    """The trained MLP as the cost model of a wider search: rewriter variants start..start+count-1
    (march scope) are generated on the host and ranked without compiling them (their register
    count, known only after compilation, set to `regs_fill`); the first `shortlist` are compiled,
    re-ranked with their real register counts, and the first `timed` of those timed at U's size
    and checked against the library's saturated kernel. `known` holds sources already measured
    (skipped). Returns the timed candidates and the fastest."""
    import torch
    vs = [v for v in distinct(generate(count, seed, binding.SCOPE_MARCH, start=start))
          if not known or v["src"] not in known]
    reg_idx = binding.acs_variant_feature_names().index("regs")
    for v in vs:
        v["feats"][reg_idx] = regs_fill
    X = torch.from_numpy(np.stack([v["feats"] for v in vs])).cuda()
    order, _ = binding.acs_variant_rank(X, params, hidden)
    short = [vs[i] for i in order[:shortlist]]
    compile_all(short)
    X2 = torch.from_numpy(np.stack([v["feats"] for v in short])).cuda()
    order2, pred2 = binding.acs_variant_rank(X2, params, hidden)
    top = [short[i] for i in order2[:timed]]
    for v in short:
        if not any(v is t for t in top):
            v["module"].close()
    time_all(top, U, R, reps=reps)
    ref = torch.empty_like(R)
    binding.acs_rhs_saturated(U, ref)
    tol = ref.abs().mul_(1e-12).add_(1e-14)
    worst = 0.0
    for v in top:
        R.fill_(float("nan"))
        v["module"].launch(U, R)
        worst = max(worst, max_err_over_tol(R, ref, tol))
        v["module"].close()
    del ref, tol
    best = min(top, key=lambda v: v["ms"])
    return {"candidates": count, "distinct_new": len(vs), "shortlist": len(short), "timed": len(top),
            "timed_ms": [round(float(v["ms"]), 4) for v in top],
            "predicted_ms_first": float(pred2[order2[0]]),
            "best_index": int(best["index"]), "best_ms": float(best["ms"]),
            "best_shape": [*best["block"], best["flags"]], "max_err_over_tol_vs_saturated": worst}


# Model-guided selection: the MLP's first TOP_K variants are timed and the fastest is kept (the
# study has every variant's time already and reads it off). The MLP's first choice alone is the
# pure model pick; a few timings cover its near-ties and the rare fast variant unlike the
# training set's fast ones.
TOP_K = 3


def study(n_variants: int = 512, n_train: int | None = None, n: int = 256, seed: int = inputs.SEED_VARIANTS,
          hidden: int = 64, epochs: int = 3000, lr: float = 3e-3, reps: int = 5,
          scope: int = binding.SCOPE_MARCH, check: bool = True, fast_weight: float = 1.0,
          extra_splits: int = 0, search_candidates: int = 0) -> dict:
    """Generate `n_variants` variants, keep the distinct ones, compile and time them at n^3, train the
    MLP on a random n_train of them (default: 400/512 of the distinct variants; squared error of the
    standardised log time weighted by exp(-fast_weight t), so the fast variants that decide the
    pick weigh more) and rank the rest, by the MLP and by the paper's analytical cost. With `check`, every variant's output is compared
    with the library's saturated kernel (itself parity-checked against the oracle) at n^3.
    `extra_splits` more random train/test splits (seeds seed + 1 ...) of the same timed variants are
    trained and ranked the same way; their MLP pick / best ratios are summarised in "splits".
    With `search_candidates`, the model trained on the first split then searches that many further
    variants (`search`, indices n_variants onwards); the result is in "search"."""
    import torch
    vs_all = generate(n_variants, seed, scope)
    vs = distinct(vs_all)
    nd = len(vs)
    if n_train is None:
        n_train = int(round(nd * 400 / 512))
    n_train = max(2, min(n_train, nd - 2))
    compile_all(vs)
    U = torch.from_numpy(inputs.rhs_field(n, halo=2, seed=inputs.SEED_RHS_LARGE)).cuda()
    R = torch.empty((5, n, n, n), dtype=torch.float64, device="cuda")
    time_all(vs, U, R, reps=reps)
    worst = None
    if check:
        ref = torch.empty_like(R)
        binding.acs_rhs_saturated(U, ref)
        tol = ref.abs().mul_(1e-12).add_(1e-14)
        worst = 0.0
        for v in vs:
            R.fill_(float("nan"))
            v["module"].launch(U, R)
            worst = max(worst, max_err_over_tol(R, ref, tol))
        del ref, tol
    perm = np.random.default_rng(seed).permutation(nd)
    tr, te = perm[:n_train], perm[n_train:]
    F = len(vs[0]["feats"])
    X = torch.from_numpy(np.stack([v["feats"] for v in vs])).cuda()
    T = torch.tensor([v["ms"] for v in vs], dtype=torch.float32, device="cuda")
    params = torch.empty(binding.acs_ranker_param_count(F, hidden), dtype=torch.float32, device="cuda")
    ws = torch.empty(binding.acs_ranker_workspace_bytes(n_train, F, hidden) // 4 + 4, dtype=torch.float32,
                     device="cuda")
    tri = torch.from_numpy(tr).cuda()
    tei = torch.from_numpy(te).cuda()
    Xtr, Ttr = X[tri].contiguous(), T[tri].contiguous()
    Xte = X[tei].contiguous()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    binding.acs_ranker_train(Xtr, Ttr, params, ws, hidden=hidden, epochs=epochs, lr=lr, seed=seed,
                             fast_weight=fast_weight)
    t1.record()
    torch.cuda.synchronize()
    train_ms = t0.elapsed_time(t1)
    order_m, pred = binding.acs_variant_rank(Xte, params, hidden)
    order_a, cost = binding.acs_variant_rank(Xte, None)
    times_te = np.array([vs[i]["ms"] for i in te])
    _, pred_tr = binding.acs_variant_rank(Xtr, params, hidden)
    times_tr = np.array([vs[i]["ms"] for i in tr])
    best = float(times_te.min())
    pick_m = float(times_te[order_m[0]])
    pick_a = float(times_te[order_a[0]])
    all_ms = np.array([v["ms"] for v in vs])
    found = None
    if search_candidates > 0:
        regs_idx = binding.acs_variant_feature_names().index("regs")
        found = search(params, hidden, n_variants, search_candidates, U, R,
                       float(np.median([v["feats"][regs_idx] for v in vs])), known={v["src"] for v in vs_all},
                       seed=seed)
        found["best_over_study_best"] = found["best_ms"] / float(all_ms.min())
    ratios, ratios_k = [], []
    for sp in range(1, extra_splits + 1):
        p2 = np.random.default_rng(seed + sp).permutation(nd)
        tr2, te2 = p2[:n_train], p2[n_train:]
        i2, j2 = torch.from_numpy(tr2).cuda(), torch.from_numpy(te2).cuda()
        binding.acs_ranker_train(X[i2].contiguous(), T[i2].contiguous(), params, ws, hidden=hidden, epochs=epochs,
                                 lr=lr, seed=seed + sp, fast_weight=fast_weight)
        o2, _ = binding.acs_variant_rank(X[j2].contiguous(), params, hidden)
        t2 = np.array([vs[i]["ms"] for i in te2])
        ratios.append(float(t2[o2[0]] / t2.min()))
        ratios_k.append(float(t2[list(o2[:TOP_K])].min() / t2.min()))
    for v in vs:
        v["module"].close()
    pm, pa, pb = vs[te[order_m[0]]], vs[te[order_a[0]]], vs[te[int(np.argmin(times_te))]]
    return {
        "scope": "march" if scope == binding.SCOPE_MARCH else "iteration",
        "variants_generated": n_variants, "variants_distinct": nd, "train": int(len(tr)), "test": int(len(te)),
        "grid": n, "hidden": hidden, "epochs": epochs, "lr": lr, "fast_weight": fast_weight, "train_ms": train_ms,
        "spearman_mlp_test": spearman(pred, times_te),
        "spearman_mlp_train": spearman(pred_tr, times_tr),
        "spearman_analytical_test": spearman(cost, times_te),
        "best_test_ms": best, "mlp_pick_ms": pick_m, "analytical_pick_ms": pick_a,
        "mlp_pick_over_best": pick_m / best, "analytical_pick_over_best": pick_a / best,
        f"mlp_top{TOP_K}_measured_over_best": float(times_te[list(order_m[:TOP_K])].min()) / best,
        "all_ms_min": float(all_ms.min()), "all_ms_median": float(np.median(all_ms)),
        "all_ms_max": float(all_ms.max()), "max_err_over_tol_vs_saturated": worst,
        "mlp_pick_index": int(pm["index"]), "analytical_pick_index": int(pa["index"]),
        "best_test_index": int(pb["index"]),
        "mlp_pick_shape": [*pm["block"], pm["flags"]],
        "best_all_index": int(vs[int(np.argmin(all_ms))]["index"]),
        "search": found,
        "splits": None if not ratios else {
            "n": len(ratios), "seeds": [seed + 1, seed + len(ratios)],
            "mlp_pick_within_5pct_of_best": int(sum(r <= 1.05 for r in ratios)),
            "mlp_pick_over_best_mean": float(np.mean(ratios)), "mlp_pick_over_best_median": float(np.median(ratios)),
            "mlp_pick_over_best_worst": float(max(ratios)),
            f"mlp_top{TOP_K}_measured_within_5pct_of_best": int(sum(r <= 1.05 for r in ratios_k)),
            f"mlp_top{TOP_K}_measured_over_best_worst": float(max(ratios_k))},
    }


def run_variant(index: int, n: int = 256, reps: int = 10, seed: int = inputs.SEED_VARIANTS,
                scope: int = binding.SCOPE_MARCH) -> dict:
    """Generate, compile and run one variant `reps` times on the n^3 RHS workload (through
    acs_rhs_saturated for a march variant); returns its mean CUDA-event time."""
    import torch
    src, _, info = binding.acs_variant_generate(seed, index, scope)
    v = binding.Variant(src, info)
    U = torch.from_numpy(inputs.rhs_field(n, halo=2, seed=inputs.SEED_RHS_LARGE)).cuda()
    R = torch.empty((5, n, n, n), dtype=torch.float64, device="cuda")
    fn = (lambda: binding.acs_rhs_saturated(U, R, variant=v)) if scope == binding.SCOPE_MARCH else \
        (lambda: v.launch(U, R))
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    b.synchronize()
    out = {"index": index, "grid": n, "ms": a.elapsed_time(b) / reps, "regs": v.regs, "block": list(v.block),
           "flags": v.flags}
    v.close()
    return out


if __name__ == "__main__":
    import argparse
    import json

    from . import build as acs_build
    ap = argparse.ArgumentParser(description="rewriter variants: the ranker study, or one variant's run")
    ap.add_argument("what", choices=["study", "run"])
    ap.add_argument("--index", type=int, default=0, help="run: the variant index")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--variants", type=int, default=512)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--scope", default="march", choices=["march", "iteration"])
    a = ap.parse_args()
    acs_build.build()
    sc = binding.SCOPE_MARCH if a.scope == "march" else binding.SCOPE_ITERATION
    if a.what == "run":
        print(json.dumps(run_variant(a.index, a.n, a.reps, scope=sc)))
    else:
        print(json.dumps(study(n_variants=a.variants, n=a.n, scope=sc)))
