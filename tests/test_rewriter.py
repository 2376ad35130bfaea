"""CPU tests of the host rewriter (no GPU): every variant's extracted program equals the
as-written body exactly over the rationals, bulk-load variants load everything before the
first store, the paper's cost model (Sec. V-B) is recomputed by hand from the DAG, and the
output is deterministic per (seed, index)."""
import re
import struct
from fractions import Fraction as Q

import numpy as np
import pytest
from scipy import stats

from oracle import exact
from paper_2306_13002_gb300 import binding, inputs, ranker
from paper_2306_13002_gb300 import build as acs_build


@pytest.fixture(scope="module", autouse=True)
def _lib():
    acs_build.build()
    binding.lib()


# Offsets (di, dj, dk) of the 13 points named in acs.h.
POINTS = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
          (2, 0, 0), (-2, 0, 0), (0, 2, 0), (0, -2, 0), (0, 0, 2), (0, 0, -2)]


def eval_dag(dag: str, U5, params, centre=(0, 0, 0), fluxes=None, tag="R"):
    """Evaluate DAG text exactly. U5: (5, 5, 5, 5) field around the centre (2, 2, 2); loads are
    taken relative to `centre`; flux leaves from `fluxes[(d, side)][(d, s)]`. Returns the
    outputs of the lines starting with `tag` (R: by component; F: by (d, s))."""
    val, outs = {}, {}
    for line in dag.strip().splitlines():
        f = line.split()
        if f[0] in ("R", "F"):
            if f[0] == "R":
                outs[int(f[1])] = val[int(f[2])]
            else:
                outs[(int(f[1]), int(f[2]))] = val[int(f[3])]
            continue
        nid, op, a, b, c, pay = int(f[0]), f[1], int(f[2]), int(f[3]), int(f[4]), int(f[5])
        A, B, C = val.get(a), val.get(b), val.get(c)
        if op == "const":
            v = Q(struct.unpack("<d", struct.pack("<q", pay))[0])
        elif op == "param":
            v = params[pay]
        elif op == "flux":
            d, rem = divmod(pay, 8)
            s1, side = divmod(rem, 2)
            v = fluxes[(d, side)][(d, s1 + 1)]
        elif op == "load":
            comp, t = divmod(pay, 13)
            di, dj, dk = POINTS[t]
            ci, cj, ck = centre
            v = Q(float(U5[comp, 2 + dk + ck, 2 + dj + cj, 2 + di + ci]))
        elif op == "add":
            v = A + B
        elif op == "sub":
            v = A - B
        elif op == "mul":
            v = A * B
        elif op == "div":
            v = A / B
        elif op == "fma":
            v = A * B + C
        elif op == "neg":
            v = -A
        elif op == "rcp":
            v = 1 / A
        else:
            raise AssertionError(op)
        val[nid] = v
    if tag == "R":
        return [outs[c] for c in range(5)]
    return outs


def eval_march(dag: str, U5, params):
    """The march-scope program exactly: the flux program at the six neighbours of the centre,
    then the combine program with those fluxes as its leaves."""
    fsec, csec = dag.split("combine\n")
    assert fsec.startswith("flux\n")
    fsec = fsec[len("flux\n"):]
    for line in fsec.splitlines():                       # the flux program reads its own point only
        f = line.split()
        if f[0] not in ("F",) and f[1] == "load":
            assert int(f[5]) % 13 == 0
    fluxes = {}
    for d in range(3):
        for side in (0, 1):
            off = [0, 0, 0]
            off[d] = 1 if side == 0 else -1
            fluxes[(d, side)] = eval_dag(fsec, U5, params, centre=tuple(off), tag="F")
    return eval_dag(csec, U5, params, fluxes=fluxes)


H = (1.0, 0.5, 2.0)
PARAMS = {0: Q(1.4), 1: Q(0.25), 2: Q(0.5) / Q(H[0]), 3: Q(0.5) / Q(H[1]), 4: Q(0.5) / Q(H[2])}


@pytest.mark.parametrize("index", list(range(0, 24)) + [57, 200, 511])
def test_variant_is_exact_identity_of_as_written(index):
    src, dag, info = binding.acs_variant_generate(inputs.SEED_VARIANTS, index)
    for trial in range(2):
        U5 = inputs.rhs_field(1, halo=2, seed=900 + 7 * index + trial)     # 5 x 5 x 5 x 5
        ref, _ = exact.rhs_point(U5, 0, 0, 0, gamma=1.4, eps=0.25, h=H, halo=2)
        got = eval_dag(dag, U5, PARAMS)
        assert got == ref, (index, trial)


def test_variant_zero_is_plain_cse_and_paper_cost_by_hand():
    src, dag, info = binding.acs_variant_generate(inputs.SEED_VARIANTS, 0)
    names = binding.acs_variant_feature_names()
    f = dict(zip(names, info.feats))
    assert f["n_load"] == 65 and f["n_div"] == 12 and f["n_fma"] == 0
    # Sec. V-B: constants 0, input variables 1, arithmetic 10, memory access / division 100
    ops = [ln.split()[1] for ln in dag.splitlines() if not ln.startswith("R ")]
    cost = sum({"const": 0, "param": 1, "load": 100, "div": 100, "rcp": 100}.get(o, 10) for o in ops)
    assert cost == info.cost == f["paper_cost"]


def test_bulk_variants_load_everything_before_the_first_store():
    seen = {0: 0, 1: 0}
    for index in range(1, 40):
        src, dag, info = binding.acs_variant_generate(inputs.SEED_VARIANTS, index)
        bulk = int(info.feats[binding.acs_variant_feature_names().index("bulk")])
        lines = src.splitlines()
        loads = [i for i, ln in enumerate(lines) if "= U[" in ln]
        stores = [i for i, ln in enumerate(lines) if ln.strip().startswith("Rp[")]
        assert len(loads) == info.feats[binding.acs_variant_feature_names().index("n_load")] == 65
        if bulk:
            assert max(loads) < min(stores)
            # ties at one location are sorted by static index (component, point)
            keys = [tuple(int(x) for x in re.search(r"U\[(\d+) \* a.isc \+ p \+ \((-?\d+)\)", lines[i]).groups())
                    for i in loads]
            assert [k[0] for k in keys] == sorted(k[0] for k in keys)
        else:
            assert max(loads) > min(stores)
        seen[bulk] += 1
    assert seen[0] and seen[1]


def test_generation_is_deterministic_and_diverse():
    a = binding.acs_variant_generate(inputs.SEED_VARIANTS, 7)
    b = binding.acs_variant_generate(inputs.SEED_VARIANTS, 7)
    assert a[0] == b[0] and a[1] == b[1]
    srcs = {binding.acs_variant_generate(inputs.SEED_VARIANTS, i)[0] for i in range(48)}
    assert len(srcs) >= 40
    feats = np.array([binding.acs_variant_generate(inputs.SEED_VARIANTS, i)[2].feats[:] for i in range(48)])
    names = binding.acs_variant_feature_names()
    assert len(set(feats[:, names.index("n_fma")])) > 5
    assert set(feats[:, names.index("n_div")]) >= {12.0, 6.0}
    assert max(binding.acs_variant_generate(inputs.SEED_VARIANTS, i)[2].enodes for i in range(48)) <= 10000 + 64


def test_generate_reports_small_buffers():
    import ctypes
    info = binding.VariantInfo()
    buf = ctypes.create_string_buffer(16)
    st = binding.lib().acs_variant_generate(1, 3, 0, buf, 16, None, 0, ctypes.byref(info))
    assert st == 1 and info.src_bytes > 16
    assert binding.lib().acs_variant_generate(1, -1, 0, None, 0, None, 0, ctypes.byref(info)) == 1
    assert binding.lib().acs_variant_generate(1, 3, 2, None, 0, None, 0, ctypes.byref(info)) == 1     # scope
    st = binding.lib().acs_variant_generate(1, 3, 1, buf, 16, None, 0, ctypes.byref(info))
    assert st == 1 and info.src_bytes > 16


def test_spearman_matches_scipy():
    rng = np.random.default_rng(3)
    for _ in range(5):
        a = rng.normal(size=40)
        b = a + rng.normal(scale=0.7, size=40)
        b[::7] = b[0]                                   # ties
        assert ranker.spearman(a, b) == pytest.approx(stats.spearmanr(a, b).statistic, abs=1e-12)


MARCH = binding.SCOPE_MARCH


@pytest.mark.parametrize("index", list(range(0, 16)) + [40, 77, 200, 311, 511])
def test_march_variant_is_exact_identity_of_as_written(index):
    """Flux program composed with the combine program = the as-written RHS, over the rationals."""
    src, dag, info = binding.acs_variant_generate(inputs.SEED_VARIANTS, index, MARCH)
    assert info.scope == MARCH
    for trial in range(2):
        U5 = inputs.rhs_field(1, halo=2, seed=1900 + 7 * index + trial)
        ref, _ = exact.rhs_point(U5, 0, 0, 0, gamma=1.4, eps=0.25, h=H, halo=2)
        assert eval_march(dag, U5, PARAMS) == ref, (index, trial)


def test_march_variant_zero_shares_the_flux_and_keeps_the_statements():
    """Index 0: hash-consing only. The flux program has the as-written 4 divisions per point
    (3 velocities and the kinetic energy, shared by the 12 flux values), the combine program
    reads 65 loads and the 24 neighbour fluxes, and the default launch shape."""
    src, dag, info = binding.acs_variant_generate(inputs.SEED_VARIANTS, 0, MARCH)
    f = dict(zip(binding.acs_variant_feature_names(), info.feats))
    assert f["n_div"] == 4 and f["n_fma"] == 0 and f["n_load_x"] == 65 and f["n_load_yz"] == 24
    assert (info.block_x, info.block_y, info.flags) == (16, 16, 3)
    fsec = dag.split("combine\n")[0]
    assert sum(1 for ln in fsec.splitlines() if ln.split()[1:2] == ["div"]) == 4
    assert "acs_variant_march" in src and "#define ACS_TMA 1" in src and "#define ACS_BALANCED 1" in src


def test_like_term_collection_reaches_the_reassociated_dissipation():
    """Some march variants with the collection family extract the dissipation as
    S2 - 4 S1 + 18 U: a constant 18 (= 6 + 6 + 6 collected exactly) appears in their combine."""
    eighteen = str(struct.unpack("<q", struct.pack("<d", 18.0))[0])
    found = 0
    for index in range(1, 64):
        dag = binding.acs_variant_generate(inputs.SEED_VARIANTS, index, MARCH)[1]
        csec = dag.split("combine\n")[1]
        if any(ln.split()[1] == "const" and ln.split()[5] == eighteen for ln in csec.splitlines()
               if not ln.startswith("R ")):
            found += 1
    assert found >= 5


def test_march_variants_are_diverse_and_compile_on_the_host():
    import ctypes
    infos = [binding.acs_variant_generate(inputs.SEED_VARIANTS, i, MARCH) for i in range(40)]
    assert len({v[0] for v in infos}) >= 36
    names = binding.acs_variant_feature_names()
    feats = np.array([v[2].feats[:] for v in infos])
    assert len(set(feats[:, names.index("dp_ops_est")])) > 10
    assert {(v[2].block_x, v[2].block_y) for v in infos} >= {(16, 16), (32, 8)}
    assert {v[2].flags for v in infos} == {0, 1, 2, 3}
    assert set(feats[:, names.index("n_rcp_fast")]) >= {0.0, 1.0}
    # NVRTC compiles without a device (out == NULL: compile check only)
    st = binding.lib().acs_variant_build(infos[0][0].encode(), ctypes.byref(infos[0][2]), None, None)
    if st == 4:
        pytest.skip("NVRTC not available")
    assert st == 0, binding.lib().acs_last_error().decode()
    for src, _, info in infos[1:6]:
        assert binding.lib().acs_variant_build(src.encode(), ctypes.byref(info), None, None) == 0, \
            binding.lib().acs_last_error().decode()


def test_threaded_generation_matches_one_at_a_time():
    """ranker.generate runs the host rewriter on several threads; the variants, their order and
    their features equal those of one-at-a-time calls (the rewriter keeps no shared state)."""
    par = ranker.generate(24, inputs.SEED_VARIANTS, binding.SCOPE_MARCH, start=500, threads=8)
    for v in par:
        src, dag, info = binding.acs_variant_generate(inputs.SEED_VARIANTS, v["index"], binding.SCOPE_MARCH)
        assert v["src"] == src and v["dag"] == dag
        assert np.array_equal(v["feats"], np.array(info.feats[:], dtype=np.float32))
    assert [v["index"] for v in par] == list(range(500, 524))
