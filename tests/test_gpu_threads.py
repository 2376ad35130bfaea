"""Calls from several host threads at once: the library's per-device caches (occupancy,
tensor-map encoder, tuned shapes, wait counter) and the host-streamed path's shared library
streams must give the same results as calls made one at a time."""
import threading

import pytest

import oracle
from paper_2306_13002_gb300 import binding, inputs
from _parity import assert_parity, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run_threads(fns):
    errors = []

    def wrap(fn):
        try:
            fn()
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(e)

    ts = [threading.Thread(target=wrap, args=(fn,)) for fn in fns]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=300)
    assert not errors, errors


def test_device_calls_from_four_threads():
    cases = []
    for q in range(4):
        if q % 2 == 0:
            U = inputs.rhs_field(40 + 8 * q, 24, 18, halo=2, seed=8100 + q)
            Ud = to_dev(U)
            R = torch.full((5, 18, 24, 40 + 8 * q), float("nan"), dtype=torch.float64, device="cuda")
            cases.append(("rhs", U, Ud, R))
        else:
            u, a = inputs.stencil_fields(48 + 4 * q, 20, 16, halo=4, seed=8100 + q)
            out = torch.full((16, 20, 48 + 4 * q), float("nan"), dtype=torch.float64, device="cuda")
            cases.append(("star", (u, a), (to_dev(u), to_dev(a)), out))
    torch.cuda.synchronize()
    before = binding.acs_wait_timeouts()

    def work(case):
        kind, _, dev_in, out = case
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            for rep in range(5):
                if kind == "rhs":
                    binding.acs_rhs_saturated(dev_in, out, tile=None if rep % 2 else (32, 8, 0, 3), stream=s)
                else:
                    binding.acs_stencil_saturated(dev_in[0], dev_in[1], out, tile=None if rep % 2 else (16, 16, 8, 2),
                                                  stream=s)
        s.synchronize()

    _run_threads([lambda c=c: work(c) for c in cases])
    torch.cuda.synchronize()
    for kind, host_in, _, out in cases:
        ref = oracle.rhs(host_in) if kind == "rhs" else oracle.stencil(*host_in)
        assert_parity(out.cpu().numpy(), ref, what=f"threaded {kind} {tuple(out.shape)}")
    assert binding.acs_wait_timeouts() == before


def test_host_streamed_calls_from_two_threads():
    cases = []
    for q in range(2):
        nx, ny, nz = 36 + 4 * q, 20, 50
        U = inputs.rhs_field(nx, ny, nz, halo=2, seed=8200 + q)
        Uh = torch.from_numpy(U).pin_memory()
        Rh = torch.full((5, nz, ny, nx), float("nan"), dtype=torch.float64).pin_memory()
        ws = torch.empty(binding.acs_rhs_host_workspace_bytes(Uh, Rh, slab=8) // 8 + 2, dtype=torch.float64,
                         device="cuda")
        cases.append((U, Uh, Rh, ws))

    def work(case):
        _, Uh, Rh, ws = case
        s = torch.cuda.Stream()
        for _ in range(3):
            binding.acs_rhs_saturated_host(Uh, Rh, ws, slab=8, stream=s)
        s.synchronize()

    _run_threads([lambda c=c: work(c) for c in cases])
    for U, _, Rh, _ in cases:
        assert_parity(Rh.numpy(), oracle.rhs(U), what=f"threaded host-streamed {U.shape}")
