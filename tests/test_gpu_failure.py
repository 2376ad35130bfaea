"""The bounded device-side wait, made to run out on the GPU without a fault.

The saturated kernels wait on mbarriers for their TMA plane copies with a bound of about one
second of SM clock cycles; a wait that runs out is counted and the kernel ends. Here the same
wait runs on an mbarrier phase that nothing completes (no copy is issued at all), so every wait
runs out: the test checks the count, the time it took, that the kernels' own counter is left
alone, and that the context still computes correct results afterwards.
"""
import time

import pytest

import oracle
from paper_2306_13002_gb300 import binding, inputs
from _parity import assert_parity, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_bounded_wait_runs_out_reports_and_leaves_the_context_usable():
    torch.cuda.synchronize()
    before = binding.acs_wait_timeouts()
    t0 = time.perf_counter()
    assert binding.acs_wait_selftest() == 32
    elapsed = time.perf_counter() - t0
    assert 0.2 < elapsed < 30.0, elapsed          # 2^31 SM cycles: ~1 s at 2 GHz
    assert binding.acs_wait_timeouts() == before
    # the context is still usable: a TMA-staged saturated call right after matches the oracle
    u, a = inputs.stencil_fields(40, 24, 12, halo=4, seed=7900)
    out = torch.full((12, 24, 40), float("nan"), dtype=torch.float64, device="cuda")
    binding.acs_stencil_saturated(to_dev(u), to_dev(a), out, tile=(32, 8, 0, binding.TILE_TMA))
    torch.cuda.synchronize()
    assert_parity(out.cpu().numpy(), oracle.stencil(u, a), what="stencil after the wait self-test")
    assert binding.acs_wait_timeouts() == before
