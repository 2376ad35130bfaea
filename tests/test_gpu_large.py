"""Large workloads: RHS 512^3 (5.5 GB in, 5.4 GB out) and the star stencil at 768^3, both forms,
checked against the oracle on sampled z-planes (block-chunk edges, first and last planes)."""
import numpy as np
import pytest

import oracle
from paper_2306_13002_gb300 import binding, inputs
from _parity import assert_parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rhs512():
    n = 512
    U = inputs.rhs_field(n, halo=2, seed=inputs.SEED_HUGE)
    yield n, U, torch.from_numpy(U).cuda()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("form", ["as_written", "saturated"])
def test_rhs_512cubed_sampled_planes(rhs512, form):
    n, U, Ud = rhs512
    R = torch.empty((5, n, n, n), dtype=torch.float64, device="cuda")
    binding.acs_rhs_form(Ud, R, form)
    torch.cuda.synchronize()
    for k in [0, 1, 31, 32, 255, 256, 383, 510, 511]:
        ref = oracle.rhs(U, k_range=(k, k + 1), threads=16)[:, k]
        assert_parity(R[:, k].cpu().numpy(), ref, what=f"rhs {form} 512^3 plane {k}")
    assert torch.isfinite(R).all()
    del R


@pytest.mark.parametrize("form", ["plain", "saturated"])
def test_stencil_768cubed_sampled_planes(form):
    n = 768
    u, a = inputs.stencil_fields(n, halo=4, seed=inputs.SEED_HUGE)
    ud, ad = torch.from_numpy(u).cuda(), torch.from_numpy(a).cuda()
    out = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
    (binding.acs_stencil_plain if form == "plain" else binding.acs_stencil_saturated)(ud, ad, out)
    torch.cuda.synchronize()
    for k in [0, 3, 4, 15, 16, 383, 384, 700, 767]:
        ref = oracle.stencil(u, a, k_range=(k, k + 1), threads=16)[k]
        assert_parity(out[k].cpu().numpy(), ref, what=f"stencil {form} 768^3 plane {k}")
    assert torch.isfinite(out).all()
    del ud, ad, out
    torch.cuda.empty_cache()
