"""GPU: both CUDA forms of both loop bodies against the stored exact values (tests/golden/),
per point within the parity tolerance |gpu - ref| <= 1e-12 |ref| + 1e-14."""
import pytest

from paper_2306_13002_gb300 import binding
from _parity import assert_parity, to_dev
import test_golden as tg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("form", ["plain", "saturated"])
@pytest.mark.parametrize("name,kind,dims,seed,h", tg.CASES, ids=[c[0] for c in tg.CASES])
def test_cuda_matches_stored_values(form, name, kind, dims, seed, h):
    args, ref = tg.golden_case(name, kind, dims, seed, h)
    nx, ny, nz = dims
    if kind == "rhs":
        U = to_dev(args[0])
        R = torch.full((5, nz, ny, nx), float("nan"), dtype=torch.float64, device="cuda")
        fn = binding.acs_rhs_plain if form == "plain" else binding.acs_rhs_saturated
        fn(U, R, h=h)
        torch.cuda.synchronize()
        assert_parity(R.cpu().numpy(), ref, what=f"{name} {form}")
    else:
        u, a = to_dev(args[0]), to_dev(args[1])
        out = torch.full((nz, ny, nx), float("nan"), dtype=torch.float64, device="cuda")
        fn = binding.acs_stencil_plain if form == "plain" else binding.acs_stencil_saturated
        fn(u, a, out)
        torch.cuda.synchronize()
        assert_parity(out.cpu().numpy(), ref, what=f"{name} {form}")
