"""The allocation-free mass tally (lbm_mass_noalloc) against the context
entry point lbm_get_diagnostics.

Callers whose device memory belongs to another allocator cannot call
cudaMalloc; lbm_mass_noalloc serves them from a fixed device array.  This
file runs last so that a failure here stops a -x run only after every other
test has run; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2512_12934_gb300 import lbm
from paper_2512_12934_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _device_copy(torch, solver, w, dtype):
    f = solver.populations()                       # host [2][9][ny][nx], exact copy of the state
    ft = torch.tensor(f, dtype=dtype, device="cuda").contiguous()
    solid = None if w.solid is None else torch.tensor(w.solid, dtype=torch.uint8, device="cuda")
    return ft, solid


@pytest.mark.parametrize("precision, dtype_name", [("fp32", "float32"), ("fp64", "float64")])
def test_noalloc_mass_matches_diagnostics_on_two_calls(precision, dtype_name):
    torch = pytest.importorskip("torch")
    dtype = getattr(torch, dtype_name)
    w = W.channel(nx=150, ny=40, R=8, xc=50, u_max=0.02, G12=1.6, Gw=(0.5, -0.5))
    s = lbm.Solver(w.cfg, w.solid, w.rho, w.u, precision=precision)
    nx, ny = w.cfg["nx"], w.cfg["ny"]
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):                          # two calls in a row share the scratch array
        s.step(40 + 17 * call)
        want = s.diagnostics()["mass"]
        ft, solid = _device_copy(torch, s, w, dtype)
        out.fill_(float("nan"))
        lbm.mass_noalloc(ft.data_ptr(), precision, nx, ny, nx, solid.data_ptr(), out.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.allclose(got, want, rtol=1e-9, atol=0.0), (call, got, want)


def test_noalloc_rejects_rows_beyond_the_scratch_limit():
    torch = pytest.importorskip("torch")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    f = torch.zeros(18 * 4, dtype=torch.float32, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.mass_noalloc(f.data_ptr(), "fp32", 1, 65537, 1, None, out.data_ptr())
    assert e.value.status == 1 and "65536" in str(e.value)
