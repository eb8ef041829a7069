"""The allocation-free mass tally (lbm_mass_noalloc) against the context
entry point lbm_get_diagnostics and against a host sum of the same
populations.

Callers whose device memory belongs to another allocator (a framework's
caching pool, a pre-reserved arena) cannot call cudaMalloc;
lbm_mass_noalloc serves them from a fixed device array.  This file runs last
so that a failure here stops a -x run only after every other test has run;
it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2512_12934_gb300 import lbm
from paper_2512_12934_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _host_mass(f, solid):
    """FP64 sum over fluid nodes of sum_i f_i, per component, on the host."""
    fluid = np.ones(f.shape[2:], dtype=bool) if solid is None else (solid == 0)
    return np.array([f[k][:, fluid].sum(dtype=np.float64) for k in range(2)])


def _pitched(torch, f, pitch, dtype):
    """[2][9][ny][pitch] device copy of host populations [2][9][ny][nx]; the
    padding columns hold NaN, so reading them shows up in the sum."""
    ny, nx = f.shape[2:]
    buf = np.full((2, 9, ny, pitch), np.nan)
    buf[..., :nx] = f
    return torch.tensor(buf, dtype=dtype, device="cuda").contiguous()


def _mask(torch, solid, pitch):
    if solid is None:
        return None
    m = np.zeros((solid.shape[0], pitch), dtype=np.uint8)  # padding fluid: a read of it brings NaN in
    m[:, :solid.shape[1]] = solid
    return torch.tensor(m, dtype=torch.uint8, device="cuda").contiguous()


@pytest.mark.parametrize("precision, dtype_name", [("fp32", "float32"), ("fp64", "float64")])
@pytest.mark.parametrize("pad", [0, 13])
def test_noalloc_mass_matches_diagnostics_on_two_calls(precision, dtype_name, pad):
    torch = pytest.importorskip("torch")
    dtype = getattr(torch, dtype_name)
    w = W.channel(nx=150, ny=40, R=8, xc=50, u_max=0.02, G12=1.6, Gw=(0.5, -0.5))
    s = lbm.Solver(w.cfg, w.solid, w.rho, w.u, precision=precision)
    nx, ny = w.cfg["nx"], w.cfg["ny"]
    pitch = nx + pad
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    solid = _mask(torch, w.solid, pitch)
    for call in range(2):                          # two calls in a row share the scratch array
        s.step(40 + 17 * call)
        want = s.diagnostics()["mass"]
        f = s.populations()                        # host [2][9][ny][nx], exact copy of the state
        ft = _pitched(torch, f, pitch, dtype)
        out.fill_(float("nan"))
        lbm.mass_noalloc(ft.data_ptr(), precision, nx, ny, pitch, solid.data_ptr(), out.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.allclose(got, want, rtol=1e-9, atol=0.0), (call, got, want)
        host = _host_mass(f.astype(np.float32 if precision == "fp32" else np.float64).astype(np.float64),
                          w.solid)
        assert np.allclose(got, host, rtol=1e-12, atol=0.0), (call, got, host)


def test_noalloc_mass_without_a_solid_mask():
    """A periodic box has no walls: solid = NULL, every node counts."""
    torch = pytest.importorskip("torch")
    w = W.laplace(nx=70, ny=41, R=12, G12=1.2)
    s = lbm.Solver(w.cfg, None, w.rho, w.u, precision="fp32")
    nx, ny = w.cfg["nx"], w.cfg["ny"]
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    for call, pitch in enumerate((nx, nx + 7)):
        s.step(30)
        want = s.diagnostics()["mass"]
        f = s.populations()
        ft = _pitched(torch, f, pitch, torch.float32)
        out.fill_(float("nan"))
        lbm.mass_noalloc(ft.data_ptr(), "fp32", nx, ny, pitch, None, out.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.allclose(got, want, rtol=1e-9, atol=0.0), (call, got, want)
        assert np.allclose(got, _host_mass(f.astype(np.float32).astype(np.float64), None), rtol=1e-12,
                           atol=0.0), call


def test_noalloc_rejects_rows_beyond_the_scratch_limit():
    torch = pytest.importorskip("torch")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    f = torch.zeros(18 * 4, dtype=torch.float32, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.mass_noalloc(f.data_ptr(), "fp32", 1, 65537, 1, None, out.data_ptr())
    assert e.value.status == 1 and "65536" in str(e.value)
