"""Moving walls beyond the closed y edges (lbm_set_wall_velocity): plane
Couette flow is exact, a sheared droplet matches the FP64 oracle with the
same walls."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_12934_gb300 import lbm
from paper_2512_12934_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("precision, tol", [("fp32", 2e-6), ("fp64", 1e-12)])
def test_plane_couette_flow_is_exact(precision, tol):
    nx, ny, U = 64, 40, 0.03
    cfg = W._base_cfg(nx, ny, (1, 0), 0.0, (0.0, 0.0), (1 / 6, 1 / 6))
    cfg["wall_ux"] = (-U, U)
    rho = np.empty((2, ny, nx))
    rho[0], rho[1] = 0.3, 0.7
    s = lbm.Solver(cfg, None, rho, np.zeros((2, ny, nx)), precision=precision)
    m0 = s.diagnostics()["mass"]
    s.step(30000)
    _, u = s.macros()
    want = -U + 2 * U * (np.arange(ny) + 0.5) / ny
    assert np.max(np.abs(u[0] - want[:, None])) <= tol * U * 10
    assert np.max(np.abs(u[1])) <= tol * U * 10
    assert np.all(np.abs(s.diagnostics()["mass"] - m0) / m0 <= (1e-6 if precision == "fp32" else 1e-12))


@pytest.mark.parametrize("variant", [0, 1])
def test_sheared_droplet_matches_oracle(variant):
    w = W.sheared_droplet(nx=96, ny=48, R=10, U=0.02, G12=1.4, M=3.0)
    s = lbm.Solver(w.cfg, w.solid, w.rho, w.u)
    s.set_tile_variant(variant)
    s.step(100)
    o = O.Oracle2D(w.cfg, w.solid, w.rho, w.u)
    o.step(100)
    ro, uo, _ = o.macros()
    rg, ug = s.macros()
    assert rel(rg, ro) <= 1e-5 and rel(ug, uo) <= 1e-5


def test_wall_velocity_refused_where_not_defined():
    w = W.laplace(nx=40, ny=40, R=8, G12=1.2)       # periodic in y: no wall to move
    s = lbm.Solver(w.cfg, w.solid, w.rho, w.u)
    with pytest.raises(lbm.LbmError) as e:
        s.set_wall_velocity("ymax", 0.01)
    assert e.value.status == 1
