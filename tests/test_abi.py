"""The C-ABI library loads and exports every entry point include/*.h
declares; host-side validation rejects bad arguments before any device
work (runs without a GPU)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2512_12934_gb300 import build as libbuild
from paper_2512_12934_gb300 import lbm
from paper_2512_12934_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(lbm[a-z0-9_]*)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return lbm.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lbm_create", "lbm_step", "lbm_get_macros", "lbm_destroy", "lbm_get_diagnostics",
                 "lbm_save", "lbm_load", "lbm_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_library_is_built_for_sm103a(L):
    assert "sm_103a" in L.lbm_version().decode()


def _create(cfg, rho, solid=None, u=None, precision="fp32"):
    return lbm.Solver(cfg, solid, rho, u, precision=precision)


@pytest.mark.parametrize("mutate, why", [
    (lambda c: c.update(nx=4), "extent"),
    (lambda c: c.update(nu=(0.0, 0.1)), "viscosities"),
    (lambda c: c.update(nu=(-1.0, 0.1)), "viscosities"),
    (lambda c: c.update(s_q=2.5), "relaxation rate"),
])
def test_invalid_parameters_are_rejected_before_device_work(L, mutate, why):
    w = W.laplace(nx=16, ny=16, R=4)
    cfg = dict(w.cfg)
    mutate(cfg)
    rho = np.ones((2, cfg["ny"], cfg["nx"]))
    with pytest.raises(lbm.LbmError) as e:
        _create(cfg, rho)
    assert e.value.status == 1
    assert why in str(e.value)


def test_bad_faces_are_rejected(L):
    w = W.channel(nx=40, ny=12, R=3, xc=10)
    # face on a periodic axis
    cfg = dict(w.cfg, periodic=(1, 0))
    with pytest.raises(lbm.LbmError) as e:
        _create(cfg, w.rho, w.solid, w.u)
    assert e.value.status == 1
    # two outlets
    cfg = dict(w.cfg)
    cfg["faces"] = w.cfg["faces"] + [dict(w.cfg["faces"][1], side="ymax", lo=1, hi=30)]
    with pytest.raises(lbm.LbmError) as e:
        _create(cfg, w.rho, w.solid, w.u)
    assert e.value.status == 1
    # inward neighbour must be fluid
    solid = w.solid.copy()
    solid[5, 1] = 1
    with pytest.raises(lbm.LbmError) as e:
        _create(w.cfg, w.rho, solid, w.u)
    assert "inward neighbour" in str(e.value)


def test_unsupported_lattice_reported(L):
    g = lbm.lbm_grid()
    g.lattice, g.nx, g.ny, g.nz = 7, 8, 8, 1
    p = lbm.lbm_params()
    p.nu[0] = p.nu[1] = 0.1
    rho = np.ones(128)
    h = ctypes.c_void_p()
    st = L.lbm_create(ctypes.byref(g), ctypes.byref(p), None, 0, None,
                      rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, None, ctypes.byref(h))
    assert st == 6 and not h.value
    assert L.lbm_last_error(None)


def test_mlp_parameter_count_and_argument_checks(L):
    from oracle import mlp_oracle as M
    assert L.lbm_mlp_num_params() == M.n_params()
    for members in (0, -1, 65):
        with pytest.raises(lbm.LbmError) as e:
            lbm.MLP(members)
        assert e.value.status == 1
