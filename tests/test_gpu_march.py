"""The column-marching step (tile variant 4, FP32 storage): interior tiles
march up their tile column, one TMA bulk copy per block of 8 rows feeding
the pull stream from shared memory; edge and general tiles keep the tile
kernels.  Results must match the FP64 oracle to the FP32 parity bar and the
tile kernels of the same tile shape (variant 0) to FP32 rounding."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_12934_gb300 import lbm
from paper_2512_12934_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MARCH = 4
TOL = 1e-5


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def run(w, variant, steps, precision="fp32"):
    s = lbm.Solver(w.cfg, w.solid, w.rho, w.u, precision=precision)
    s.set_tile_variant(variant)
    s.step(steps)
    s.sync()
    return s


CASES = {
    "channel_300x72": lambda: W.channel(nx=300, ny=72, R=10, xc=90, u_max=0.02, G12=1.6, Gw=(0.5, -0.5)),
    "walled_random_solids": lambda: W.random_box(140, 77, 11, periodic=(0, 0), solid_frac=0.06, G12=0.9,
                                                 Gw=(0.2, -0.1)),
    "tjunction": lambda: W.tjunction(Wc=24, length_factor=10, Wd=12, side_len=20, x_side=60, G12=1.2,
                                     Gw=(0.1, -0.1)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_march_variant_matches_oracle_and_tile_kernels(name):
    w = CASES[name]()
    m = run(w, MARCH, 100)
    st = m.tile_stats()
    assert st["variant"] == MARCH
    t = run(w, 0, 100)
    o = O.Oracle2D(w.cfg, w.solid, w.rho, w.u)
    o.step(100)
    ro, uo, _ = o.macros()
    rm, um = m.macros()
    rt, ut = t.macros()
    print("\n[march %s] vs oracle rho %.2e u %.2e; vs tile kernels rho %.2e u %.2e (bitwise %s)"
          % (name, rel(rm, ro), rel(um, uo), rel(rm, rt), rel(um, ut),
             np.array_equal(m.populations(), t.populations())))
    assert rel(rm, ro) <= TOL and rel(um, uo) <= TOL
    assert rel(rm, rt) <= 1e-6 and rel(um, ut) <= 1e-6
    dm, dt = m.diagnostics(), t.diagnostics()
    assert dm["status"] == 0 and np.allclose(dm["mass"], dt["mass"], rtol=1e-9)


def test_march_variant_on_a_large_channel_matches_tile_kernels():
    """8192 x 512 with the channel physics: thousands of marching runs,
    several launches of graph replay."""
    w = W.channel(nx=8192, ny=512, R=60, xc=1000, u_max=0.01, G12=2.0, Gw=(0.5, -0.5))
    m = run(w, MARCH, 70)
    t = run(w, 0, 70)
    rm, um = m.macros()
    rt, ut = t.macros()
    assert rel(rm, rt) <= 1e-6 and rel(um, ut) <= 1e-6
    assert m.diagnostics()["status"] == 0


def test_march_variant_falls_back_to_tile_kernels_for_other_precisions():
    w = CASES["channel_300x72"]()
    for prec in ("fp64", "fp16store"):
        a = run(w, MARCH, 40, prec)
        b = run(w, 0, 40, prec)
        assert np.array_equal(a.populations(), b.populations())


def test_autotune_considers_the_march_variant():
    w = W.channel(nx=2048, ny=512, R=40, xc=300, u_max=0.01, G12=2.0, Gw=(0.5, -0.5))
    s = lbm.Solver(w.cfg, w.solid, w.rho, w.u)
    s.step(10)
    v, ms = s.autotune(steps=20)
    assert 0 <= v <= MARCH and ms > 0
    assert s.tile_stats()["variant"] == v
    s.step(40)
    t = run(w, 0, 50)
    assert rel(s.macros()[1], t.macros()[1]) <= 1e-6
