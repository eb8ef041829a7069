"""Persistent schedule: one cooperative launch runs many time steps of every
member of a batch, with a grid-wide barrier between steps whose waits are
bounded (lbm_batch_set_schedule, lbm_set_schedule).

Its results equal the graph schedule's to the FP32 parity bar and the FP64
oracle's after 100 steps; a barrier that can never complete (host-side fault
injection: the barrier waits for one CTA more than the grid has) ends the
launch after its bounded wait, lbm_batch_sync reports LBM_ERR_TIMEOUT, and
the members can be reset and stepped again."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_12934_gb300 import lbm
from paper_2512_12934_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5  # FP32 against FP64 after 100 steps, max-norm relative (rho and u)


def members():
    return [W.laplace(nx=70, ny=50, R=12, G12=1.2),
            W.channel(nx=130, ny=30, R=6, xc=40, u_max=0.02, G12=1.4, Gw=(0.3, -0.3)),
            W.tjunction(Wc=12, length_factor=12, Wd=6, side_len=10, x_side=30, G12=1.2, Gw=(0.1, -0.1)),
            W.random_box(45, 37, 5, periodic=(1, 0), solid_frac=0.05, G12=0.9)]


def solvers(ws, variant=1):
    out = []
    for w in ws:
        s = lbm.Solver(w.cfg, w.solid, w.rho, w.u, precision="fp32")
        s.set_tile_variant(variant)
        out.append(s)
    return out


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_persistent_batch_matches_graph_schedule_and_oracle(variant):
    ws = members()
    ref = solvers(ws, variant)
    rb = lbm.Batch(ref)
    rb.step(100)
    rb.sync()
    per = solvers(ws, variant)
    pb = lbm.Batch(per)
    pb.set_schedule("persistent")
    pb.step(37)          # two calls: parity and macro output carry over
    pb.step(63)
    pb.sync()
    assert 0 < pb.persistent_grid() <= pb.info()["fast_tiles"] + pb.info()["general_tiles"]
    for w, a, c in zip(ws, ref, per):
        assert c.diagnostics()["step"] == 100 and c.diagnostics()["status"] == 0
        ra, ua = a.macros()
        rc, uc = c.macros()
        assert rel(rc, ra) <= TOL and rel(uc, ua) <= TOL
        o = O.Oracle2D(w.cfg, w.solid, w.rho, w.u)
        o.step(100)
        ro, uo, _ = o.macros()
        assert rel(rc, ro) <= TOL and rel(uc, uo) <= TOL


def test_persistent_runs_span_several_launches():
    """2085 steps = three launches of up to 1024 steps, odd in total."""
    w = W.channel(nx=200, ny=36, R=7, xc=60, u_max=0.02, G12=1.4, Gw=(0.3, -0.3))
    a = lbm.Solver(w.cfg, w.solid, w.rho, w.u)
    a.step(2085)
    c = lbm.Solver(w.cfg, w.solid, w.rho, w.u)
    c.set_schedule("persistent")
    c.step(2085)
    c.sync()
    ra, ua = a.macros()
    rc, uc = c.macros()
    assert rel(rc, ra) <= TOL and rel(uc, ua) <= TOL
    da, dc = a.diagnostics(), c.diagnostics()
    assert dc["step"] == 2085 and abs(dc["chi"] - da["chi"]) < 1e-4 and abs(dc["lambda"] / da["lambda"] - 1) < 1e-4


def test_single_context_persistent_schedule_matches_oracle():
    w = W.channel(nx=256, ny=64, R=10, xc=80, u_max=0.02, G12=1.6, Gw=(0.5, -0.5))
    s = lbm.Solver(w.cfg, w.solid, w.rho, w.u)
    s.set_schedule("persistent")
    s.step(100)
    s.sync()
    o = O.Oracle2D(w.cfg, w.solid, w.rho, w.u)
    o.step(100)
    ro, uo, _ = o.macros()
    rg, ug = s.macros()
    assert rel(rg, ro) <= TOL and rel(ug, uo) <= TOL


def test_barrier_that_cannot_complete_times_out_and_the_batch_recovers():
    ws = members()
    per = solvers(ws)
    pb = lbm.Batch(per)
    pb.set_schedule("persistent")
    pb.step(5)
    pb.sync()
    # every barrier now waits for one CTA more than the grid has; each wait
    # gives up after 2e7 SM clock cycles (about 10 ms)
    pb.inject_barrier_fault(1, 20_000_000)
    pb.step(50)
    with pytest.raises(lbm.LbmError) as e:
        pb.sync()
    assert e.value.status == 5  # LBM_ERR_TIMEOUT
    # back to normal: reset the members and run the same steps as a fresh batch
    pb.inject_barrier_fault(0)
    for w, s in zip(ws, per):
        s.reset(w.rho, w.u)
    pb.step(100)
    pb.sync()
    for w, s in zip(ws, per):
        o = O.Oracle2D(w.cfg, w.solid, w.rho, w.u)
        o.step(100)
        ro, uo, _ = o.macros()
        rg, ug = s.macros()
        assert rel(rg, ro) <= TOL and rel(ug, uo) <= TOL
