"""Early-launch step graphs (LBM_SCHEDULE_GRAPHS_EARLY): the captured graphs'
kernel-to-kernel dependencies become programmatic ones, each step kernel
waits on the device for the grids it depends on, and the populations stay
bit-identical to the plain graph schedule (every memory access keeps its
order; only launches move earlier)."""
import time

import numpy as np
import pytest

from paper_2512_12934_gb300 import lbm
from paper_2512_12934_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def run(w, schedule, steps, variant=None, same_step=False, precision="fp32"):
    s = lbm.Solver(w.cfg, w.solid, w.rho, w.u, precision=precision)
    if variant is not None:
        s.set_tile_variant(variant)
    if same_step:
        s.set_chi_timing(True)
    s.set_schedule(schedule)
    s.step(steps)
    s.sync()
    f = s.populations()
    d = s.diagnostics()
    sched = s.schedule()
    s.close()
    return f, d, sched


@pytest.mark.parametrize("variant, same_step, precision", [
    (None, False, "fp32"), (None, True, "fp32"), (4, False, "fp32"), (None, False, "fp64"),
    (None, False, "fp16store")])
def test_early_graphs_are_bit_identical_to_plain_graphs(variant, same_step, precision):
    w = W.channel(nx=512, ny=96, R=14, xc=120, u_max=0.02, G12=1.6)
    steps = 3 * 32 + 5  # three graph replays and single launches after them
    f0, d0, s0 = run(w, "graphs", steps, variant, same_step, precision)
    f1, d1, s1 = run(w, "graphs_early", steps, variant, same_step, precision)
    assert s0 == ("graphs", False)
    assert s1 == ("graphs_early", True), "the driver refused the programmatic edges"
    assert d0["status"] == 0 and d1["status"] == 0
    assert np.array_equal(f0.view(np.uint8), f1.view(np.uint8))
    assert d0["lambda"] == d1["lambda"] and d0["chi"] == d1["chi"]


def test_early_batch_graphs_are_bit_identical():
    shapes = [(300, 72, 10, 80), (200, 40, 8, 60), (420, 80, 12, 100)]

    def batch_state(schedule):
        ws = [W.channel(nx=nx, ny=ny, R=R, xc=xc, u_max=0.02, G12=1.6) for nx, ny, R, xc in shapes]
        ms = [lbm.Solver(w.cfg, w.solid, w.rho, w.u) for w in ws]
        b = lbm.Batch(ms)
        b.set_schedule(schedule)
        b.step(2 * 32 + 3)
        b.sync()
        out = [m.populations() for m in ms], b.schedule()
        b.close()
        for m in ms:
            m.close()
        return out

    plain, sp = batch_state("graphs")
    early, se = batch_state("graphs_early")
    assert sp == ("graphs", False) and se == ("graphs_early", True)
    for a, b in zip(plain, early):
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8))


def test_early_graphs_step_time_on_the_1024x128_channel():
    """Informational timing on the droplet-migration channel (1024 x 128,
    FP32): the early-launch graphs must not be slower than the plain ones
    by more than noise."""
    w = W.channel()
    t = {}
    for sched in ("graphs", "graphs_early", "graphs", "graphs_early"):
        s = lbm.Solver(w.cfg, w.solid, w.rho, w.u)
        s.set_schedule(sched)
        s.step(640)
        s.sync()
        t0 = time.perf_counter()
        s.step(6400)
        s.sync()
        t[sched] = min(t.get(sched, 1e9), (time.perf_counter() - t0) / 6400 * 1e6)
        assert s.diagnostics()["status"] == 0
        s.close()
    print("\n[early launch] 1024x128 channel: %.2f us/step plain graphs, %.2f us/step early graphs"
          % (t["graphs"], t["graphs_early"]))
    assert t["graphs_early"] <= 1.05 * t["graphs"]
