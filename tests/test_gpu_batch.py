"""Batched ensembles: many instances in one launch per tile list per step.

While the batch's general list is at most two CTAs per SM, a batch step
applies to every member exactly the arithmetic of stepping that member alone
with the same tile shape, so results are bit-identical; longer general lists
stage serially (same method, different code) and agree to the FP32 parity
bar.  The autotuner leaves the run unchanged."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_12934_gb300 import lbm
from paper_2512_12934_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def members():
    return [W.laplace(nx=70, ny=50, R=12, G12=1.2),
            W.channel(nx=130, ny=30, R=6, xc=40, u_max=0.02, G12=1.4, Gw=(0.3, -0.3)),
            W.tjunction(Wc=12, length_factor=12, Wd=6, side_len=10, x_side=30, G12=1.2, Gw=(0.1, -0.1)),
            W.random_box(45, 37, 5, periodic=(1, 0), solid_frac=0.05, G12=0.9)]


def solvers(ws, precision="fp32", variant=1):
    out = []
    for w in ws:
        s = lbm.Solver(w.cfg, w.solid, w.rho, w.u, precision=precision)
        s.set_tile_variant(variant)
        out.append(s)
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp16store"])
def test_batch_step_is_bitwise_equal_to_member_steps(precision):
    ws = members()
    solo = solvers(ws, precision)
    for s in solo:
        s.step(73)
    batched = solvers(ws, precision)
    b = lbm.Batch(batched)
    b.step(40)
    b.step(33)
    b.sync()
    for a, c in zip(solo, batched):
        assert np.array_equal(a.populations(), c.populations())
        assert np.array_equal(a.macros()[1], c.macros()[1])
        assert c.diagnostics()["step"] == 73
    info = b.info()
    assert info["fast_tiles"] > 0 and info["general_tiles"] > 0


def test_long_general_list_stages_serially():
    """A batch whose general list is longer than two CTAs per SM stages its
    general tiles serially on the node threads (FP32 storage); members
    stepped alone stage theirs with the extra staging warps.  The two kernels
    inline the face reconstruction differently (multiply-add contraction), so
    they agree to the FP32 parity bar, not bit for bit; one member is also
    checked against the FP64 oracle."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ws = [W.channel(nx=130, ny=30, R=5 + (i % 3), xc=30 + 2 * i, u_max=0.015 + 0.001 * (i % 4), G12=1.3,
                    Gw=(0.3, -0.3)) for i in range(24)]
    solo = solvers(ws)
    for s in solo:
        s.step(61)
    batched = solvers(ws)
    b = lbm.Batch(batched)
    assert b.info()["general_tiles"] > 2 * sms
    b.step(61)
    b.sync()
    for a, c in zip(solo, batched):
        fa, fc = a.populations(), c.populations()
        assert np.abs(fa - fc).max() <= 1e-5 * np.abs(fa).max()
        d = c.diagnostics()
        assert d["status"] == 0 and d["step"] == 61
    o = O.Oracle2D(ws[5].cfg, ws[5].solid, ws[5].rho, ws[5].u)
    o.step(61)
    ro, uo, _ = o.macros()
    rg, ug = batched[5].macros()
    assert np.max(np.abs(rg - ro)) / np.max(np.abs(ro)) < 1e-5
    assert np.max(np.abs(ug - uo)) / np.max(np.abs(uo)) < 1e-5


def test_batch_members_can_be_stepped_alone_in_between():
    ws = members()
    solo = solvers(ws)
    for s in solo:
        s.step(50)
    batched = solvers(ws)
    b = lbm.Batch(batched)
    b.step(20)
    batched[1].step(7)      # one member advances on its own
    b.step(13)              # the batch re-syncs its argument blocks
    for i, (a, c) in enumerate(zip(solo, batched)):
        want = 33 + (7 if i == 1 else 0)
        assert c.diagnostics()["step"] == want
    # member 1 took 40 steps in total, the others 33: compare against the oracle
    o = O.Oracle2D(ws[1].cfg, ws[1].solid, ws[1].rho, ws[1].u)
    o.step(40)
    ro, uo, _ = o.macros()
    rg, ug = batched[1].macros()
    assert np.max(np.abs(rg - ro)) / np.max(np.abs(ro)) < 1e-5


def test_batch_autotune_leaves_the_run_unchanged():
    ws = [W.laplace(nx=96, ny=64, R=14, G12=1.2), W.random_box(80, 50, 6, periodic=(1, 1), G12=0.8)]
    ref = solvers(ws)
    for s in ref:
        s.step(60)
    tuned = solvers(ws)
    b = lbm.Batch(tuned)
    b.step(25)
    v, ms = b.autotune(steps=8)
    assert 0 <= v < 4 and ms > 0
    b.step(35)
    for a, c in zip(ref, tuned):   # periodic members: bit-identical whatever the tile shape
        assert np.array_equal(a.populations(), c.populations())


def test_single_context_autotune():
    w = W.channel(nx=160, ny=34, R=6, xc=50, u_max=0.02, G12=1.4)
    a = lbm.Solver(w.cfg, w.solid, w.rho, w.u)
    a.step(30)
    v, ms = a.autotune(steps=6)
    assert a.tile_stats()["variant"] == v
    a.step(30)
    o = O.Oracle2D(w.cfg, w.solid, w.rho, w.u)
    o.step(60)
    assert np.max(np.abs(a.macros()[1] - o.macros()[1])) / np.max(np.abs(o.macros()[1])) < 1e-5


def test_batch_rejects_mixed_precision():
    w = W.laplace(nx=20, ny=20, R=4)
    a = lbm.Solver(w.cfg, w.solid, w.rho, w.u, precision="fp32")
    c = lbm.Solver(w.cfg, w.solid, w.rho, w.u, precision="fp64")
    with pytest.raises(lbm.LbmError) as e:
        lbm.Batch([a, c])
    assert e.value.status == 1


def test_member_retiled_on_its_own_is_picked_up():
    ws = members()[:2]
    ref = solvers(ws)
    for s in ref:
        s.set_tile_variant(0)
        s.step(30)
    batched = solvers(ws)
    b = lbm.Batch(batched)
    b.step(10)
    for s in batched:
        s.set_tile_variant(0)   # every member re-tiled behind the batch's back
    b.step(20)
    for a, c in zip(ref, batched):
        assert np.max(np.abs(a.macros()[0] - c.macros()[0])) / np.max(np.abs(a.macros()[0])) < 1e-5
