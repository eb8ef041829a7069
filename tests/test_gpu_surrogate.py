"""The learned surrogate end to end: solver-generated T-junction labels,
ensemble training in the library's MLP kernels, and queries answered by the
network where its ensemble spread is within 5 % and by the solver elsewhere.
The solver is the reference: held-out points are compared with their solver
labels, and fallback answers must equal the solver's bit for bit."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def data():
    from paper_2512_12934_gb300 import surrogate as S
    dev = S.Device(Wc=16, length_factor=20, steps=80000, every=100)
    pts = S.sample_points(240, 2512006)
    Y, valid, sec_per_point = S.generate(pts, dev)
    return S, dev, pts, Y, valid, sec_per_point


def test_labels_follow_the_plug_length_trend(data):
    """Sec. III D: the plug grows linearly with the flow-rate ratio."""
    S, dev, pts, Y, valid, _ = data
    assert valid.mean() > 0.7
    q, D = pts[valid, 1], Y[valid, 0]
    slope, icpt = np.polyfit(q, D, 1)
    assert 0.5 < slope < 1.5 and 0.8 < icpt < 1.2, (slope, icpt)
    # the generation period falls as the dispersed flow rate rises
    assert np.corrcoef(np.log(q), np.log(Y[valid, 1]))[0, 1] < -0.5


def test_surrogate_matches_solver_and_falls_back(data):
    S, dev, pts, Y, valid, sec_per_point = data
    gamma = S.surface_tension()
    assert 0.05 < gamma < 0.2
    tr = np.arange(192)[valid[:192]]
    te = 192 + np.arange(48)[valid[192:]]
    sur = S.Surrogate(members=5, gamma=gamma, dev=dev)
    try:
        sur.fit(pts[tr], Y[tr], epochs=300, batch=16, lr=2e-3)
        # held-out points: the ensemble against the solver's labels
        val, spread = sur.predict(pts[te])
        err = np.abs(val / Y[te] - 1.0)
        acc = spread <= 0.05
        assert acc.mean() > 0.5
        assert np.median(err[acc, 0]) < 0.03, err[acc, 0]
        assert np.percentile(err[acc, 0], 90) < 0.06, err[acc, 0]
        assert np.median(err[acc, 1]) < 0.06, err[acc, 1]
        # queries outside the training box go to the solver, whose answer is
        # exactly the label it produced for the same point
        out = pts[te[:2]].copy()
        out[:, 1] = 0.8  # flow-rate ratio above the box
        ref, vref, _ = S.generate(out, dev)
        q = np.concatenate([pts[te[:4]], out])
        ans, fb, ok, t = sur.query(q, tol=0.05)
        assert fb[4:].all() and t["n_fallback"] >= 2
        assert np.array_equal(ok[4:], vref)
        assert np.array_equal(ans[4:][vref], ref[vref])
        lbl = fb[:4] & valid[te[:4]]
        assert np.array_equal(ans[:4][lbl], Y[te[:4]][lbl])
        # gain over the solver alone: inference on 65536 points against the
        # solver's cost per point
        big = S.sample_points(65536, 99)
        sur.predict(big[:1024])
        t0 = time.perf_counter()
        sur.predict(big)
        per_point = (time.perf_counter() - t0) / len(big)
        assert sec_per_point / per_point > 1e3, (sec_per_point, per_point)
    finally:
        sur.close()
