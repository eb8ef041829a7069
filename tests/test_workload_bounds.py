"""Host-side bounds of the seeded T-junction ensemble generator (Sec. III D):
every inlet's peak speed stays at or below the cap, and the drawn viscosity
ratios stay inside the generator's box.  No GPU needed."""
import numpy as np

from paper_2512_12934_gb300 import workloads as W


def test_tjunction_ensemble_inlet_speeds_are_capped():
    u_cap = 0.05
    for w in W.tjunction_ensemble(24, u_cap=u_cap):
        peaks = [float(np.max(np.abs(np.asarray(f["profile"])))) for f in w.cfg["faces"] if f["kind"] == "inlet"]
        assert len(peaks) == 2  # main channel and side channel
        assert max(peaks) <= u_cap * (1 + 1e-12), (w.name, peaks)


def test_tjunction_ensemble_viscosity_ratio_box():
    lo, hi = 0.25, 4.0
    for w in W.tjunction_ensemble(24, m_range=(lo, hi)):
        nu_d, nu_c = w.cfg["nu"]
        assert lo * (1 - 1e-12) <= nu_d / nu_c <= hi * (1 + 1e-12), (w.name, nu_d / nu_c)
