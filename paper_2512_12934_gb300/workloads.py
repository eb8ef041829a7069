"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the method: it only lays out geometry
masks, initial component densities, initial velocities and inlet profiles,
plus the plain parameter dictionaries that both front ends translate into
their own structures.  Random numbers come from NumPy's PCG64
(``default_rng(seed)``).

Configuration dictionary (``cfg``) keys:
  nx, ny            grid (x fastest)
  periodic          (px, py) booleans
  G12, Gw, nu       Eq. 10 strength, Eq. 11 strengths per component,
                    kinematic viscosities per component (Eq. 5)
  s_e, s_q          moment rates (s_e <= 0 -> s_nu,k); s_eps_mode 1 = from
                    the most viscous phase, 0 = own viscosity
  body              body-force density (x, y), shared by rho_k / rho
  faces             list of open faces: kind ('inlet'|'outlet'), side
                    ('xmin'|'xmax'|'ymin'|'ymax'), lo, hi (inclusive
                    extent along the face), rho_in (2), alpha, chi, profile
                    (inward normal speed per face position, inlets)
Fields are float64 arrays shaped [component][y][x] (rho) and [dim][y][x] (u).
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

FLOOR = 0.001  # minor-phase density floor (initial fields and inlet compositions)


@dataclass
class Workload:
    name: str
    cfg: dict
    solid: Optional[np.ndarray]
    rho: np.ndarray
    u: np.ndarray
    steps: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def nodes(self) -> int:
        return self.cfg["nx"] * self.cfg["ny"]

    @property
    def fluid_nodes(self) -> int:
        if self.solid is None:
            return self.nodes
        return int((self.solid == 0).sum())


def _base_cfg(nx, ny, periodic, G12, Gw, nu, s_q=1.2, s_e=0.0, s_eps_mode=1, body=(0.0, 0.0)):
    return {"nx": int(nx), "ny": int(ny), "periodic": (bool(periodic[0]), bool(periodic[1])),
            "G12": float(G12), "Gw": (float(Gw[0]), float(Gw[1])),
            "nu": (float(nu[0]), float(nu[1])), "s_e": float(s_e), "s_q": float(s_q),
            "s_eps_mode": int(s_eps_mode), "body": (float(body[0]), float(body[1])), "faces": []}


def droplet_fields(nx, ny, cx, cy, R, inside=0, floor=FLOOR, solid=None, rng=None, noise=0.0,
                   width=0.0):
    """Component `inside` = 1 within radius R of (cx, cy), floor elsewhere;
    the other component is the complement.  width > 0 smooths the step with
    a tanh profile of that width; optional uniform noise."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    if width > 0.0:
        phi = 0.5 * (1.0 - np.tanh(2.0 * (r - R) / width))
    else:
        phi = (r <= R).astype(np.float64)
    rho = np.empty((2, ny, nx))
    a, b = inside, 1 - inside
    rho[a] = floor + (1.0 - floor) * phi
    rho[b] = floor + (1.0 - floor) * (1.0 - phi)
    if rng is not None and noise > 0.0:
        rho += rng.uniform(-noise, noise, size=rho.shape)
    if solid is not None:
        rho[:, solid != 0] = 0.0
    return rho


def laplace(nx=100, ny=100, R=20.0, cx=None, cy=None, G12=3.0, nu=(1.0 / 6, 1.0 / 6),
            seed=2512001, noise=1e-4, steps=5000, s_eps_mode=1) -> Workload:
    """Static droplet in a fully periodic box (Laplace test, Sec. III A)."""
    rng = np.random.default_rng(seed)
    cx = nx / 2 if cx is None else cx
    cy = ny / 2 if cy is None else cy
    cfg = _base_cfg(nx, ny, (1, 1), G12, (0.0, 0.0), nu, s_eps_mode=s_eps_mode)
    rho = droplet_fields(nx, ny, cx, cy, R, rng=rng, noise=noise)
    u = np.zeros((2, ny, nx))
    return Workload("laplace_%dx%d_R%g" % (nx, ny, R), cfg, None, rho, u, steps,
                    {"R": R, "cx": cx, "cy": cy})


def channel_profile(ny, u_max):
    """Parabolic inflow between halfway walls at y=1/2 and y=ny-3/2."""
    H = ny - 2
    y = np.arange(1, ny - 1, dtype=np.float64)
    return 4.0 * u_max * (y - 0.5) * (H + 0.5 - y) / (H * H)


def channel(nx=1024, ny=128, R=30.0, xc=200.0, yc=None, u_max=0.01, G12=2.0, Gw=(0.5, -0.5),
            nu=(1.0 / 30, 1.0 / 6), alpha=True, chi=True, steps=50000, seed=2512002,
            noise=0.0, droplet=True, s_eps_mode=1, width=4.0) -> Workload:
    """Droplet migration in a walled channel with a velocity inlet at x=0 and
    a convective outlet at x=nx-1 (Sec. III C; walls are solid rows 0, ny-1).
    G12 defaults to 2.0: with the printed interaction weights, G12 = 3.2
    diverges within ~50 steps at these viscosities and wall strengths.  The
    droplet starts with a tanh interface of the given width."""
    rng = np.random.default_rng(seed)
    yc = ny / 2 if yc is None else yc
    solid = np.zeros((ny, nx), dtype=np.uint8)
    solid[0, :] = 1
    solid[ny - 1, :] = 1
    cfg = _base_cfg(nx, ny, (0, 0), G12, Gw, nu, s_eps_mode=s_eps_mode)
    prof = channel_profile(ny, u_max)
    cfg["faces"] = [
        {"kind": "inlet", "side": "xmin", "lo": 1, "hi": ny - 2, "rho_in": (FLOOR, 1.0),
         "alpha": int(alpha), "chi": 0, "profile": prof},
        {"kind": "outlet", "side": "xmax", "lo": 1, "hi": ny - 2, "rho_in": (0.0, 0.0),
         "alpha": 0, "chi": int(chi), "profile": np.zeros(ny - 2)},
    ]
    if droplet:
        rho = droplet_fields(nx, ny, xc, yc, R, solid=solid, rng=rng, noise=noise, width=width)
    else:
        rho = np.zeros((2, ny, nx))
        rho[0] = FLOOR
        rho[1] = 1.0
        rho[:, solid != 0] = 0.0
    u = np.zeros((2, ny, nx))
    u[0, 1:ny - 1, :] = prof[:, None]
    return Workload("channel_%dx%d" % (nx, ny), cfg, solid, rho, u, steps,
                    {"R": R, "xc": xc, "yc": yc, "u_max": u_max})


def poiseuille(nx=5, half=20, a=10, rho0=1.02, nu2=1.0 / 6, M=1.0, Fb=1e-6, G12=3.0,
               steps=20000) -> Workload:
    """Two-phase layered Poiseuille flow driven by a body force, periodic in x
    (Sec. III B, Eq. 27): fluid 1 for |y| <= a, fluid 2 for a <= |y| <= L,
    walls (solid rows) so that the halfway walls sit at y = +-L."""
    ny = 2 * half + 2
    solid = np.zeros((ny, nx), dtype=np.uint8)
    solid[0, :] = 1
    solid[ny - 1, :] = 1
    cfg = _base_cfg(nx, ny, (1, 0), G12, (0.0, 0.0), (M * nu2, nu2), body=(Fb, 0.0))
    yc = (ny - 1) / 2.0
    y = np.arange(ny, dtype=np.float64) - yc
    inner = np.abs(y) <= a
    rho = np.zeros((2, ny, nx))
    rho[0] = np.where(inner, rho0, FLOOR)[:, None]
    rho[1] = np.where(inner, FLOOR, rho0)[:, None]
    rho[:, solid != 0] = 0.0
    u = np.zeros((2, ny, nx))
    return Workload("poiseuille_M%g" % M, cfg, solid, rho, u, steps,
                    {"L": half, "a": a, "rho0": rho0, "yc": yc, "Fb": Fb, "M": M})


def random_box(nx, ny, seed, periodic=(1, 1), solid_frac=0.0, G12=1.0, Gw=(0.0, 0.0),
               nu=(0.1, 0.2), u_amp=0.02, rho_lo=0.2, rho_hi=1.0) -> Workload:
    """Small random state for invariants and parity on ragged grids."""
    rng = np.random.default_rng(seed)
    solid = None
    if solid_frac > 0.0:
        solid = (rng.random((ny, nx)) < solid_frac).astype(np.uint8)
    cfg = _base_cfg(nx, ny, periodic, G12, Gw, nu)
    rho = rng.uniform(rho_lo, rho_hi, size=(2, ny, nx))
    u = rng.uniform(-u_amp, u_amp, size=(2, ny, nx))
    if solid is not None:
        rho[:, solid != 0] = 0.0
        u[:, solid != 0] = 0.0
    return Workload("random_%dx%d_s%d" % (nx, ny, seed), cfg, solid, rho, u, 0, {})


def tjunction(Wc=40, length_factor=20, Wd=None, side_len=None, x_side=None, Ca=0.01, q_ratio=1.0,
              M=1.0, G12=1.6, Gw=(0.2, -0.2), u_c=0.01, nu_c=1.0 / 6, seed=2512004, front=None) -> Workload:
    """T-junction droplet generator (Sec. III D): a main channel of width Wc
    along x (continuous phase, component 2, velocity inlet at x=0, outlet at
    x=nx-1) and a side channel of width Wd entering from the top (dispersed
    phase, component 1, velocity inlet on the top face, unknowns 4, 7, 8 of
    Eq. 14).  Solid walls one node thick.  Ca is recorded for reference; the
    flow-rate ratio sets the side inflow speed."""
    Wd = int(Wd if Wd is not None else max(4, Wc // 2))
    side_len = int(side_len if side_len is not None else 2 * Wc)
    nx = int(length_factor * Wc)
    ny = Wc + 2 + side_len
    x_side = int(x_side if x_side is not None else 4 * Wc)
    solid = np.ones((ny, nx), dtype=np.uint8)
    solid[1:Wc + 1, :] = 0                                   # main channel rows 1..Wc
    solid[Wc + 1:ny, x_side:x_side + Wd] = 0                 # side channel up to the top edge
    cfg = _base_cfg(nx, ny, (0, 0), G12, Gw, (M * nu_c, nu_c))
    prof_main = 4.0 * u_c * (np.arange(1, Wc + 1) - 0.5) * (Wc + 0.5 - np.arange(1, Wc + 1)) / (Wc * Wc)
    q_c = prof_main.sum()
    xs = np.arange(Wd, dtype=np.float64)
    prof_side = (xs + 0.5) * (Wd - 0.5 - xs)                 # parabola between the side walls
    prof_side *= (q_ratio * q_c) / prof_side.sum()           # side flow rate = q_ratio * main flow rate
    cfg["faces"] = [
        {"kind": "inlet", "side": "xmin", "lo": 1, "hi": Wc, "rho_in": (FLOOR, 1.0), "alpha": 1, "chi": 0,
         "profile": prof_main},
        {"kind": "inlet", "side": "ymax", "lo": x_side, "hi": x_side + Wd - 1, "rho_in": (1.0, FLOOR),
         "alpha": 1, "chi": 0, "profile": prof_side},
        {"kind": "outlet", "side": "xmax", "lo": 1, "hi": Wc, "rho_in": (0.0, 0.0), "alpha": 0, "chi": 1,
         "profile": np.zeros(Wc)},
    ]
    rho = np.zeros((2, ny, nx))
    rho[0] = FLOOR
    rho[1] = 1.0
    if front is None:
        rho[0, Wc + 1:, :] = 1.0                             # side channel filled with dispersed phase
        rho[1, Wc + 1:, :] = FLOOR
    else:
        yy = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
        ph = 0.5 * (1.0 + np.tanh((yy - (Wc + 1 + front)) / 2.0))
        rho[0] = FLOOR + (1.0 - FLOOR) * ph
        rho[1] = FLOOR + (1.0 - FLOOR) * (1.0 - ph)
    rho[:, solid != 0] = 0.0
    u = np.zeros((2, ny, nx))
    u[0, 1:Wc + 1, :] = prof_main[:, None]
    u[:, solid != 0] = 0.0
    return Workload("tjunction_Wc%d" % Wc, cfg, solid, rho, u, 0,
                    {"Wc": Wc, "Wd": Wd, "x_side": x_side, "Ca": Ca, "q_ratio": q_ratio, "M": M})


def tjunction_ensemble(n=256, seed=2512004, wc_range=(40, 120), G12=2.0, Gw=(0.2, -0.2), gamma=0.25,
                       u_cap=0.05, length_factor=20):
    """Seeded ensemble of T-junction droplet generators with uneven sizes and
    parameters: W_c ~ U{wc_range}, W_d = U(0.5, 1) W_c, main channel length
    length_factor * W_c, side channel 2 W_c, Ca ~ logU[0.002, 0.05],
    Q_d/Q_c ~ logU[0.2, 5], M = nu_d/nu_c ~ logU[0.1, 10].  The continuous
    inflow speed follows Ca = u_c nu_c rho / gamma with nu_c = 1/6, rho = 1 and
    the given surface tension gamma (lattice units), capped at u_cap."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(n):
        Wc = int(rng.integers(wc_range[0], wc_range[1] + 1))
        Wd = max(4, int(round(rng.uniform(0.5, 1.0) * Wc)))
        Ca = float(np.exp(rng.uniform(np.log(0.002), np.log(0.05))))
        q = float(np.exp(rng.uniform(np.log(0.2), np.log(5.0))))
        M = float(np.exp(rng.uniform(np.log(0.1), np.log(10.0))))
        nu_c = 1.0 / 6.0
        u_c = min(u_cap, Ca * gamma / nu_c)
        w = tjunction(Wc=Wc, length_factor=length_factor, Wd=Wd, side_len=2 * Wc, x_side=4 * Wc, Ca=Ca,
                      q_ratio=q, M=M, G12=G12, Gw=Gw, u_c=u_c, nu_c=nu_c, seed=seed + j)
        w.name = "tjunction_%03d" % j
        out.append(w)
    return out
