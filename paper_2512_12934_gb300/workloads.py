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
        return self.cfg["nx"] * self.cfg["ny"] * self.cfg.get("nz", 1)

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


def channel_obstacle(nx=640, ny=320, R=30.0, xc=70.0, yc=160.0, obstacle=(200, 240, 140, 260), u_max=0.01,
                     G12=1.6, Gw=(0.5, -0.5), nu=(0.17, 1.67), rho0=1.02, wetting_delta=0.5, width=4.0,
                     seed=2512009) -> Workload:
    """Droplet migrating past a rectangular obstacle (Sec. III C, Fig. 7):
    walls top and bottom, velocity inlet at x = 0 (parabolic, u_max), convective
    outlet at x = nx - 1, droplet (component 1) of radius R at (xc, yc), both
    fluids of density rho0, viscosities nu (fluid 2 the more viscous, 1.67 in
    the paper).  The paper does not give the obstacle's coordinates; here it
    is the solid rectangle x in [x0, x1), y in [y0, y1) (obstacle argument),
    centred above the droplet's path so that the flow deflects the droplet
    downwards.  Eq. 12's phase-dependent wetting with the given delta; s_e and
    s_eps from the most viscous fluid (the adjusted rates that stay stable at
    this viscosity ratio).  G12 = 1.6: at 2.0 the Eq. 12 reading with
    G_w = +-0.5 diverges within 1000 steps (+-0.2: 17k steps), constant
    coefficients do not."""
    solid = np.zeros((ny, nx), dtype=np.uint8)
    solid[0, :] = 1
    solid[ny - 1, :] = 1
    x0, x1, y0, y1 = obstacle
    solid[y0:y1, x0:x1] = 1
    cfg = _base_cfg(nx, ny, (0, 0), G12, Gw, nu, s_eps_mode=1)
    cfg["s_e"] = 1.0 / (3.0 * max(nu) + 0.5)
    if wetting_delta:
        cfg["wetting_delta"] = float(wetting_delta)
    prof = channel_profile(ny, u_max)
    cfg["faces"] = [
        {"kind": "inlet", "side": "xmin", "lo": 1, "hi": ny - 2, "rho_in": (FLOOR, rho0), "alpha": 1, "chi": 0,
         "profile": prof},
        {"kind": "outlet", "side": "xmax", "lo": 1, "hi": ny - 2, "rho_in": (0.0, 0.0), "alpha": 0, "chi": 1,
         "profile": np.zeros(ny - 2)},
    ]
    rho = droplet_fields(nx, ny, xc, yc, R, solid=solid, width=width) * rho0
    rho[:, solid != 0] = 0.0
    u = np.zeros((2, ny, nx))
    u[0, 1:ny - 1, :] = prof[:, None]
    u[:, solid != 0] = 0.0
    return Workload("channel_obstacle_%dx%d" % (nx, ny), cfg, solid, rho, u, 0,
                    {"R": R, "xc": xc, "yc": yc, "obstacle": obstacle, "u_max": u_max})


def sheared_droplet(nx=200, ny=100, R=20.0, U=0.01, G12=1.4, M=1.0, nu_m=1.0 / 6, seed=2512008,
                    width=4.0) -> Workload:
    """Taylor deformation (Sec. III A, Fig. 4): a droplet (component 1,
    viscosity M nu_m) centred between walls beyond the closed y edges that
    move along x at -U (bottom) and +U (top), periodic in x; matrix
    component 2 with viscosity nu_m.  The walls sit halfway beyond rows 0
    and ny - 1, a distance ny apart, so the imposed shear rate is 2U / ny."""
    cfg = _base_cfg(nx, ny, (1, 0), G12, (0.0, 0.0), (M * nu_m, nu_m))
    cfg["wall_ux"] = (-float(U), float(U))
    rho = droplet_fields(nx, ny, nx / 2 - 0.5, ny / 2 - 0.5, R, width=width)
    u = np.zeros((2, ny, nx))
    u[0] = (-U + 2.0 * U * (np.arange(ny) + 0.5) / ny)[:, None]
    return Workload("sheared_droplet_%dx%d" % (nx, ny), cfg, None, rho, u, 0,
                    {"R": R, "U": U, "M": M, "shear_rate": 2.0 * U / ny})


def tjunction_ensemble(n=256, seed=2512004, wc_range=(40, 120), G12=1.6, Gw=(0.2, -0.2), gamma=0.25,
                       u_cap=0.05, length_factor=20, m_range=(0.25, 4.0)):
    """Seeded ensemble of T-junction droplet generators with uneven sizes and
    parameters: W_c ~ U{wc_range}, W_d = U(0.5, 1) W_c, main channel length
    length_factor * W_c, side channel 2 W_c, Ca ~ logU[0.002, 0.05],
    Q_d/Q_c ~ logU[0.2, 5], M = nu_d/nu_c ~ logU[m_range].  The continuous
    inflow speed follows Ca = u_c nu_c rho / gamma with nu_c = 1/6, rho = 1 and
    the given surface tension gamma (lattice units), capped so that neither
    inlet's peak speed exceeds u_cap: the side channel carries Q_d/Q_c times
    the main flow through W_d, so its peak is about (Q_d/Q_c)(W_c/W_d) u_c
    (uncapped, up to 0.5 in lattice units, and such members blow up).
    G12 = 1.6 and M within [0.25, 4]: on GB300, 64 members stepped 4000
    times, 39 blew up at G12 = 2.0 (M in [0.1, 10]) and 12 at 1.6, those all
    with M below 0.16 or above 6.6."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(n):
        Wc = int(rng.integers(wc_range[0], wc_range[1] + 1))
        Wd = max(4, int(round(rng.uniform(0.5, 1.0) * Wc)))
        Ca = float(np.exp(rng.uniform(np.log(0.002), np.log(0.05))))
        q = float(np.exp(rng.uniform(np.log(0.2), np.log(5.0))))
        M = float(np.exp(rng.uniform(np.log(m_range[0]), np.log(m_range[1]))))
        nu_c = 1.0 / 6.0
        u_c = min(u_cap, Ca * gamma / nu_c, u_cap * Wd / (q * Wc))
        w = tjunction(Wc=Wc, length_factor=length_factor, Wd=Wd, side_len=2 * Wc, x_side=4 * Wc, Ca=Ca,
                      q_ratio=q, M=M, G12=G12, Gw=Gw, u_c=u_c, nu_c=nu_c, seed=seed + j)
        w.name = "tjunction_%03d" % j
        out.append(w)
    return out


# ---------------------------------------------------------------------------
# D3Q19 workloads (fields [component or axis][z][y][x]; face lo/hi are pairs
# over the two tangential axes in x, y, z order)
# ---------------------------------------------------------------------------

def _base_cfg3(nx, ny, nz, periodic, G12, Gw, nu, s_q=1.2, s_e=0.0, s_eps_mode=1, body=(0.0, 0.0, 0.0)):
    return {"lattice": "d3q19", "nx": int(nx), "ny": int(ny), "nz": int(nz),
            "periodic": tuple(bool(p) for p in periodic), "G12": float(G12),
            "Gw": (float(Gw[0]), float(Gw[1])), "nu": (float(nu[0]), float(nu[1])), "s_e": float(s_e),
            "s_q": float(s_q), "s_eps_mode": int(s_eps_mode), "body": tuple(float(b) for b in body),
            "faces": []}


def random_box3(nx, ny, nz, seed, periodic=(1, 1, 1), solid_frac=0.0, G12=1.0, Gw=(0.0, 0.0),
                nu=(0.1, 0.2), u_amp=0.02, rho_lo=0.2, rho_hi=1.0) -> Workload:
    """Small random 3D state for invariants and parity on ragged grids."""
    rng = np.random.default_rng(seed)
    cfg = _base_cfg3(nx, ny, nz, periodic, G12, Gw, nu)
    solid = (rng.random((nz, ny, nx)) < solid_frac).astype(np.uint8)
    rho = rng.uniform(rho_lo, rho_hi, size=(2, nz, ny, nx))
    u = rng.uniform(-u_amp, u_amp, size=(3, nz, ny, nx))
    rho[:, solid != 0] = 0.0
    u[:, solid != 0] = 0.0
    return Workload("random3_%dx%dx%d" % (nx, ny, nz), cfg, solid, rho, u, 0, {})


def laplace3(n=32, R=8.0, G12=3.0, nu=(1.0 / 6, 1.0 / 6), seed=2512011, noise=1e-4, width=0.0) -> Workload:
    """Static droplet in a fully periodic cube (3D Laplace test)."""
    rng = np.random.default_rng(seed)
    z, y, x = np.mgrid[0:n, 0:n, 0:n].astype(np.float64)
    c = n / 2.0
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    phi = 0.5 * (1.0 - np.tanh(2.0 * (r - R) / width)) if width > 0 else (r <= R).astype(np.float64)
    rho = np.empty((2, n, n, n))
    rho[0] = FLOOR + (1.0 - FLOOR) * phi
    rho[1] = FLOOR + (1.0 - FLOOR) * (1.0 - phi)
    if noise:
        rho += rng.uniform(-noise, noise, size=rho.shape)
    cfg = _base_cfg3(n, n, n, (1, 1, 1), G12, (0.0, 0.0), nu)
    return Workload("laplace3_%d_R%g" % (n, R), cfg, None, rho, np.zeros((3, n, n, n)), 0, {"R": R})


def slit3(nx=4, half=8, nz=4, Fb=1e-6, nu=1.0 / 6) -> Workload:
    """Single-phase flow between two walls (solid planes y = 0 and y = ny-1)
    driven by a body force along x, periodic in x and z; the halfway walls
    sit at y = 1/2 and y = ny - 3/2."""
    ny = 2 * half + 2
    solid = np.zeros((nz, ny, nx), dtype=np.uint8)
    solid[:, 0, :] = 1
    solid[:, ny - 1, :] = 1
    cfg = _base_cfg3(nx, ny, nz, (1, 0, 1), 0.0, (0.0, 0.0), (nu, nu), body=(Fb, 0.0, 0.0))
    rho = np.zeros((2, nz, ny, nx))
    rho[0] = 1.0
    rho[1] = FLOOR
    rho[:, solid != 0] = 0.0
    return Workload("slit3", cfg, solid, rho, np.zeros((3, nz, ny, nx)), 0, {"H": ny - 2, "Fb": Fb, "nu": nu})


def _duct_profile(ny, nz, u_max):
    """Product of parabolas over the open cross-section y, z in [1, n-2]
    (halfway walls at 1/2 and n-3/2), zero on the wall layers; [nz][ny]."""
    def par(n):
        H = n - 2
        t = np.arange(n, dtype=np.float64)
        p = 4.0 * (t - 0.5) * (H + 0.5 - t) / (H * H)
        p[0] = p[-1] = 0.0
        return p
    return u_max * np.outer(par(nz), par(ny))


def duct3(nx=24, ny=10, nz=9, R=3.0, xc=8.0, u_max=0.01, G12=1.6, Gw=(0.2, -0.2), nu=(1.0 / 10, 1.0 / 6),
          alpha=True, chi=True, droplet=True, width=3.0, periodic_z=False) -> Workload:
    """Droplet in a duct along x: solid layers at y = 0, ny-1 (and z = 0,
    nz-1 unless periodic_z), velocity inlet on x = 0 and convective outlet
    on x = nx-1 over the whole open cross-section."""
    solid = np.zeros((nz, ny, nx), dtype=np.uint8)
    solid[:, 0, :] = 1
    solid[:, ny - 1, :] = 1
    if not periodic_z:
        solid[0, :, :] = 1
        solid[nz - 1, :, :] = 1
    cfg = _base_cfg3(nx, ny, nz, (0, 0, int(periodic_z)), G12, Gw, nu)
    prof = _duct_profile(ny, nz, u_max)
    if periodic_z:
        H = ny - 2
        t = np.arange(ny, dtype=np.float64)
        p = 4.0 * (t - 0.5) * (H + 0.5 - t) / (H * H)
        p[0] = p[-1] = 0.0
        prof = u_max * np.outer(np.ones(nz), p)
    cfg["faces"] = [
        {"kind": "inlet", "side": "xmin", "lo": (0, 0), "hi": (ny - 1, nz - 1), "rho_in": (FLOOR, 1.0),
         "alpha": int(alpha), "chi": 0, "profile": prof},
        {"kind": "outlet", "side": "xmax", "lo": (0, 0), "hi": (ny - 1, nz - 1), "rho_in": (0.0, 0.0),
         "alpha": 0, "chi": int(chi), "profile": np.zeros((nz, ny))},
    ]
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((x - xc) ** 2 + (y - (ny - 1) / 2.0) ** 2 + (z - (nz - 1) / 2.0) ** 2)
    phi = 0.5 * (1.0 - np.tanh(2.0 * (r - R) / width)) if droplet else np.zeros_like(r)
    rho = np.empty((2, nz, ny, nx))
    rho[0] = FLOOR + (1.0 - FLOOR) * phi
    rho[1] = FLOOR + (1.0 - FLOOR) * (1.0 - phi)
    u = np.zeros((3, nz, ny, nx))
    u[0] = prof[:, :, None]
    rho[:, solid != 0] = 0.0
    u[:, solid != 0] = 0.0
    return Workload("duct3_%dx%dx%d" % (nx, ny, nz), cfg, solid, rho, u, 0, {"u_max": u_max})


def coflow3(nx=512, ny=96, nz=96, r_in=12, wall=2, r_out=46, nozzle=48, q_ratio=0.5, M=0.2, G12=1.2,
            Gw=(0.2, -0.2), u_c=0.01, nu_c=1.0 / 6) -> Workload:
    """Coaxial co-flow droplet generator (Sec. III D, Fig. 10): a tube of
    radius r_out along x; a nozzle (solid shell r_in < r <= r_in + wall)
    from x = 0 to x = nozzle; the dispersed phase (component 1) enters
    through the nozzle bore (r <= r_in), the continuous phase (component 2)
    through the annulus.  One velocity inlet covers x = 0 (per-node speed
    and composition), one convective outlet covers x = nx-1.  Pipe-flow
    profiles: Poiseuille in the bore, the annular Poiseuille profile in the
    annulus, scaled so the dispersed/continuous flow-rate ratio is q_ratio
    and the continuous peak speed is u_c.  G12 defaults to 1.2: with the
    derived 3D interaction weights this device diverges within 250 steps at
    G12 >= 2.0 and within ~1000 steps at 1.6 (with wall adhesion), and stays
    finite for >= 3000 steps at 1.2 over M in {0.2, 1}, u_c in {0.005, 0.01}
    and G_w in {0, 0.2}."""
    cy, cz = (ny - 1) / 2.0, (nz - 1) / 2.0
    z, y = np.mgrid[0:nz, 0:ny].astype(np.float64)
    r = np.sqrt((y - cy) ** 2 + (z - cz) ** 2)
    sect_solid = r > r_out
    shell = (r > r_in) & (r <= r_in + wall)
    solid = np.zeros((nz, ny, nx), dtype=np.uint8)
    solid[:, :, :] = sect_solid[:, :, None]
    solid[:, :, :nozzle] |= shell[:, :, None]
    bore = r <= r_in
    ann = (r > r_in + wall) & (r <= r_out)
    a, b = r_in + wall, r_out
    # annular Poiseuille: u ~ (b^2 - r^2) + (b^2 - a^2) ln(r/b) / ln(b/a)
    ua = np.where(ann, (b * b - r * r) + (b * b - a * a) * np.log(np.maximum(r, 1e-12) / b) / np.log(b / a), 0.0)
    ua = u_c * ua / ua.max()
    ub = np.where(bore, 1.0 - (r / (r_in + 0.5)) ** 2, 0.0)
    ub *= q_ratio * ua.sum() / ub.sum()
    prof = ua + ub
    rprof = np.stack([np.where(bore, 1.0, FLOOR), np.where(bore, FLOOR, 1.0)])
    cfg = _base_cfg3(nx, ny, nz, (0, 0, 0), G12, Gw, (M * nu_c, nu_c))
    cfg["faces"] = [
        {"kind": "inlet", "side": "xmin", "lo": (0, 0), "hi": (ny - 1, nz - 1), "rho_in": (FLOOR, 1.0),
         "alpha": 1, "chi": 0, "profile": prof, "rho_profile": rprof},
        {"kind": "outlet", "side": "xmax", "lo": (0, 0), "hi": (ny - 1, nz - 1), "rho_in": (0.0, 0.0),
         "alpha": 0, "chi": 1, "profile": np.zeros((nz, ny))},
    ]
    xx = np.arange(nx, dtype=np.float64)
    front = 0.5 * (1.0 - np.tanh((xx - nozzle) / 2.0))      # dispersed phase fills the bore up to the tip
    phi = bore[:, :, None] * front[None, None, :]
    rho = np.empty((2, nz, ny, nx))
    rho[0] = FLOOR + (1.0 - FLOOR) * phi
    rho[1] = FLOOR + (1.0 - FLOOR) * (1.0 - phi)
    u = np.zeros((3, nz, ny, nx))
    u[0] = (ua + ub)[:, :, None]
    rho[:, solid != 0] = 0.0
    u[:, solid != 0] = 0.0
    return Workload("coflow3_%dx%dx%d" % (nx, ny, nz), cfg, solid, rho, u, 0,
                    {"r_in": r_in, "r_out": r_out, "nozzle": nozzle, "q_ratio": q_ratio, "M": M, "u_c": u_c})
