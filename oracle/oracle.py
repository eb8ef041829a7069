"""FP64 CPU oracle: Python front end over the plain C restatement.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The product path (the CUDA library and its binding) never does, and
this module never imports the product.  The only code both sides share is the
seeded input generator module, which holds no arithmetic of the method.

What is computed (paper, Sec. II and App. B): one time step of the
two-component MRT pseudopotential LBM with corrected open boundaries, in
FP64, with naive loops and dense 9x9 moment transforms (lbm_oracle.c).

Readings taken where the paper is silent, garbled or inconsistent:

 1. Eq. 3 (T): rows 3-8 as printed are singular; T is the standard
    orthogonal D2Q9 moment basis in the order of Eq. 4 (rho, e, eps, j_x,
    q_x, j_y, q_y, p_xx, p_xy).  Rows 0-2 equal the printed ones.
 2. Eq. 6: the quadratic term is (e.u)^2 / (2 c_s^4) (second-order
    equilibrium), not over 2 c_s^2.
 3. Eq. 10: psi_k(x) times the OTHER component's psi at x+e (fluid-fluid
    interaction "between different components"), summed over the 24
    vectors with |e|^2 in {1,2,4,5,8}.
 4. Eq. 26 prints s_q = 1.0 and 1.2; both q rates take one value s_q
    (default 1.2).  s_e defaults to s_nu,k.  s_eps = 1/(3 max nu + 1/2)
    ("adjusted based on the phase with the highest viscosity", Sec. III A);
    the unadjusted scheme uses each component's own s_nu,k.
 5. Eq. 12 (G_w interpolation) depends on quantities the paper does not
    define (rho^e, delta, g1, g2).  By default G_w,k is a constant per
    component.  With cfg["wetting_delta"] = delta > 0 one coefficient
    G_w(rho^e) acts on both components, rho^e = (rho_1 - rho_2)/(rho_1 +
    rho_2): G_w,1 for rho^e > delta, G_w,2 for rho^e < -delta, and the
    linear pieces G_w,1 rho^e/delta on (0, delta], -G_w,2 rho^e/delta on
    (-delta, 0] between them (zero on the interface itself).
 6. psi = 0 on solid nodes; wettability enters only through Eq. 11.
    Outside a closed (non-periodic, non-open) edge the lattice is solid.
 7. Eq. 10 is used with the printed weights as is (their second moment
    is 1); the G12 of a configuration is used as given.
 8. Eq. 19: alpha_i = w_i [e_ix D_x / sum_U e_x^2 w + e_iy D_y / sum_U e_y^2 w]
    with D = rho_in,k u_in - (sum_i e_i f_i + F_k/2) after Eq. 13.  Density
    is not re-imposed after the correction.  F_k at x1 and at x2 (and in
    the u^eq(x2) of Eq. 13) is the force of the previous step at that node.
 9. lambda (Eq. 21) and chi (Eq. 23) are computed from the fields of the
    previous step (one-step lag); lambda is the mean of u^eq.n over the
    fluid nodes of column x_{N-1}, clamped at >= 0; chi = Q_in / Q_out with
    Q over (rho_1 + rho_2) u^eq.n; chi = 1 when |Q_out| < 1e-14 or there
    is no inlet.  lambda = 0 and chi = 1 before the first step.  With
    cfg["chi_same_step"] = 1, chi is taken from the step's own velocities
    (t + dt, as Eq. 23 prints it) just before Eq. 22 uses it; lambda cannot
    be (Eq. 20 needs it before the step's velocities exist) and stays
    lagged.
10. Eq. 22 overwrites the outlet node's normal component of u^eq (the
    velocity the collision uses) with chi times that of x_{N-1}, same row;
    the tangential component is kept.
11. Eq. 20's f_i(x_N, t) is the post-boundary population of the previous
    step (the initial f before the first step).
12. Ghost layers (Eqs. 24, 25) mirror across every side that carries an
    open face: x = -1 -> x1, x = -2 -> x2, and likewise at the far side.
13. Initial state f = feq(rho_k, u_init); the macroscopic fields reported
    after n steps are those the n-th collision used.
14. Moving walls (the Taylor deformation test of Sec. III A shears a
    droplet between plates moving in opposite directions; the paper does not
    give the wall scheme): cfg["wall_ux"] = (u_bottom, u_top) moves the
    walls beyond the closed edges y = 0 and y = ny - 1 along x.  A
    population reflected there gains 2 w_i rho_k (e_i . u_w) / c_s^2, with
    rho_k the node's own density (sum of its post-collision populations).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("periodic_x", ctypes.c_int), ("periodic_y", ctypes.c_int),
        ("G12", ctypes.c_double), ("Gw", ctypes.c_double * 2), ("nu", ctypes.c_double * 2),
        ("s_e", ctypes.c_double), ("s_q", ctypes.c_double), ("s_eps_mode", ctypes.c_int),
        ("body", ctypes.c_double * 2), ("use_s_full", ctypes.c_int),
        ("s_full", (ctypes.c_double * 9) * 2), ("chi_same_step", ctypes.c_int),
        ("wall_ux", ctypes.c_double * 2), ("wet_interp", ctypes.c_int), ("wet_delta", ctypes.c_double),
    ]


class _Face(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int), ("side", ctypes.c_int), ("lo", ctypes.c_int), ("hi", ctypes.c_int),
        ("rho_in", ctypes.c_double * 2), ("alpha_on", ctypes.c_int), ("chi_on", ctypes.c_int),
    ]


SIDES = {"xmin": 0, "xmax": 1, "ymin": 2, "ymax": 3}
KINDS = {"inlet": 1, "outlet": 2}

_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, ctypes.POINTER(_Face),
                                 ctypes.POINTER(_dp), ctypes.c_void_p, _dp, _dp]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_set_threads.argtypes = [ctypes.c_void_p, ctypes.c_int]
        for name in ("orc_get_f", "orc_set_f", "orc_get_fpost", "orc_set_fpost", "orc_get_force_prev",
                     "orc_get_scalars"):
            getattr(L, name).argtypes = [ctypes.c_void_p, _dp]
        L.orc_get_macros.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
        L.orc_set_outlet_coeffs.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
        L.orc_eval_forces.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.orc_feq.argtypes = [ctypes.c_double] * 3 + [_dp]
        L.orc_fbar.argtypes = [ctypes.c_double] * 4 + [_dp]
        L.orc_collide.argtypes = [_dp] + [ctypes.c_double] * 5 + [_dp, _dp]
        L.orc_moment_matrix.argtypes = [_dp, _dp]
        L.orc_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _dp,
                                  ctypes.POINTER(ctypes.c_int)]
        L.orc_stencil.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _dp]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dp)


# ---- single-node building blocks ------------------------------------------

def feq(rho, ux, uy):
    out = np.zeros(9)
    lib().orc_feq(rho, ux, uy, _ptr(out))
    return out


def fbar(ux, uy, Fx, Fy):
    out = np.zeros(9)
    lib().orc_fbar(ux, uy, Fx, Fy, _ptr(out))
    return out


def collide(f, rho, ux, uy, Fx, Fy, s):
    f = np.ascontiguousarray(f, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    out = np.zeros(9)
    lib().orc_collide(_ptr(f), rho, ux, uy, Fx, Fy, _ptr(s), _ptr(out))
    return out


def moment_matrix():
    T = np.zeros(81)
    Ti = np.zeros(81)
    lib().orc_moment_matrix(_ptr(T), _ptr(Ti))
    return T.reshape(9, 9), Ti.reshape(9, 9)


def lattice():
    ex = (ctypes.c_int * 9)()
    ey = (ctypes.c_int * 9)()
    opp = (ctypes.c_int * 9)()
    w = np.zeros(9)
    lib().orc_lattice(ex, ey, _ptr(w), opp)
    return np.array(ex[:]), np.array(ey[:]), w, np.array(opp[:])


def stencil():
    dx = (ctypes.c_int * 24)()
    dy = (ctypes.c_int * 24)()
    w = np.zeros(24)
    lib().orc_stencil(dx, dy, _ptr(w))
    return np.array(dx[:]), np.array(dy[:]), w


# ---- full solver ---------------------------------------------------------------

class Oracle2D:
    """FP64 D2Q9 two-component solver state.

    cfg keys: nx, ny, periodic (px, py), G12, Gw (2), nu (2), s_e, s_q,
    s_eps_mode, body (2), s_full (2x9 or None), faces (list of dicts with
    kind, side, lo, hi, rho_in, alpha, chi, profile).
    Fields are numpy arrays indexed [component][y][x].
    """

    def __init__(self, cfg, solid, rho_init, u_init=None, threads=1):
        L = lib()
        nx, ny = cfg["nx"], cfg["ny"]
        self.nx, self.ny, self.N = nx, ny, nx * ny
        p = _Params()
        p.nx, p.ny = nx, ny
        p.periodic_x, p.periodic_y = [int(v) for v in cfg.get("periodic", (0, 0))[:2]]
        p.G12 = cfg.get("G12", 0.0)
        gw = cfg.get("Gw", (0.0, 0.0))
        p.Gw[0], p.Gw[1] = gw[0], gw[1]
        nu = cfg["nu"]
        p.nu[0], p.nu[1] = nu[0], nu[1]
        p.s_e = cfg.get("s_e", 0.0)
        p.s_q = cfg.get("s_q", 1.2)
        p.s_eps_mode = int(cfg.get("s_eps_mode", 1))
        body = cfg.get("body", (0.0, 0.0))
        p.body[0], p.body[1] = body[0], body[1]
        p.chi_same_step = int(cfg.get("chi_same_step", 0))
        wet = cfg.get("wetting_delta")
        p.wet_interp = 1 if wet else 0
        p.wet_delta = float(wet) if wet else 1.0
        wu = cfg.get("wall_ux", (0.0, 0.0))
        p.wall_ux[0], p.wall_ux[1] = float(wu[0]), float(wu[1])
        sf = cfg.get("s_full")
        if sf is not None:
            p.use_s_full = 1
            for k in range(2):
                for r in range(9):
                    p.s_full[k][r] = float(sf[k][r])
        faces = cfg.get("faces", [])
        FA = (_Face * max(1, len(faces)))()
        prof_arrays = []
        PP = (_dp * max(1, len(faces)))()
        for j, fc in enumerate(faces):
            FA[j].kind = KINDS[fc["kind"]]
            FA[j].side = SIDES[fc["side"]]
            FA[j].lo, FA[j].hi = fc["lo"], fc["hi"]
            r = fc.get("rho_in", (0.0, 0.0))
            FA[j].rho_in[0], FA[j].rho_in[1] = r[0], r[1]
            FA[j].alpha_on = int(fc.get("alpha", 1))
            FA[j].chi_on = int(fc.get("chi", 1))
            prof = np.ascontiguousarray(fc.get("profile", np.zeros(fc["hi"] - fc["lo"] + 1)),
                                        dtype=np.float64)
            prof_arrays.append(prof)
            PP[j] = _ptr(prof)
        self._keep = (prof_arrays, FA, PP)
        sol = None
        if solid is not None:
            sol = np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
            self._sol = sol
        rho = np.ascontiguousarray(rho_init, dtype=np.float64).reshape(-1)
        uu = None if u_init is None else np.ascontiguousarray(u_init, dtype=np.float64).reshape(-1)
        self._init = (rho, uu)
        h = L.orc_create(ctypes.byref(p), len(faces), FA, PP,
                         None if sol is None else sol.ctypes.data_as(ctypes.c_void_p),
                         _ptr(rho), None if uu is None else _ptr(uu))
        if not h:
            raise ValueError("oracle rejected the configuration")
        self.h = h
        L.orc_set_threads(h, int(threads))

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def set_threads(self, n):
        lib().orc_set_threads(self.h, int(n))

    def step(self, n=1):
        lib().orc_step(self.h, int(n))

    def macros(self):
        rho = np.zeros(2 * self.N)
        u = np.zeros(2 * self.N)
        F = np.zeros(4 * self.N)
        lib().orc_get_macros(self.h, _ptr(rho), _ptr(u), _ptr(F))
        return (rho.reshape(2, self.ny, self.nx), u.reshape(2, self.ny, self.nx),
                F.reshape(2, 2, self.ny, self.nx))

    def f(self):
        out = np.zeros(18 * self.N)
        lib().orc_get_f(self.h, _ptr(out))
        return out.reshape(2, 9, self.ny, self.nx)

    def set_f(self, f):
        a = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        lib().orc_set_f(self.h, _ptr(a))

    def fpost(self):
        out = np.zeros(18 * self.N)
        lib().orc_get_fpost(self.h, _ptr(out))
        return out.reshape(2, 9, self.ny, self.nx)

    def set_fpost(self, f):
        """Replace the last step's post-boundary populations (the f(x_N, t)
        that the next step's Eq. 20 reads)."""
        a = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        lib().orc_set_fpost(self.h, _ptr(a))

    def set_outlet_coeffs(self, lam, chi):
        """Replace lambda and chi that the next step uses."""
        lib().orc_set_outlet_coeffs(self.h, float(lam), float(chi))

    def force_prev(self):
        out = np.zeros(4 * self.N)
        lib().orc_get_force_prev(self.h, _ptr(out))
        return out.reshape(2, 2, self.ny, self.nx)

    def scalars(self):
        out = np.zeros(8 + 18)
        lib().orc_get_scalars(self.h, _ptr(out))
        return {"lambda": out[0], "chi": out[1], "Qin": out[2], "Qout": out[3],
                "Umean": out[4], "mass": out[5:7].copy(), "step": int(out[7]),
                "s": out[8:].reshape(2, 9).copy()}

    def eval_forces(self, psi):
        a = np.ascontiguousarray(psi, dtype=np.float64).reshape(-1)
        out = np.zeros(4 * self.N)
        lib().orc_eval_forces(self.h, _ptr(a), _ptr(out))
        return out.reshape(2, 2, self.ny, self.nx)


def pressure(rho, G12):
    """Bulk pressure implied by Eq. 10 with weights of unit second moment:
    p = c_s^2 (rho_1 + rho_2) + G12 psi_1 psi_2 (psi = rho)."""
    return (rho[0] + rho[1]) / 3.0 + G12 * rho[0] * rho[1]
