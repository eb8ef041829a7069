"""FP64 CPU oracle of the D3Q19 variant: Python front end over
lbm_oracle_3d.c.

TEST INFRASTRUCTURE (same rules as oracle.py: only tests/, smoke() and
bench.py's CPU legs may use it; it never imports the product).

The paper prints only 2D operators; the 3D readings (lattice order, the
19-moment basis, the 3D-only relaxation rates, the derived 8th-order 3D
interaction weights, the 5-unknown open faces) are stated in the C file's
header.  Every other reading of oracle.py carries over unchanged.

Fields are numpy arrays indexed [component or axis][z][y][x].  A face dict
has kind ('inlet'/'outlet'), side ('xmin'..'zmax'), lo/hi (pairs over the
two tangential axes in x, y, z order), rho_in, alpha, chi, profile (normal
speed per face position, shape [len1][len0]) and optionally rho_profile
(composition per face position, shape [2][len1][len0]).
"""
import ctypes

import numpy as np

from . import build as _build

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
SIDES = {"xmin": 0, "xmax": 1, "ymin": 2, "ymax": 3, "zmin": 4, "zmax": 5}
KINDS = {"inlet": 1, "outlet": 2}


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("periodic", ctypes.c_int * 3), ("G12", ctypes.c_double), ("Gw", ctypes.c_double * 2),
                ("nu", ctypes.c_double * 2), ("s_e", ctypes.c_double), ("s_q", ctypes.c_double),
                ("s_eps_mode", ctypes.c_int), ("body", ctypes.c_double * 3)]


class _Face(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("side", ctypes.c_int), ("lo", ctypes.c_int * 2),
                ("hi", ctypes.c_int * 2), ("rho_in", ctypes.c_double * 2), ("alpha_on", ctypes.c_int),
                ("chi_on", ctypes.c_int)]


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build.build())
        L.orc3_create.restype = ctypes.c_void_p
        L.orc3_create.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, ctypes.POINTER(_Face),
                                  ctypes.POINTER(_dp), ctypes.POINTER(_dp), ctypes.c_void_p, _dp, _dp]
        L.orc3_destroy.argtypes = [ctypes.c_void_p]
        L.orc3_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc3_set_threads.argtypes = [ctypes.c_void_p, ctypes.c_int]
        for name in ("orc3_get_f", "orc3_set_f", "orc3_get_scalars", "orc3_get_fpost", "orc3_get_force_prev"):
            getattr(L, name).argtypes = [ctypes.c_void_p, _dp]
        L.orc3_get_macros.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
        L.orc3_eval_forces.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.orc3_feq.argtypes = [ctypes.c_double] * 4 + [_dp]
        L.orc3_fbar.argtypes = [ctypes.c_double] * 6 + [_dp]
        L.orc3_collide.argtypes = [_dp, ctypes.c_double, _dp, _dp, _dp, _dp]
        L.orc3_moment_matrix.argtypes = [_dp, _dp]
        ip = ctypes.POINTER(ctypes.c_int)
        L.orc3_lattice.argtypes = [ip, ip, ip, _dp, ip]
        L.orc3_stencil.restype = ctypes.c_int
        L.orc3_stencil.argtypes = [ip, ip, ip, _dp]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dp)


def feq(rho, u):
    out = np.zeros(19)
    lib().orc3_feq(rho, u[0], u[1], u[2], _ptr(out))
    return out


def fbar(u, F):
    out = np.zeros(19)
    lib().orc3_fbar(u[0], u[1], u[2], F[0], F[1], F[2], _ptr(out))
    return out


def collide(f, rho, u, F, s):
    f = np.ascontiguousarray(f, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    out = np.zeros(19)
    lib().orc3_collide(_ptr(f), rho, _ptr(u), _ptr(F), _ptr(s), _ptr(out))
    return out


def moment_matrix():
    T = np.zeros(361)
    Ti = np.zeros(361)
    lib().orc3_moment_matrix(_ptr(T), _ptr(Ti))
    return T.reshape(19, 19), Ti.reshape(19, 19)


def lattice():
    ex, ey, ez, opp = [(ctypes.c_int * 19)() for _ in range(4)]
    w = np.zeros(19)
    lib().orc3_lattice(ex, ey, ez, _ptr(w), opp)
    return np.array(ex[:]), np.array(ey[:]), np.array(ez[:]), w, np.array(opp[:])


def stencil():
    dx, dy, dz = [(ctypes.c_int * 92)() for _ in range(3)]
    w = np.zeros(92)
    n = lib().orc3_stencil(dx, dy, dz, _ptr(w))
    return np.array(dx[:n]), np.array(dy[:n]), np.array(dz[:n]), w[:n]


class Oracle3D:
    """FP64 D3Q19 two-component solver state (cfg keys as Oracle2D, with
    nz, three periodic flags, a 3-vector body force and 3D faces)."""

    def __init__(self, cfg, solid, rho_init, u_init=None, threads=1):
        L = lib()
        nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        p = _Params()
        p.nx, p.ny, p.nz = nx, ny, nz
        per = cfg.get("periodic", (0, 0, 0))
        for a in range(3):
            p.periodic[a] = int(per[a])
        p.G12 = cfg.get("G12", 0.0)
        gw = cfg.get("Gw", (0.0, 0.0))
        p.Gw[0], p.Gw[1] = gw
        p.nu[0], p.nu[1] = cfg["nu"]
        p.s_e = cfg.get("s_e", 0.0)
        p.s_q = cfg.get("s_q", 1.2)
        p.s_eps_mode = int(cfg.get("s_eps_mode", 1))
        b = cfg.get("body", (0.0, 0.0, 0.0))
        for a in range(3):
            p.body[a] = b[a] if a < len(b) else 0.0
        faces = cfg.get("faces", [])
        FA = (_Face * max(1, len(faces)))()
        PP = (_dp * max(1, len(faces)))()
        RP = (_dp * max(1, len(faces)))()
        keep = []
        for j, fc in enumerate(faces):
            FA[j].kind = KINDS[fc["kind"]]
            FA[j].side = SIDES[fc["side"]]
            FA[j].lo[0], FA[j].lo[1] = fc["lo"]
            FA[j].hi[0], FA[j].hi[1] = fc["hi"]
            r = fc.get("rho_in", (0.0, 0.0))
            FA[j].rho_in[0], FA[j].rho_in[1] = r
            FA[j].alpha_on = int(fc.get("alpha", 1))
            FA[j].chi_on = int(fc.get("chi", 1))
            n = (fc["hi"][0] - fc["lo"][0] + 1) * (fc["hi"][1] - fc["lo"][1] + 1)
            prof = np.ascontiguousarray(fc.get("profile", np.zeros(n)), dtype=np.float64).reshape(-1)
            keep.append(prof)
            PP[j] = _ptr(prof)
            if fc.get("rho_profile") is not None:
                rp = np.ascontiguousarray(fc["rho_profile"], dtype=np.float64).reshape(-1)
                keep.append(rp)
                RP[j] = _ptr(rp)
        sol = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
        rho = np.ascontiguousarray(rho_init, dtype=np.float64).reshape(-1)
        uu = None if u_init is None else np.ascontiguousarray(u_init, dtype=np.float64).reshape(-1)
        self._keep = (keep, FA, PP, RP, sol, rho, uu)
        h = L.orc3_create(ctypes.byref(p), len(faces), FA, PP, RP,
                          None if sol is None else sol.ctypes.data_as(ctypes.c_void_p), _ptr(rho),
                          None if uu is None else _ptr(uu))
        if not h:
            raise ValueError("oracle rejected the configuration")
        self.h = h
        L.orc3_set_threads(h, int(threads))

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc3_destroy(self.h)
            self.h = None

    def step(self, n=1):
        lib().orc3_step(self.h, int(n))

    def macros(self):
        rho, u, F = np.zeros(2 * self.N), np.zeros(3 * self.N), np.zeros(6 * self.N)
        lib().orc3_get_macros(self.h, _ptr(rho), _ptr(u), _ptr(F))
        return rho.reshape(2, *self.shape), u.reshape(3, *self.shape), F.reshape(2, 3, *self.shape)

    def f(self):
        out = np.zeros(38 * self.N)
        lib().orc3_get_f(self.h, _ptr(out))
        return out.reshape(2, 19, *self.shape)

    def fpost(self):
        out = np.zeros(38 * self.N)
        lib().orc3_get_fpost(self.h, _ptr(out))
        return out.reshape(2, 19, *self.shape)

    def force_prev(self):
        out = np.zeros(6 * self.N)
        lib().orc3_get_force_prev(self.h, _ptr(out))
        return out.reshape(2, 3, *self.shape)

    def set_f(self, f):
        a = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        lib().orc3_set_f(self.h, _ptr(a))

    def scalars(self):
        out = np.zeros(8 + 38)
        lib().orc3_get_scalars(self.h, _ptr(out))
        return {"lambda": out[0], "chi": out[1], "Qin": out[2], "Qout": out[3], "Umean": out[4],
                "mass": out[5:7].copy(), "step": int(out[7]), "s": out[8:].reshape(2, 19).copy()}

    def eval_forces(self, psi):
        a = np.ascontiguousarray(psi, dtype=np.float64).reshape(-1)
        out = np.zeros(6 * self.N)
        lib().orc3_eval_forces(self.h, _ptr(a), _ptr(out))
        return out.reshape(2, 3, *self.shape)
