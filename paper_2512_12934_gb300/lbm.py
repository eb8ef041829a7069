"""Thin ctypes binding of liblbm.so (include/lbm.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Loading fails loudly when the library is missing; there is
no CPU fallback.
"""
import ctypes
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "liblbm.so")

LBM_OK = 0
STATUS = {0: "LBM_OK", 1: "LBM_ERR_INVALID_ARG", 2: "LBM_ERR_CUDA", 3: "LBM_ERR_OOM",
          4: "LBM_ERR_DIVERGED", 5: "LBM_ERR_TIMEOUT", 6: "LBM_ERR_UNSUPPORTED", 7: "LBM_ERR_IO"}
LBM_D2Q9, LBM_D3Q19 = 0, 1
LBM_FP32, LBM_FP32_FP16STORE, LBM_FP64 = 0, 1, 2
PRECISIONS = {"fp32": LBM_FP32, "fp16store": LBM_FP32_FP16STORE, "fp64": LBM_FP64}
LBM_INLET_VELOCITY, LBM_OUTLET_CONVECTIVE = 1, 2
SCHEDULES = {"graphs": 0, "persistent": 1, "graphs_early": 2}
SCHEDULE_NAMES = {v: k for k, v in SCHEDULES.items()}
SIDES = {"xmin": 0, "xmax": 1, "ymin": 2, "ymax": 3, "zmin": 4, "zmax": 5}


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class lbm_grid(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("periodic", ctypes.c_int * 3)]


class lbm_params(ctypes.Structure):
    _fields_ = [("G12", ctypes.c_double), ("Gw", ctypes.c_double * 2), ("nu", ctypes.c_double * 2),
                ("s_e", ctypes.c_double), ("s_q", ctypes.c_double), ("s_eps_mode", ctypes.c_int),
                ("body_force", ctypes.c_double * 3), ("precision", ctypes.c_int),
                ("rho0_store", ctypes.c_double)]


class lbm_open_bc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("side", ctypes.c_int), ("lo", ctypes.c_int * 2),
                ("hi", ctypes.c_int * 2), ("u_profile", ctypes.POINTER(ctypes.c_double)),
                ("rho_in", ctypes.c_double * 2), ("alpha_correction", ctypes.c_int),
                ("chi_correction", ctypes.c_int), ("rho_profile", ctypes.POINTER(ctypes.c_double))]


class lbm_diag(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double * 2), ("lambda_", ctypes.c_double), ("chi", ctypes.c_double),
                ("q_in", ctypes.c_double), ("q_out", ctypes.c_double), ("max_speed", ctypes.c_double),
                ("step", ctypes.c_int64), ("launches", ctypes.c_int64), ("status", ctypes.c_int)]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)


def load():
    """Load liblbm.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    if not _build.up_to_date():
        _build.build()
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("liblbm.so is missing and could not be built: no CUDA path available")
    L = ctypes.CDLL(LIB_PATH)
    c_ctx = ctypes.c_void_p
    L.lbm_create.restype = ctypes.c_int
    L.lbm_create.argtypes = [ctypes.POINTER(lbm_grid), ctypes.POINTER(lbm_params), ctypes.POINTER(lbm_open_bc),
                             ctypes.c_int, ctypes.c_void_p, _dp, _dp, ctypes.c_void_p, ctypes.POINTER(c_ctx)]
    L.lbm_step.restype = ctypes.c_int
    L.lbm_step.argtypes = [c_ctx, ctypes.c_int64]
    L.lbm_reset.restype = ctypes.c_int
    L.lbm_reset.argtypes = [c_ctx, _dp, _dp]
    L.lbm_sync.restype = ctypes.c_int
    L.lbm_sync.argtypes = [c_ctx]
    L.lbm_get_macros.restype = ctypes.c_int
    L.lbm_get_macros.argtypes = [c_ctx, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    L.lbm_get_macros_f64.restype = ctypes.c_int
    L.lbm_get_macros_f64.argtypes = [c_ctx, _dp, _dp]
    L.lbm_get_populations.restype = ctypes.c_int
    L.lbm_get_populations.argtypes = [c_ctx, _dp]
    L.lbm_set_populations.restype = ctypes.c_int
    L.lbm_set_populations.argtypes = [c_ctx, _dp]
    L.lbm_get_diagnostics.restype = ctypes.c_int
    L.lbm_get_diagnostics.argtypes = [c_ctx, ctypes.POINTER(lbm_diag)]
    L.lbm_save.restype = ctypes.c_int
    L.lbm_save.argtypes = [c_ctx, ctypes.c_char_p]
    L.lbm_load.restype = ctypes.c_int
    L.lbm_load.argtypes = [c_ctx, ctypes.c_char_p]
    L.lbm_destroy.restype = None
    L.lbm_destroy.argtypes = [c_ctx]
    L.lbm_last_error.restype = ctypes.c_char_p
    L.lbm_last_error.argtypes = [c_ctx]
    L.lbm_enable_kernel_timing.restype = ctypes.c_int
    L.lbm_enable_kernel_timing.argtypes = [c_ctx, ctypes.c_int]
    L.lbm_kernel_time.restype = ctypes.c_int
    L.lbm_kernel_time.argtypes = [c_ctx, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    L.lbm_kernel_time_split.restype = ctypes.c_int
    L.lbm_kernel_time_split.argtypes = [c_ctx, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int64)]
    L.lbm_set_tile_variant.restype = ctypes.c_int
    L.lbm_set_tile_variant.argtypes = [c_ctx, ctypes.c_int]
    L.lbm_num_tile_variants.restype = ctypes.c_int
    L.lbm_num_tile_variants.argtypes = []
    L.lbm_tile_stats.restype = ctypes.c_int
    L.lbm_tile_stats.argtypes = [c_ctx] + [ctypes.POINTER(ctypes.c_int)] * 3 + [ctypes.POINTER(ctypes.c_int64)] * 2
    L.lbm_set_graph_mode.restype = ctypes.c_int
    L.lbm_set_graph_mode.argtypes = [c_ctx, ctypes.c_int]
    L.lbm_set_wall_velocity.restype = ctypes.c_int
    L.lbm_set_wall_velocity.argtypes = [c_ctx, ctypes.c_int, ctypes.c_double]
    L.lbm_set_wetting.restype = ctypes.c_int
    L.lbm_set_wetting.argtypes = [c_ctx, ctypes.c_double]
    L.lbm_set_chi_timing.restype = ctypes.c_int
    L.lbm_set_chi_timing.argtypes = [c_ctx, ctypes.c_int]
    L.lbm_set_schedule.restype = ctypes.c_int
    L.lbm_set_schedule.argtypes = [c_ctx, ctypes.c_int]
    L.lbm_get_schedule.restype = ctypes.c_int
    L.lbm_get_schedule.argtypes = [c_ctx, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.lbm_mass_noalloc.restype = ctypes.c_int
    L.lbm_mass_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.lbm_batch_create.restype = ctypes.c_int
    L.lbm_batch_create.argtypes = [ctypes.POINTER(c_ctx), ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(c_ctx)]
    L.lbm_batch_set_schedule.restype = ctypes.c_int
    L.lbm_batch_set_schedule.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.lbm_batch_get_schedule.restype = ctypes.c_int
    L.lbm_batch_get_schedule.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.lbm_batch_persistent_grid.restype = ctypes.c_int
    L.lbm_batch_persistent_grid.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]
    L.lbm_batch_inject_barrier_fault.restype = ctypes.c_int
    L.lbm_batch_inject_barrier_fault.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64]
    L.lbm_batch_step.restype = ctypes.c_int
    L.lbm_batch_step.argtypes = [c_ctx, ctypes.c_int64]
    L.lbm_batch_sync.restype = ctypes.c_int
    L.lbm_batch_sync.argtypes = [c_ctx]
    L.lbm_batch_set_tile_variant.restype = ctypes.c_int
    L.lbm_batch_set_tile_variant.argtypes = [c_ctx, ctypes.c_int]
    L.lbm_batch_autotune.restype = ctypes.c_int
    L.lbm_batch_autotune.argtypes = [c_ctx, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    L.lbm_autotune.restype = ctypes.c_int
    L.lbm_autotune.argtypes = [c_ctx, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    L.lbm_batch_info.restype = ctypes.c_int
    L.lbm_batch_info.argtypes = [c_ctx] + [ctypes.POINTER(ctypes.c_int)] * 3 + [ctypes.POINTER(ctypes.c_int64)]
    L.lbm_batch_set_graph_mode.restype = ctypes.c_int
    L.lbm_batch_set_graph_mode.argtypes = [c_ctx, ctypes.c_int]
    L.lbm_batch_destroy.restype = None
    L.lbm_batch_destroy.argtypes = [c_ctx]
    L.lbm_batch_last_error.restype = ctypes.c_char_p
    L.lbm_batch_last_error.argtypes = [c_ctx]
    L.lbm_version.restype = ctypes.c_char_p
    L.lbm_version.argtypes = []
    c_mlp = ctypes.c_void_p
    L.lbm_mlp_num_params.restype = ctypes.c_int64
    L.lbm_mlp_num_params.argtypes = []
    L.lbm_mlp_create.restype = ctypes.c_int
    L.lbm_mlp_create.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER(c_mlp)]
    L.lbm_mlp_set_params.restype = ctypes.c_int
    L.lbm_mlp_set_params.argtypes = [c_mlp, _fp]
    L.lbm_mlp_get_params.restype = ctypes.c_int
    L.lbm_mlp_get_params.argtypes = [c_mlp, _fp]
    L.lbm_mlp_forward.restype = ctypes.c_int
    L.lbm_mlp_forward.argtypes = [c_mlp, _fp, ctypes.c_int, _fp]
    L.lbm_mlp_gradient.restype = ctypes.c_int
    L.lbm_mlp_gradient.argtypes = [c_mlp, _fp, _fp, ctypes.c_int, _fp]
    L.lbm_mlp_train.restype = ctypes.c_int
    L.lbm_mlp_train.argtypes = [c_mlp, _fp, _fp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                ctypes.c_uint64]
    L.lbm_mlp_predict.restype = ctypes.c_int
    L.lbm_mlp_predict.argtypes = [c_mlp, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    L.lbm_mlp_set_infer_path.restype = ctypes.c_int
    L.lbm_mlp_set_infer_path.argtypes = [c_mlp, ctypes.c_int]
    L.lbm_mlp_set_wait_limit.restype = ctypes.c_int
    L.lbm_mlp_set_wait_limit.argtypes = [c_mlp, ctypes.c_longlong]
    L.lbm_mlp_destroy.restype = None
    L.lbm_mlp_destroy.argtypes = [c_mlp]
    L.lbm_mlp_last_error.restype = ctypes.c_char_p
    L.lbm_mlp_last_error.argtypes = [c_mlp]
    _lib = L
    return L


def _check(status, ctx=None):
    if status != LBM_OK:
        msg = load().lbm_last_error(ctx)
        raise LbmError(status, msg.decode() if msg else "")


def _dptr(a):
    return a.ctypes.data_as(_dp)


class Solver:
    """One lbm_ctx built from a plain configuration dictionary (see
    paper_2512_12934_gb300.workloads for the keys)."""

    def __init__(self, cfg, solid, rho_init, u_init=None, precision="fp32", stream=None, rho0_store=1.0):
        L = load()
        three = cfg.get("lattice", "d2q9") == "d3q19"
        nx, ny, nz = cfg["nx"], cfg["ny"], cfg.get("nz", 1) if three else 1
        self.nx, self.ny, self.nz, self.N = nx, ny, nz, nx * ny * nz
        self.dim = 3 if three else 2
        self.Q = 19 if three else 9
        self.shape = (nz, ny, nx) if three else (ny, nx)
        g = lbm_grid()
        g.lattice = LBM_D3Q19 if three else LBM_D2Q9
        g.nx, g.ny, g.nz = nx, ny, nz
        per = tuple(cfg.get("periodic", (0, 0, 0))) + (0, 0, 0)
        g.periodic[0], g.periodic[1], g.periodic[2] = int(per[0]), int(per[1]), int(per[2]) if three else 0
        p = lbm_params()
        p.G12 = cfg.get("G12", 0.0)
        gw = cfg.get("Gw", (0.0, 0.0))
        p.Gw[0], p.Gw[1] = gw
        p.nu[0], p.nu[1] = cfg["nu"]
        p.s_e = cfg.get("s_e", 0.0)
        p.s_q = cfg.get("s_q", 1.2)
        p.s_eps_mode = int(cfg.get("s_eps_mode", 1))
        b = tuple(cfg.get("body", (0.0, 0.0))) + (0.0, 0.0, 0.0)
        p.body_force[0], p.body_force[1], p.body_force[2] = b[0], b[1], b[2] if three else 0.0
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p.rho0_store = rho0_store
        faces = cfg.get("faces", [])
        BC = (lbm_open_bc * max(1, len(faces)))()
        keep = []
        for j, fc in enumerate(faces):
            BC[j].kind = LBM_INLET_VELOCITY if fc["kind"] == "inlet" else LBM_OUTLET_CONVECTIVE
            BC[j].side = SIDES[fc["side"]]
            if three:
                BC[j].lo[0], BC[j].lo[1] = fc["lo"]
                BC[j].hi[0], BC[j].hi[1] = fc["hi"]
                npos = (fc["hi"][0] - fc["lo"][0] + 1) * (fc["hi"][1] - fc["lo"][1] + 1)
            else:
                BC[j].lo[0], BC[j].hi[0] = fc["lo"], fc["hi"]
                npos = fc["hi"] - fc["lo"] + 1
            # the library reads one inflow speed per face position of an inlet
            # (outlets ignore it); extents it rejects are reported by the library
            prof = fc.get("profile")
            if fc["kind"] != "inlet" or prof is None:
                prof = np.zeros(max(npos, 1))
            prof = np.ascontiguousarray(prof, dtype=np.float64).reshape(-1)
            if npos > 0 and prof.size != npos:
                raise ValueError("inlet profile needs %d values, got %d" % (npos, prof.size))
            keep.append(prof)
            BC[j].u_profile = _dptr(prof)
            if fc["kind"] == "inlet" and fc.get("rho_profile") is not None:
                rp = np.ascontiguousarray(fc["rho_profile"], dtype=np.float64).reshape(-1)
                if rp.size != 2 * npos:
                    raise ValueError("face rho_profile needs %d values" % (2 * npos))
                keep.append(rp)
                BC[j].rho_profile = _dptr(rp)
            r = fc.get("rho_in", (0.0, 0.0))
            BC[j].rho_in[0], BC[j].rho_in[1] = r
            BC[j].alpha_correction = int(fc.get("alpha", 1))
            BC[j].chi_correction = int(fc.get("chi", 1))
        sol = None
        if solid is not None:
            sol = np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
        rho = np.ascontiguousarray(rho_init, dtype=np.float64).reshape(-1)
        uu = None if u_init is None else np.ascontiguousarray(u_init, dtype=np.float64).reshape(-1)
        h = ctypes.c_void_p()
        st = L.lbm_create(ctypes.byref(g), ctypes.byref(p), BC, len(faces),
                          None if sol is None else sol.ctypes.data_as(ctypes.c_void_p), _dptr(rho),
                          None if uu is None else _dptr(uu), ctypes.c_void_p(stream or 0), ctypes.byref(h))
        _check(st, None)
        self.h = h
        self.precision = precision
        if cfg.get("wetting_delta") and not three:
            self.set_wetting(cfg["wetting_delta"])
        wu = cfg.get("wall_ux")
        if wu is not None and not three:
            for side, v in zip(("ymin", "ymax"), wu):
                if v:
                    self.set_wall_velocity(side, v)

    def close(self):
        if getattr(self, "h", None):
            load().lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, rho_init, u_init=None):
        rho = np.ascontiguousarray(rho_init, dtype=np.float64).reshape(-1)
        uu = None if u_init is None else np.ascontiguousarray(u_init, dtype=np.float64).reshape(-1)
        _check(load().lbm_reset(self.h, _dptr(rho), None if uu is None else _dptr(uu)), self.h)

    def step(self, n=1):
        _check(load().lbm_step(self.h, int(n)), self.h)

    def sync(self):
        _check(load().lbm_sync(self.h), self.h)

    def macros(self):
        """(rho[2][...], u[dim][...]) as float64 on the host ([ny][nx] in
        2D, [nz][ny][nx] in 3D)."""
        rho = np.zeros(2 * self.N)
        u = np.zeros(self.dim * self.N)
        _check(load().lbm_get_macros_f64(self.h, _dptr(rho), _dptr(u)), self.h)
        return rho.reshape(2, *self.shape), u.reshape(self.dim, *self.shape)

    def macros_f32(self, rho_ptr=None, u_ptr=None, device=False):
        """float32 fields into caller buffers (host numpy arrays, or device
        pointers when device=True); returns the numpy arrays if none given."""
        if rho_ptr is None:
            rho = np.zeros(2 * self.N, dtype=np.float32)
            u = np.zeros(self.dim * self.N, dtype=np.float32)
            _check(load().lbm_get_macros(self.h, rho.ctypes.data, u.ctypes.data, 0), self.h)
            return rho.reshape(2, *self.shape), u.reshape(self.dim, *self.shape)
        _check(load().lbm_get_macros(self.h, ctypes.c_void_p(rho_ptr), ctypes.c_void_p(u_ptr), int(device)), self.h)
        return None

    def populations(self):
        f = np.zeros(2 * self.Q * self.N)
        _check(load().lbm_get_populations(self.h, _dptr(f)), self.h)
        return f.reshape(2, self.Q, *self.shape)

    def set_populations(self, f):
        a = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        _check(load().lbm_set_populations(self.h, _dptr(a)), self.h)

    def diagnostics(self):
        d = lbm_diag()
        _check(load().lbm_get_diagnostics(self.h, ctypes.byref(d)), self.h)
        return {"mass": np.array(d.mass[:]), "lambda": d.lambda_, "chi": d.chi, "Qin": d.q_in,
                "Qout": d.q_out, "max_speed": d.max_speed, "step": d.step, "launches": d.launches,
                "status": d.status}

    def enable_kernel_timing(self, every):
        _check(load().lbm_enable_kernel_timing(self.h, int(every)), self.h)

    def kernel_time(self):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(load().lbm_kernel_time(self.h, ctypes.byref(ms), ctypes.byref(n)), self.h)
        return ms.value, n.value

    def kernel_time_split(self):
        a = ctypes.c_double()
        b = ctypes.c_double()
        n = ctypes.c_int64()
        _check(load().lbm_kernel_time_split(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)), self.h)
        return a.value, b.value, n.value

    def set_tile_variant(self, v):
        _check(load().lbm_set_tile_variant(self.h, int(v)), self.h)

    def tile_stats(self):
        v, a, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        fn, gn = ctypes.c_int64(), ctypes.c_int64()
        _check(load().lbm_tile_stats(self.h, ctypes.byref(v), ctypes.byref(a), ctypes.byref(b), ctypes.byref(fn),
                                     ctypes.byref(gn)), self.h)
        return {"variant": v.value, "fast_tiles": a.value, "general_tiles": b.value,
                "fast_nodes": fn.value, "general_nodes": gn.value}

    def set_graph_mode(self, on):
        _check(load().lbm_set_graph_mode(self.h, int(bool(on))), self.h)

    def set_schedule(self, name):
        """'graphs' (default), 'graphs_early' or 'persistent' (lbm_set_schedule)."""
        _check(load().lbm_set_schedule(self.h, SCHEDULES[name]), self.h)

    def schedule(self):
        """(schedule name, whether the step graphs launch early) (lbm_get_schedule)."""
        sch, early = ctypes.c_int(), ctypes.c_int()
        _check(load().lbm_get_schedule(self.h, ctypes.byref(sch), ctypes.byref(early)), self.h)
        return SCHEDULE_NAMES[sch.value], bool(early.value)

    def set_wall_velocity(self, side, ux):
        """Moving wall beyond the closed edge 'ymin' or 'ymax' (lbm_set_wall_velocity)."""
        _check(load().lbm_set_wall_velocity(self.h, SIDES[side], float(ux)), self.h)

    def set_wetting(self, delta):
        """Eq. 12's phase-dependent adhesion coefficient (lbm_set_wetting);
        delta <= 0 switches it off."""
        _check(load().lbm_set_wetting(self.h, float(delta)), self.h)

    def set_chi_timing(self, same_step):
        """chi from the step's own fluxes (True) or the previous step's
        (False, default): lbm_set_chi_timing."""
        _check(load().lbm_set_chi_timing(self.h, int(bool(same_step))), self.h)

    def autotune(self, steps=20):
        v = ctypes.c_int()
        ms = ctypes.c_double()
        _check(load().lbm_autotune(self.h, int(steps), ctypes.byref(v), ctypes.byref(ms)), self.h)
        return v.value, ms.value

    def save(self, path):
        _check(load().lbm_save(self.h, path.encode()), self.h)

    def load_checkpoint(self, path):
        _check(load().lbm_load(self.h, path.encode()), self.h)


class Batch:
    """A batched ensemble over existing Solver objects (lbm_batch_*)."""

    def __init__(self, members, stream=None):
        L = load()
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m.h.value for m in self.members])
        h = ctypes.c_void_p()
        st = L.lbm_batch_create(ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), len(self.members),
                                ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if st != LBM_OK:
            msg = L.lbm_batch_last_error(None)
            raise LbmError(st, msg.decode() if msg else "")
        self.h = h

    def _check(self, st):
        if st != LBM_OK:
            msg = load().lbm_batch_last_error(self.h)
            raise LbmError(st, msg.decode() if msg else "")

    def step(self, n=1):
        self._check(load().lbm_batch_step(self.h, int(n)))

    def sync(self):
        self._check(load().lbm_batch_sync(self.h))

    def set_tile_variant(self, v):
        self._check(load().lbm_batch_set_tile_variant(self.h, int(v)))

    def autotune(self, steps=20):
        v = ctypes.c_int()
        ms = ctypes.c_double()
        self._check(load().lbm_batch_autotune(self.h, int(steps), ctypes.byref(v), ctypes.byref(ms)))
        return v.value, ms.value

    def info(self):
        v, a, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        n = ctypes.c_int64()
        self._check(load().lbm_batch_info(self.h, ctypes.byref(v), ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)))
        return {"variant": v.value, "fast_tiles": a.value, "general_tiles": b.value, "launches": n.value}

    def set_graph_mode(self, on):
        self._check(load().lbm_batch_set_graph_mode(self.h, int(bool(on))))

    def set_schedule(self, name):
        """'graphs' (default), 'graphs_early' or 'persistent' (lbm_batch_set_schedule)."""
        self._check(load().lbm_batch_set_schedule(self.h, SCHEDULES[name]))

    def schedule(self):
        """(schedule name, whether the step graphs launch early) (lbm_batch_get_schedule)."""
        sch, early = ctypes.c_int(), ctypes.c_int()
        self._check(load().lbm_batch_get_schedule(self.h, ctypes.byref(sch), ctypes.byref(early)))
        return SCHEDULE_NAMES[sch.value], bool(early.value)

    def persistent_grid(self):
        n = ctypes.c_int()
        self._check(load().lbm_batch_persistent_grid(self.h, ctypes.byref(n)))
        return n.value

    def inject_barrier_fault(self, extra_arrivals, spin_limit_cycles=0):
        """Test hook: persistent barriers wait for `extra_arrivals` CTAs that
        never come, so their bounded waits run out (LBM_ERR_TIMEOUT)."""
        self._check(load().lbm_batch_inject_barrier_fault(self.h, int(extra_arrivals), int(spin_limit_cycles)))

    def close(self):
        if getattr(self, "h", None):
            load().lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mass_noalloc(f_ptr, precision, nx, ny, pitch, solid_ptr, mass_ptr, stream=None):
    """FP64 component masses of caller-owned device populations, written to
    the caller's device pair `mass_ptr`; allocates no device memory."""
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(load().lbm_mass_noalloc(ctypes.c_void_p(f_ptr), p, int(nx), int(ny), int(pitch),
                                   ctypes.c_void_p(solid_ptr or 0), ctypes.c_void_p(mass_ptr),
                                   ctypes.c_void_p(stream or 0)), None)


class MLP:
    """Surrogate MLP ensemble (lbm_mlp_*): members of 4 -> 128 -> 128 ->
    128 -> 2 with GELU, trained and evaluated by the library's kernels."""

    def __init__(self, members=5, seed=0, stream=None):
        L = load()
        h = ctypes.c_void_p()
        st = L.lbm_mlp_create(int(members), int(seed), ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if st != LBM_OK:
            msg = L.lbm_mlp_last_error(None)
            raise LbmError(st, msg.decode() if msg else "")
        self.h = h
        self.members = int(members)
        self.P = int(L.lbm_mlp_num_params())

    def _check(self, st):
        if st != LBM_OK:
            msg = load().lbm_mlp_last_error(self.h)
            raise LbmError(st, msg.decode() if msg else "")

    INFER_PATHS = {"simt": 0, "tensor": 1}

    def set_infer_path(self, name):
        """'simt' (FP32 FMAs) or 'tensor' (tcgen05 split products) for
        forward and predict (lbm_mlp_set_infer_path)."""
        self._check(load().lbm_mlp_set_infer_path(self.h, self.INFER_PATHS[name]))

    def set_wait_limit(self, cycles):
        """Longest tensor-core wait in SM cycles (0: default) (lbm_mlp_set_wait_limit)."""
        self._check(load().lbm_mlp_set_wait_limit(self.h, int(cycles)))

    @staticmethod
    def _f32(a, cols):
        a = np.ascontiguousarray(a, dtype=np.float32)
        if a.ndim != 2 or a.shape[1] != cols:
            raise ValueError("expected an [n][%d] array, got %s" % (cols, a.shape))
        return a

    def set_params(self, flat):
        """flat: [members][P] (or members*P) floats; resets Adam."""
        a = np.ascontiguousarray(flat, dtype=np.float32).reshape(-1)
        if a.size != self.members * self.P:
            raise ValueError("expected %d parameters" % (self.members * self.P))
        self._check(load().lbm_mlp_set_params(self.h, a.ctypes.data_as(_fp)))

    def params(self):
        out = np.zeros(self.members * self.P, dtype=np.float32)
        self._check(load().lbm_mlp_get_params(self.h, out.ctypes.data_as(_fp)))
        return out.reshape(self.members, self.P)

    def forward(self, X):
        X = self._f32(X, 4)
        Y = np.zeros((self.members, X.shape[0], 2), dtype=np.float32)
        self._check(load().lbm_mlp_forward(self.h, X.ctypes.data_as(_fp), X.shape[0], Y.ctypes.data_as(_fp)))
        return Y

    def gradient(self, X, T):
        X, T = self._f32(X, 4), self._f32(T, 2)
        g = np.zeros((self.members, self.P), dtype=np.float32)
        self._check(load().lbm_mlp_gradient(self.h, X.ctypes.data_as(_fp), T.ctypes.data_as(_fp), X.shape[0],
                                            g.ctypes.data_as(_fp)))
        return g

    def train(self, X, T, epochs, batch=256, lr=1e-3, shuffle_seed=0):
        X, T = self._f32(X, 4), self._f32(T, 2)
        self._check(load().lbm_mlp_train(self.h, X.ctypes.data_as(_fp), T.ctypes.data_as(_fp), X.shape[0],
                                         int(epochs), int(batch), float(lr), int(shuffle_seed)))

    def predict(self, X):
        """Ensemble mean [n][2] and relative spread [n] (host arrays)."""
        X = self._f32(X, 4)
        n = X.shape[0]
        mean = np.zeros((n, 2), dtype=np.float32)
        spread = np.zeros(n, dtype=np.float32)
        self._check(load().lbm_mlp_predict(self.h, X.ctypes.data, n, mean.ctypes.data, spread.ctypes.data, 0))
        return mean, spread

    def predict_device(self, x_ptr, n, mean_ptr, spread_ptr):
        """Device-pointer form: X [n][4], mean [n][2], spread [n] (float32)."""
        self._check(load().lbm_mlp_predict(self.h, ctypes.c_void_p(x_ptr), int(n), ctypes.c_void_p(mean_ptr),
                                           ctypes.c_void_p(spread_ptr), 1))

    def close(self):
        if getattr(self, "h", None):
            load().lbm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def version():
    return load().lbm_version().decode()
