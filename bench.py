#!/usr/bin/env python
"""Throughput benchmark of the fused D2Q9 two-component MRT pseudopotential
step (one JSON line on rank 0).

Workload: the 1024x128 droplet-migration channel (walls with bounce-back and
adhesion, velocity inlet with the alpha correction, convective outlet with
the chi mass-flux correction, one droplet R=30 at x=200, M = 1/5), FP32.
A benchmark step is a run of LBM time steps of that job (--lbm-steps, by
default 5000: one tenth of the 50k-step job); the state carries over from
one benchmark step to the next, as in the real run, and once the 50k steps
are done the job restarts from its initial fields (outside the timed
events), so the timed work does not depend on --steps or --warmup.  MLUPS
counts fluid-node updates.

--impl reference times the FP64 CPU oracle (the method's plain restatement)
on the host cores, on the same workload and metric.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

KERNEL_SRC = [os.path.join(ROOT, "paper_2512_12934_gb300", "csrc", f)
              for f in ("lbm_d2q9.cu", "d2q9_tile.cuh", "lbm_internal.h")]
KERNEL_SRC_3D = os.path.join(ROOT, "paper_2512_12934_gb300", "csrc", "lbm_d3q19.cu")
PROFILE_SUMMARY_3D = os.path.join(ROOT, "profiles", "d3q19_step_coflow_512x96x96.md")
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "d2q9_step_channel_1024x128.md")
BYTES_PER_NODE = {"fp32": 144, "fp16store": 80, "fp64": 288}
BYTES_PER_NODE_3D = {"fp32": 304, "fp16store": 160, "fp64": 608}  # 38 populations read + written per node and step (+ 2 half references read + written for fp16store)
DTYPE = {"fp32": "f32", "fp16store": "f16-storage/f32", "fp64": "f64"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--lbm-steps", type=int, default=5000, help="LBM time steps per benchmark step")
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp16store", "fp64"])
    p.add_argument("--workload", default="channel",
                   choices=["channel", "channel_hbm", "tjunction_batch", "surrogate", "coflow3d"],
                   help="channel: the 1024x128 config; channel_hbm: the same physics on 8192x2048; "
                        "tjunction_batch: the T-junction ensemble, batched vs sequential")
    p.add_argument("--instances", type=int, default=256, help="ensemble size for tjunction_batch")
    p.add_argument("--no-batch", action="store_true", help="skip the batched-ensemble entry of the default line")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-hbm", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--sur-train", type=int, default=1024, help="solver runs used to train the surrogate")
    p.add_argument("--sur-test", type=int, default=256, help="held-out solver runs judging the surrogate")
    p.add_argument("--no-mlp", action="store_true", help="skip the surrogate-kernel entry of the default line")
    p.add_argument("--no-3d", action="store_true", help="skip the D3Q19 co-flow entry of the default line")
    p.add_argument("--no-accuracy", action="store_true", help="skip the paper-accuracy entry of the default line")
    p.add_argument("--hbm-nx", type=int, default=8192, help="x extent of the HBM-resident channel grid")
    p.add_argument("--hbm-ny", type=int, default=2048, help="y extent of the HBM-resident channel grid")
    p.add_argument("--lbm-steps-3d", type=int, default=200, help="D3Q19 time steps per benchmark step")
    p.add_argument("--tile-variant", type=int, default=-1,
                   help="tile variant of the channel solver (default: the library's choice for the grid)")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, dist, device):
    """The largest x over the job's ranks (x itself on one rank).  A
    collective: every rank calls it."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, elapsed_max):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (each rank processes the same units: weak scaling)."""
    return world * units_per_rank / elapsed_max


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def guarded(fn):
    """Run one optional entry of the bench line; an exception (a diverged
    member, an unsupported configuration) becomes that entry's "error"
    field instead of ending the run."""
    try:
        return fn()
    except Exception as e:  # noqa: BLE001 - reported in the line
        return {"error": "%s: %s" % (type(e).__name__, e)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash(paths):
    """First 16 hex digits of the SHA-256 of the kernel's source files, read
    in order (a profile summary records it; counters apply only while the
    source is unchanged)."""
    h = hashlib.sha256()
    for p in (paths if isinstance(paths, (list, tuple)) else [paths]):
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    if not os.path.exists(PROFILE_SUMMARY):
        return None
    text = open(PROFILE_SUMMARY).read()
    h = kernel_source_hash(KERNEL_SRC)
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_traffic = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_traffic or m_hash.group(1) != h:
        return None
    return float(m_traffic.group(1))


def profiled_traffic_3d():
    """DRAM bytes of one D3Q19 co-flow step from the committed ncu summary, if
    it was taken on the current kernel source; else None."""
    if not os.path.exists(PROFILE_SUMMARY_3D):
        return None
    text = open(PROFILE_SUMMARY_3D).read()
    h = kernel_source_hash(KERNEL_SRC_3D)
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_traffic = re.search(r"dram_bytes_per_step_full_size:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_traffic or m_hash.group(1) != h:
        return None
    return float(m_traffic.group(1))


def cpu_oracle_sample(w, seconds, threads, min_steps=1):
    """Time the FP64 oracle on the host cores on the same grid; returns MLUPS."""
    from oracle import oracle as O

    o = O.Oracle2D(w.cfg, w.solid, w.rho, w.u, threads=threads)
    o.step(1)  # first touch outside the clock
    steps = 0
    t0 = time.perf_counter()
    while True:
        o.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds and steps >= min_steps:
            break
    return w.fluid_nodes * steps / el / 1e6, steps, el


def batched_vs_sequential(n, steps, reps, precision, stream_handle, world=1, rank=0):
    """Aggregate MLUPS of an n-instance T-junction ensemble stepped as one
    autotuned batch, against the same instances stepped one after another
    (each replaying its own captured graphs).  With world > 1 ranks the
    instances are split by fluid nodes (paper_2512_12934_gb300.ensemble) and
    this rank runs its own share only; rates and times are this rank's."""
    import torch

    from paper_2512_12934_gb300 import ensemble
    from paper_2512_12934_gb300 import lbm
    from paper_2512_12934_gb300 import workloads as W

    full = W.tjunction_ensemble(n)
    mine = ensemble.share_of([w.fluid_nodes for w in full], world, rank)
    ens = [full[i] for i in mine]
    solvers = [lbm.Solver(w.cfg, w.solid, w.rho, w.u, precision=precision, stream=stream_handle) for w in ens]
    fluid = sum(w.fluid_nodes for w in ens)
    batch = lbm.Batch(solvers, stream=stream_handle)
    variant, tuned_ms = batch.autotune(steps=8)
    batch.step(steps)
    batch.sync()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(reps):
        batch.step(steps)
    ev1.record()
    torch.cuda.synchronize()
    t_batch = ev0.elapsed_time(ev1) / 1e3
    info = batch.info()
    batch.close()
    for sv in solvers:              # per-instance graphs captured outside the clock
        sv.set_tile_variant(variant)
        sv.step(steps)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(reps):
        for sv in solvers:
            sv.step(steps)
    ev1.record()
    torch.cuda.synchronize()
    t_seq = ev0.elapsed_time(ev1) / 1e3
    # members whose flow blew up (non-finite fields; low-viscosity dispersed
    # phases at G12 = 2.0 can, in the FP64 oracle too): kept in the timing,
    # reported here
    member_status = [sv.diagnostics()["status"] for sv in solvers]
    status = max(member_status)
    diverged = sum(1 for st in member_status if st != 0)
    for sv in solvers:
        sv.close()
    mb = fluid * steps * reps / t_batch / 1e6
    ms = fluid * steps * reps / t_seq / 1e6
    return {"instances": len(ens), "instances_total": n, "fluid_nodes": fluid,
            "t_batch_s": t_batch, "t_seq_s": t_seq, "lbm_steps": steps * reps, "tile_variant": variant,
            "fast_tiles": info["fast_tiles"], "general_tiles": info["general_tiles"],
            "batched_mlups": mb, "sequential_mlups": ms, "speedup": mb / ms,
            "batched_ms_per_step": t_batch / (steps * reps) * 1e3,
            "roofline_frac_of_measured_hbm": mb * 1e6 * BYTES_PER_NODE[precision] / (measured_peaks()[0] * 1e9),
            "status": status, "diverged_members": diverged}


# FLOPs of the surrogate network per sample and member (4-128-128-128-2):
# forward 2(4*128 + 2*128^2 + 128*2); backward 4*2*128 + 8*128^2 + 2*128*4.
MLP_FWD_FLOP = 2 * (4 * 128 + 2 * 128 * 128 + 128 * 2)
MLP_BWD_FLOP = 4 * 2 * 128 + 8 * 128 * 128 + 2 * 128 * 4


def accuracy_figures(stream_handle):
    """The paper's headline accuracy quantities, measured with the FP32 GPU
    path (context, not a target; quoted beside the paper's own figures).

    Spurious currents (Sec. III A, Fig. 3d): a static droplet (100 x 100
    periodic, R = 20, G12 = 1.2, the wide-interface regime), nu_2 = 0.067
    and nu_1 = M nu_2, largest |u^eq| averaged over steps 4000-5000.  Rates
    "original": s_e = s_eps = each component's s_nu; "adjusted": s_e and
    s_eps from the most viscous phase for both components (taking s_eps
    alone from it, with s_e at each component's own rate, diverges for
    M >= 10, in the FP64 oracle as well).
    Mass deviation (Sec. III B, C): the 1024 x 128 droplet channel for its
    50k steps with and without the chi correction (Eqs. 22, 23); total mass
    (m(t) - m(0)) / m(0), final and time-averaged over 1000-step samples."""
    import numpy as np
    from paper_2512_12934_gb300 import lbm
    from paper_2512_12934_gb300 import workloads as W

    us = {}
    for M in (1, 10, 50, 150):
        row = {}
        for label in ("original", "adjusted"):
            nu = (0.067 * M, 0.067)
            w = W.laplace(G12=1.2, nu=nu, s_eps_mode=1 if label == "adjusted" else 0)
            if label == "adjusted":
                w.cfg["s_e"] = 1.0 / (3.0 * max(nu) + 0.5)
            s = lbm.Solver(w.cfg, w.solid, w.rho, w.u, stream=stream_handle)
            s.step(4000)
            acc = []
            for _ in range(10):
                s.step(100)
                _, u = s.macros()
                acc.append(float(np.hypot(u[0], u[1]).max()))
            row[label] = float(np.mean(acc))
            s.close()
        row["reduction_pct"] = 100.0 * (1.0 - row["adjusted"] / row["original"])
        us["M=%d" % M] = row
    red = [us[k]["reduction_pct"] for k in us if k != "M=1"]
    mass = {}
    for chi in (1, 0):
        w = W.channel(chi=bool(chi))
        s = lbm.Solver(w.cfg, w.solid, w.rho, w.u, stream=stream_handle)
        m0 = float(s.diagnostics()["mass"].sum())
        dev = []
        status = 0
        for _ in range(50):
            s.step(1000)
            d = s.diagnostics()
            status = d["status"]
            if status:
                break
            dev.append((float(d["mass"].sum()) - m0) / m0)
        s.close()
        mass["chi_on" if chi else "chi_off"] = {
            "final_pct": 100.0 * dev[-1] if dev else None,
            "mean_abs_pct": 100.0 * float(np.mean(np.abs(dev))) if dev else None,
            "steps": 1000 * len(dev), "status": status}
    return {"spurious_current_max": us, "mean_reduction_pct_M_gt_1": float(np.mean(red)),
            "paper_mean_reduction_pct": 65.8, "mass_deviation": mass, "paper_mass_deviation_pct": 3.5,
            "setup": "u_s: 100x100 periodic droplet R=20, G12=1.2, nu2=0.067, nu1=M*nu2, steps 4000-5000; "
                     "mass: 1024x128 channel, 50k steps"}


# FP32 FMA peak of the SIMT pipes: 152 SMs x 128 lanes x 2 FLOP at 2070 MHz.
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def split_tensor_peak():
    """Peak of the tensor-core inference path in FP32-equivalent FLOP/s: each
    hidden-layer FLOP is one TF32 product Ah.Wh, one TF32 product Al.Wh and
    one BF16 product Ab.Wl; TF32 runs at half the BF16 rate (2.25 against
    1.1 PFLOP/s dense, nominal), so the tensor pipes deliver the measured
    burst BF16 rate / (2 * 2 + 1)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["bf16_tflops"]) / 5.0, "measured bf16_tflops (burst) / 5"
    return 1900.0 / 5.0, "fallback bf16 1.9 PFLOP/s / 5"


def coflow3d(precision, stream_handle, bench_steps, lbm_steps, warmup, e2e=True):
    """The 512x96x96 coaxial co-flow device on the D3Q19 path: device-timed
    MLUPS over bench_steps x lbm_steps time steps (CUDA events), the sampled
    split between the pull and collide phases, and the step roofline."""
    import numpy as np
    import torch

    from paper_2512_12934_gb300 import lbm
    from paper_2512_12934_gb300 import workloads as W

    w = W.coflow3()
    s = lbm.Solver(w.cfg, w.solid, w.rho, w.u, precision=precision, stream=stream_handle)
    try:
        for _ in range(warmup):
            s.step(lbm_steps)
        s.sync()
        s.enable_kernel_timing(17)
        launches0 = s.diagnostics()["launches"]
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = torch.cuda.current_stream()
        ev0.record(st)
        for _ in range(bench_steps):
            s.step(lbm_steps)
        ev1.record(st)
        torch.cuda.synchronize()
        elapsed = ev0.elapsed_time(ev1) / 1e3
        pull_ms, collide_ms, nsamp = s.kernel_time_split()
        d = s.diagnostics()
        launches = d["launches"] - launches0 - 1
        e2e_res = None
        if e2e:
            rho_h = np.ascontiguousarray(w.rho, dtype=np.float64)
            u_h = np.ascontiguousarray(w.u, dtype=np.float64)
            out_r = np.empty((2,) + w.rho.shape[1:], dtype=np.float32)
            out_u = np.empty((3,) + w.rho.shape[1:], dtype=np.float32)
            s.enable_kernel_timing(0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.reset(rho_h, u_h)                       # H2D: populations, fields, open-face state
            s.step(lbm_steps)
            s.macros_f32(out_r.ctypes.data, out_u.ctypes.data, device=False)  # D2H
            el = time.perf_counter() - t0
            nodes = w.cfg["nx"] * w.cfg["ny"] * w.cfg["nz"]
            e2e_res = {"value": w.fluid_nodes * lbm_steps / el / 1e6, "unit": "MLUPS",
                       "h2d_bytes_per_step": nodes * 8 * (2 + 3), "d2h_bytes_per_step": nodes * 4 * 5,
                       "api": "lbm_reset(host fields) + lbm_step + lbm_get_macros(host)"}
    finally:
        s.close()
    nsteps = bench_steps * lbm_steps
    step_s = elapsed / nsteps
    bpn = BYTES_PER_NODE_3D[precision]
    achieved = bpn * w.fluid_nodes / step_s / 1e9
    peak, kind = measured_peaks()
    return {"workload": "coflow3d_512x96x96", "fluid_nodes": w.fluid_nodes, "lbm_steps": nsteps,
            "mlups": w.fluid_nodes / step_s / 1e6, "ms_per_lbm_step": step_s * 1e3,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": profiled_traffic_3d(),
                         "kernel": "one D3Q19 step (pull + face + collide + outlet + reduce kernels)",
                         "algorithmic_bytes_per_launch": bpn * w.fluid_nodes,
                         "peak_source": "%s hbm_gbs (copy, burst)" % kind},
            "sampled_pull_ms": pull_ms, "sampled_collide_ms": collide_ms, "kernel_samples": nsamp,
            "gpu_launches": launches, "e2e": e2e_res, "status": d["status"],
            "config": {"G12": w.cfg["G12"], "Gw": list(w.cfg["Gw"]), "nu": list(w.cfg["nu"]),
                       "r_in": w.meta["r_in"], "r_out": w.meta["r_out"], "q_ratio": w.meta["q_ratio"],
                       "M": w.meta["M"], "u_c": w.meta["u_c"]}}


def surrogate_cpu_baseline(solver_s_per_point, n=4096, members=5):
    """The FP64 reference MLP (oracle) timed on the host: solver seconds per
    point over its seconds per point."""
    import numpy as np

    from oracle import mlp_oracle as M

    rng = np.random.default_rng(0)
    ps = [M.init_params(rng) for _ in range(members)]
    X = rng.standard_normal((n, 4))
    t0 = time.perf_counter()
    for p in ps:
        M.forward(p, X)
    el = time.perf_counter() - t0
    return {"value": solver_s_per_point / (el / n), "unit": "x", "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": "FP64 numpy forward of %d members on %d points, %.2f s" % (members, n, el)}


def mlp_kernels(stream_handle, n_infer=65536, n_train=4096, members=5, reps=10):
    """Device-resident timings of the surrogate kernels: ensemble inference on
    n_infer points (forward + mean/spread) on the tensor-core path (default)
    against the split-product tensor peak and on the FP32 path against the
    FP32 ALU peak, and Adam training steps on n_train samples (forward +
    backward + update, FP32 pipes)."""
    import numpy as np
    import torch

    from paper_2512_12934_gb300 import lbm

    net = lbm.MLP(members, seed=1, stream=stream_handle)
    try:
        rng = np.random.default_rng(0)
        X = torch.from_numpy(rng.standard_normal((n_infer, 4)).astype(np.float32)).cuda()
        mean = torch.empty((n_infer, 2), dtype=torch.float32, device="cuda")
        spread = torch.empty(n_infer, dtype=torch.float32, device="cuda")
        st = torch.cuda.current_stream()

        def time_infer(path):
            net.set_infer_path(path)
            net.predict_device(X.data_ptr(), n_infer, mean.data_ptr(), spread.data_ptr())
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(st)
            for _ in range(reps):
                net.predict_device(X.data_ptr(), n_infer, mean.data_ptr(), spread.data_ptr())
            ev1.record(st)
            torch.cuda.synchronize()
            return ev0.elapsed_time(ev1) / 1e3 / reps

        t_simt = time_infer("simt")
        t_inf = time_infer("tensor")
        Xt = rng.standard_normal((n_train, 4)).astype(np.float32)
        Tt = rng.standard_normal((n_train, 2)).astype(np.float32)
        net.train(Xt, Tt, epochs=2, batch=n_train, lr=1e-3)
        t0 = time.perf_counter()
        net.train(Xt, Tt, epochs=reps, batch=n_train, lr=1e-3)
        t_step = (time.perf_counter() - t0) / reps
    finally:
        net.close()
    inf_tf = n_infer * members * MLP_FWD_FLOP / t_inf / 1e12
    simt_tf = n_infer * members * MLP_FWD_FLOP / t_simt / 1e12
    tr_tf = n_train * members * (MLP_FWD_FLOP + MLP_BWD_FLOP) / t_step / 1e12
    tpk, tpk_src = split_tensor_peak()
    return {"members": members,
            "infer_points": n_infer, "infer_path": "tensor (tcgen05, 3-term split product)",
            "infer_ms": t_inf * 1e3, "infer_points_per_s": n_infer / t_inf,
            "infer_tflops": inf_tf, "infer_frac_of_split_tensor_peak": inf_tf / tpk,
            "split_tensor_peak_tflops": tpk, "split_tensor_peak_source": tpk_src,
            "infer_simt_ms": t_simt * 1e3, "infer_simt_tflops": simt_tf,
            "infer_simt_frac_of_fp32_alu_peak": simt_tf / FP32_ALU_PEAK_TFLOPS,
            "train_samples": n_train, "train_step_ms": t_step * 1e3, "train_tflops": tr_tf,
            "train_frac_of_fp32_alu_peak": tr_tf / FP32_ALU_PEAK_TFLOPS,
            "fp32_alu_peak_tflops": FP32_ALU_PEAK_TFLOPS,
            "note": "infer: CUDA events over device-pointer lbm_mlp_predict calls; train: wall time of "
                    "lbm_mlp_train epochs of one full-batch Adam step (includes the per-epoch shuffle upload)"}


def surrogate_eval(args, stream_handle):
    """Train the surrogate on solver runs and evaluate it on held-out runs."""
    import numpy as np
    import torch

    from paper_2512_12934_gb300 import surrogate as SU

    dev = SU.Device()
    gamma = SU.surface_tension()
    n_tr, n_te = args.sur_train, args.sur_test
    pts = SU.sample_points(n_tr + n_te, 2512007)
    t0 = time.perf_counter()
    Y, valid, solver_s = SU.generate(pts, dev)
    gen_wall = time.perf_counter() - t0
    tr = np.arange(n_tr)[valid[:n_tr]]
    te = n_tr + np.arange(n_te)[valid[n_tr:]]
    sur = SU.Surrogate(members=5, gamma=gamma, dev=dev)
    try:
        t0 = time.perf_counter()
        sur.fit(pts[tr], Y[tr], epochs=300, batch=32, lr=2e-3)
        train_s = time.perf_counter() - t0
        val, spread = sur.predict(pts[te])
        err = np.abs(val / Y[te] - 1.0)
        acc = spread <= 0.05
        big = SU.sample_points(65536, 99)
        F = sur._x(big)
        Xd = torch.from_numpy(F).cuda()
        md = torch.empty((len(big), 2), dtype=torch.float32, device="cuda")
        sd = torch.empty(len(big), dtype=torch.float32, device="cuda")
        sur.net.predict_device(Xd.data_ptr(), len(big), md.data_ptr(), sd.data_ptr())
        torch.cuda.synchronize()
        reps = 10
        t0 = time.perf_counter()
        for _ in range(reps):
            sur.net.predict_device(Xd.data_ptr(), len(big), md.data_ptr(), sd.data_ptr())
        torch.cuda.synchronize()
        dev_pp = (time.perf_counter() - t0) / reps / len(big)
        t0 = time.perf_counter()
        for _ in range(reps):
            sur.predict(big)  # host parameter points in, host answers out
        host_pp = (time.perf_counter() - t0) / reps / len(big)
    finally:
        sur.close()

    def stats(e):
        return {"median": float(np.median(e)), "p90": float(np.percentile(e, 90)),
                "p95": float(np.percentile(e, 95)), "max": float(e.max())} if len(e) else None

    return {
        "gamma": gamma, "train_runs": n_tr, "test_runs": n_te, "valid_train": int(len(tr)),
        "valid_test": int(len(te)), "solver_s_per_point": solver_s, "generate_wall_s": gen_wall,
        "train_wall_s": train_s, "accepted_frac": float(acc.mean()),
        "D_rel_err_accepted": stats(err[acc, 0]), "T_rel_err_accepted": stats(err[acc, 1]),
        "D_rel_err_all": stats(err[:, 0]), "T_rel_err_all": stats(err[:, 1]),
        "D_within_5pct_frac": float((err[acc, 0] <= 0.05).mean()) if acc.any() else None,
        "net_s_per_point_device": dev_pp, "net_s_per_point_host": host_pp,
        "speedup_device": solver_s / dev_pp, "speedup_host": solver_s / host_pp,
        "device": {"Wc": dev.Wc, "length_factor": dev.length_factor, "steps": dev.steps,
                   "G12": SU.G12_TJ, "Gw": SU.GW_TJ, "ranges": SU.RANGES},
    }


def run_reference(args, world, rank):
    from paper_2512_12934_gb300 import workloads as W

    if rank != 0:
        return 0
    w = W.channel()
    threads = os.cpu_count() or 1
    from oracle import oracle as O

    o = O.Oracle2D(w.cfg, w.solid, w.rho, w.u, threads=threads)
    per_step = 2  # LBM steps of the full grid per benchmark step (bounded sample)
    for _ in range(args.warmup):
        o.step(per_step)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(per_step)
    el = time.perf_counter() - t0
    mlups = w.fluid_nodes * per_step * args.steps / el / 1e6
    line = {
        "impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "channel_1024x128_droplet_migration", "grid": [w.cfg["nx"], w.cfg["ny"]],
                   "fluid_nodes": w.fluid_nodes, "lbm_steps_per_step": per_step, "G12": w.cfg["G12"],
                   "Gw": list(w.cfg["Gw"]), "nu": list(w.cfg["nu"]), "parallelism": "openmp-host"},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                         "sample": "%d x %d full-grid FP64 oracle steps on %d host threads" % (
                             args.steps, per_step, threads)},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch

    from paper_2512_12934_gb300 import lbm
    from paper_2512_12934_gb300 import workloads as W

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU: the solver has no CPU path")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://", world_size=world, rank=rank,
                                device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    lbm.load()
    stream = torch.cuda.current_stream()
    if args.workload == "tjunction_batch":
        ck = Clocks(local)
        ck.start()
        barrier()
        res = batched_vs_sequential(args.instances, args.lbm_steps, args.steps, args.precision, stream.cuda_stream,
                                    world, rank)
        barrier()
        clk = ck.stop()
        # every rank steps its own share of the instances (no data-path
        # collective); the job's rate is all ranks' node updates over the
        # slowest rank's time
        t_max = max_over_ranks(res["t_batch_s"], dist, "cuda")
        units = res["fluid_nodes"] * res["lbm_steps"]
        if dist is not None:
            tt = torch.tensor([float(units)], dtype=torch.float64, device="cuda")
            dist.all_reduce(tt)
            units = float(tt.item())
        value_b = units / t_max / 1e6
        if rank == 0:
            print(json.dumps({"metric": "MLUPS", "value": value_b, "unit": "MLUPS", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": res["batched_ms_per_step"] * args.lbm_steps,
                              "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                              "dtype": DTYPE[args.precision], "data": "synthetic",
                              "config": {"workload": "tjunction_ensemble_batched", "instances": args.instances,
                                         "lbm_steps_per_step": args.lbm_steps, "precision": args.precision,
                                         "parallelism": "instances split over %d rank(s) by fluid nodes" % world},
                              "batched_ensemble": res, "clocks": clk}))
        return 0
    if args.workload == "coflow3d":
        prec = args.precision if args.precision in BYTES_PER_NODE_3D else "fp32"
        ck = Clocks(local)
        ck.start()
        barrier()
        res = coflow3d(prec, stream.cuda_stream, args.steps, args.lbm_steps_3d, args.warmup, e2e=not args.no_e2e)
        barrier()
        clk = ck.stop()
        # the slowest rank's time per step sets the job's rate
        ms_step = max_over_ranks(res["ms_per_lbm_step"], dist, "cuda")
        value3 = job_rate(res["fluid_nodes"], world, ms_step * 1e-3) / 1e6
        cpu = None
        if rank == 0 and not args.no_cpu:
            from oracle import oracle3d as O3
            w3 = W.coflow3()
            threads = os.cpu_count() or 1
            o = O3.Oracle3D(w3.cfg, w3.solid, w3.rho, w3.u, threads=threads)
            t0 = time.perf_counter()
            o.step(1)
            el = time.perf_counter() - t0
            cpu = {"value": w3.fluid_nodes / el / 1e6, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                   "sample": "1 full-grid FP64 D3Q19 oracle step of the 512x96x96 co-flow, %.1f s, %d threads" % (
                       el, threads)}
        if rank == 0:
            print(json.dumps({
                "metric": "MLUPS", "value": value3, "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step * args.lbm_steps_3d,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[prec],
                "data": "synthetic",
                "config": {"workload": res["workload"], "grid": [512, 96, 96], "fluid_nodes": res["fluid_nodes"],
                           "lbm_steps_per_step": args.lbm_steps_3d, "precision": prec,
                           "l2": "state (1.4 GB) far larger than L2", **res["config"]},
                "roofline": res["roofline"], "cpu_baseline": cpu, "e2e": res["e2e"],
                "gpu_launches": res["gpu_launches"], "clocks": clk, "status": res["status"],
                "sampled_pull_ms": res["sampled_pull_ms"], "sampled_collide_ms": res["sampled_collide_ms"]}))
        return 0
    if args.workload == "surrogate":
        ck = Clocks(local)
        ck.start()
        res = surrogate_eval(args, stream.cuda_stream)
        kern = mlp_kernels(stream.cuda_stream)
        clk = ck.stop()
        cpu = None
        if rank == 0 and not args.no_cpu:
            cpu = surrogate_cpu_baseline(res["solver_s_per_point"])
        if rank == 0:
            print(json.dumps({
                "metric": "surrogate speedup per parameter point", "value": res["speedup_device"] * world,
                "unit": "x", "n_gpus": world, "steps": 1, "warmup": 1,
                "ms_per_step": res["net_s_per_point_device"] * 65536 * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "tjunction_surrogate", "members": 5, "network": "4-128-128-128-2 GELU",
                           "inference_batch": 65536, "train_runs": args.sur_train, "test_runs": args.sur_test},
                "surrogate": res,
                "roofline": {"bound": "tensor", "achieved": kern["infer_tflops"],
                             "peak": kern["split_tensor_peak_tflops"], "unit": "TFLOP/s",
                             "frac": kern["infer_frac_of_split_tensor_peak"], "traffic": None,
                             "peak_source": kern["split_tensor_peak_source"],
                             "kernel": "mlp_infer_tc_kernel + mlp_reduce_kernel (65536 points x 5 members)"},
                "mlp_kernels": kern,
                "e2e": {"value": res["speedup_host"], "unit": "x", "h2d_bytes_per_step": 65536 * 4 * 4,
                        "d2h_bytes_per_step": 65536 * 3 * 4,
                        "api": "Surrogate.predict(host points) -> lbm_mlp_predict(host arrays)"},
                "cpu_baseline": cpu, "gpu_launches": 2 * 10, "clocks": clk}))
        return 0
    w = W.channel() if args.workload == "channel" else W.channel(nx=args.hbm_nx, ny=args.hbm_ny, R=240, xc=1600)
    S = args.lbm_steps
    solver = lbm.Solver(w.cfg, w.solid, w.rho, w.u, precision=args.precision, stream=stream.cuda_stream)
    if args.tile_variant >= 0:
        solver.set_tile_variant(args.tile_variant)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    rho_h = np.ascontiguousarray(w.rho, dtype=np.float64)
    u_h = np.ascontiguousarray(w.u, dtype=np.float64)
    # The job is w.steps (50k) LBM steps from the initial fields; a benchmark
    # step runs the next S of them.  When the job is complete the solver
    # restarts it from the initial fields (between timed steps, outside the
    # CUDA events), so the timed work is the same whatever --steps and
    # --warmup are, and the run never goes beyond the job's length.
    segments = max(1, w.steps // S)
    job = {"seg": 0, "restarts": 0}

    def next_segment(ev_a=None, ev_b=None):
        if job["seg"] == segments:
            solver.reset(rho_h, u_h)
            job["seg"] = 0
            job["restarts"] += 1
        if ev_a is not None:
            ev_a.record(stream)
        solver.step(S)
        if ev_b is not None:
            ev_b.record(stream)
        job["seg"] += 1

    for _ in range(args.warmup):
        next_segment()
        flush.zero_()
    solver.sync()
    solver.enable_kernel_timing(97)  # every 97th step launch sampled between CUDA events
    launches0 = solver.diagnostics()["launches"]

    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        next_segment(*evs[k])
        if k + 1 < args.steps:
            flush.zero_()  # L2 flush between timed steps (256 MiB > 129 MB L2)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    # device time of the K benchmark steps: each bracketed by CUDA events on
    # the launching stream (the flushes and job restarts between them excluded)
    elapsed = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    solver.sync()
    kfast, kgen, ksamples = solver.kernel_time_split()
    kms = kfast + kgen
    diag = solver.diagnostics()
    launches = diag["launches"] - launches0 - 1  # minus the diagnostics launch itself
    elapsed = max_over_ranks(elapsed, dist, "cuda")

    nodes = w.fluid_nodes
    value = job_rate(nodes * S * args.steps, world, elapsed) / 1e6
    bpn = BYTES_PER_NODE[args.precision]
    peak, peak_kind = measured_peaks()
    # one step = the fused step kernel over both tile lists (fast tiles and the
    # tiles that see an open face, run as parallel graph branches); its mean
    # duration is the CUDA-event time of the timed region over the steps run
    step_s = elapsed / (S * args.steps)
    achieved = bpn * nodes / step_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": profiled_traffic(),
                "kernel": "d2q9_step_kernel (fast + general tile lists, one step)",
                "step_us": step_s * 1e6,
                "sampled_fast_list_us": kfast * 1e3, "sampled_general_list_us": kgen * 1e3,
                "kernel_samples": ksamples,
                "algorithmic_bytes_per_launch": bpn * nodes,
                "peak_source": "%s hbm_gbs (copy, burst)" % peak_kind,
                "note": "the 1024x128 state (38 MB ping-pong) stays in L2 between steps; "
                        "see roofline_hbm_resident for the same kernel on an HBM-resident grid"}

    # ---- the same physics on an HBM-resident grid (roofline of the kernel proper)
    def hbm_resident():
        big = W.channel(nx=args.hbm_nx, ny=args.hbm_ny, R=240, xc=1600)
        per_variant = {}
        for v in (0, 4):   # 32x8 tile kernels; 32x8 with the column-marching kernel for interior tiles
            sb = lbm.Solver(big.cfg, big.solid, big.rho, big.u, precision=args.precision,
                            stream=stream.cuda_stream)
            sb.set_tile_variant(v)
            sb.step(20)
            sb.sync()
            sb.enable_kernel_timing(1)
            sb.step(60)
            bfast, bgen, bn = sb.kernel_time_split()
            fast_nodes = sb.tile_stats()["fast_nodes"]  # nodes outside the general list (99 % of this grid)
            sb.sync()
            sb.close()
            per_variant[v] = (bfast, bgen, bn, fast_nodes)
        v = min(per_variant, key=lambda k: per_variant[k][0] / per_variant[k][3])
        bfast, bgen, bn, fast_nodes = per_variant[v]
        bach = bpn * fast_nodes / (bfast / 1e3) / 1e9
        hbm = {"bound": "hbm", "achieved": bach, "peak": peak, "unit": "GB/s", "frac": bach / peak,
               "kernel": ("d2q9_march_kernel (interior runs) + d2q9_step_kernel (edge tiles)" if v == 4
                          else "d2q9_step_kernel fast tile list"),
               "tile_variant": v, "kernel_ms": bfast,
               "general_list_ms": bgen, "kernel_samples": bn, "grid": [args.hbm_nx, args.hbm_ny],
               "algorithmic_bytes_per_launch": bpn * fast_nodes,
               "mlups_step": big.fluid_nodes / ((bfast + bgen) / 1e3) / 1e6,
               "per_variant_fast_GBs": {str(k): bpn * val[3] / (val[0] / 1e3) / 1e9 for k, val in per_variant.items()}}
        return hbm

    hbm = None if args.no_hbm else guarded(hbm_resident)

    # ---- end to end through the public API with host buffers
    def end_to_end():
        out_rho = np.empty((2, w.cfg["ny"], w.cfg["nx"]), dtype=np.float32)
        out_u = np.empty((2, w.cfg["ny"], w.cfg["nx"]), dtype=np.float32)
        e2e_steps = max(1, min(args.steps, 5))
        solver.reset(rho_h, u_h)
        solver.step(S)
        solver.macros_f32(out_rho.ctypes.data, out_u.ctypes.data, device=False)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            solver.reset(rho_h, u_h)                 # H2D: populations, macros, outlet state
            solver.step(S)
            solver.macros_f32(out_rho.ctypes.data, out_u.ctypes.data, device=False)  # D2H
        torch.cuda.synchronize()
        barrier()
        el = time.perf_counter() - t0
        pitch = (w.cfg["nx"] + 31) // 32 * 32
        plane = pitch * w.cfg["ny"]
        sb_ = {"fp32": 4, "fp16store": 2, "fp64": 8}[args.precision]
        rb_ = 8 if args.precision == "fp64" else 4
        nfn = sum(f["hi"] - f["lo"] + 1 for f in w.cfg["faces"])
        h2d = 18 * plane * sb_ + 4 * plane * rb_ + 2 * nfn * 18 * rb_ + 2 * 64
        d2h = 4 * plane * rb_ + 4
        e2e = {"value": world * nodes * S * e2e_steps / el / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "api": "lbm_reset(host fields) + lbm_step + lbm_get_macros(host)"}
        return e2e

    e2e = None if args.no_e2e else guarded(end_to_end)

    main_line = args.workload == "channel"
    batched = None
    if not args.no_batch and main_line:
        batched = guarded(lambda: batched_vs_sequential(64, 64, 3, args.precision, stream.cuda_stream))
    mlp = None
    if not args.no_mlp and main_line:
        mlp = guarded(lambda: mlp_kernels(stream.cuda_stream))
    acc = None
    if not args.no_accuracy and main_line:
        acc = guarded(lambda: accuracy_figures(stream.cuda_stream))
    d3 = None
    if not args.no_3d and main_line:
        d3 = guarded(lambda: coflow3d("fp32", stream.cuda_stream, 2, 100, 1, e2e=False))

    cpu = None
    if rank == 0 and not args.no_cpu:
        threads = os.cpu_count() or 1
        mlups, steps_done, el = cpu_oracle_sample(w, args.cpu_seconds, threads)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": "%d full-grid FP64 oracle steps of the 1024x128 channel, %.1f s, %d threads" % (
                   steps_done, el, threads)}

    if rank == 0:
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": "channel_%dx%d_droplet_migration" % (w.cfg["nx"], w.cfg["ny"]),
                       "grid": [w.cfg["nx"], w.cfg["ny"]],
                       "fluid_nodes": nodes, "lbm_steps_per_step": S, "precision": args.precision,
                       "G12": w.cfg["G12"], "Gw": list(w.cfg["Gw"]), "nu": list(w.cfg["nu"]),
                       "u_max": w.meta["u_max"], "droplet_R": w.meta["R"],
                       "l2": "256 MiB written between timed steps; within a step the 38 MB state stays in L2",
                       "job_steps": w.steps, "job_restarts": job["restarts"],
                       "parallelism": "replicas" if world > 1 else "single-gpu"},
            "roofline": roofline,
            "roofline_hbm_resident": hbm,
            "batched_ensemble": batched,
            "surrogate_kernels": mlp,
            "d3q19_coflow": d3,
            "accuracy": acc,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": ck,
            "status": diag["status"],
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
