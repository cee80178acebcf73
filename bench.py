#!/usr/bin/env python3
"""Throughput of the FR/LES hot path on one GB300 per rank.

A step is one classic RK4 step (four FR residual evaluations of the
compressible Navier-Stokes equations with Rusanov and BR2 fluxes, fused with
the stage updates) of the 3D Taylor-Green vortex at Re = 1600, M = 0.1 on a
periodic 32^3 hexahedral box at FR order p = 3 (2,097,152 solution points per
variable).  The metric is DOF x RK-stages per second (DOF = solution points,
counted once).  Inputs are synthetic and seeded; the mesh is generated.

The timed region replays a CUDA graph of one step K times on one stream with
the state resident in HBM; the working set (~0.27 GB in FP32) is larger than
the 129 MB L2.  `value` is the FP32 path; the FP64 path on the same workload
is reported beside it, with the FP32 state deviation from FP64 after the
timed steps.  `--gpus N` under torchrun runs N independent replicas (the path
does not need a collective); value = all replicas' work / max time.

After the headline workload the same measurement runs on the batched poll
(12 NACA candidates of uneven meshes in one context, mixed precision, each at
its own time step) and is reported under "batched", with its FP64 path and the
per-candidate mean C_L / C_D of both precisions.

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload (the only other place this script runs it) and prints its line.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF*RK-stages/s per GB300 (mixed/batched vs FP64 plain at stated error), %roofline"
UNIT = "DOF*RK-stages/s"
GAMMA = 1.4
MACH = 0.1
DT = 2.5e-4


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------- CPU oracle leg
ORACLE_BOX = 8   # elements per direction of the oracle's sample of the TGV box


def oracle_sample(n=ORACLE_BOX, min_seconds=10.0, max_steps=10000, warmup=1):
    """FP64 numpy oracle: RK4 steps of the same TGV workload on an n^3 box,
    one BLAS thread, for at least min_seconds (and at most max_steps steps);
    min_seconds <= 0 runs exactly max_steps steps.  Returns (DOF*stages/s,
    steps, seconds, dof)."""
    import numpy as np

    from oracle.fr import FRSolver
    from oracle.mesh import Mesh
    from oracle.physics import NavierStokes
    from paper_2501_05709_gb300 import workloads as W
    nodes, conn = W.box_mesh(3, n, 0.0, 2 * math.pi, q=1)
    m = Mesh(nodes, conn, 3)
    s = FRSolver(m, NavierStokes(3, mu=1.0 / 1600.0))
    u = np.ascontiguousarray(np.moveaxis(W.taylor_green(m.xsp, mach=MACH), 0, 1))
    for _ in range(max(warmup, 0)):
        u = s.rk4_step(u, DT)
    t0 = time.perf_counter()
    k = 0
    while k < max_steps and (min_seconds <= 0 or time.perf_counter() - t0 < min_seconds or k == 0):
        u = s.rk4_step(u, DT)
        k += 1
    dt = time.perf_counter() - t0
    dof = m.E * m.Nsp
    return dof * 4 * k / dt, k, dt, dof


def run_oracle_subprocess(min_seconds, max_steps=10000, warmup=1):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_sample(min_seconds=%f, max_steps=%d, warmup=%d)))"
            % (ROOT, min_seconds, max_steps, warmup))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    v, k, dt, dof = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
            "steps_timed": k, "seconds": dt,
            "sample": f"TGV p=3 on a {ORACLE_BOX}^3-element box ({dof} DOF; the same per-element work as the "
                      f"32^3 workload), {k} RK4 steps in {dt:.1f} s, numpy FP64, 1 BLAS thread"}


def run_oracle_all_cores(min_seconds):
    """The same oracle sample in one single-threaded process per host core,
    all at once; value = the sum of their rates (element-parallel work spread
    over the cores, without changing the oracle)."""
    try:
        ncores = len(os.sched_getaffinity(0))
    except AttributeError:
        ncores = os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_sample(min_seconds=%f)))" % (ROOT, min_seconds))
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                              env=env) for _ in range(ncores)]
    rates, steps, secs = [], 0, 0.0
    for pr in procs:
        out, err = pr.communicate(timeout=900)
        if pr.returncode != 0:
            raise RuntimeError(err[-2000:])
        v, k, dt, dof = json.loads(out.strip().splitlines()[-1])
        rates.append(v)
        steps += k
        secs = max(secs, dt)
    return {"value": float(sum(rates)), "unit": UNIT, "cores": ncores, "kind": "oracle",
            "sample": f"{ncores} concurrent single-threaded processes, each TGV p=3 on a {ORACLE_BOX}^3-element box "
                      f"({dof} DOF) for >= {min_seconds:.0f} s ({steps} RK4 steps in total), numpy FP64"}


# ----------------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = str(gpu_index)
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", self.idx, f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" == r[5 + i].strip()})
        sm_sorted = sorted(sm)
        return {"sm_mhz": sm_sorted[len(sm_sorted) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- ncu counters
KERNEL_SOURCES = ("csrc/fr_kernels.cuh", "csrc/fr_common.h", "csrc/fr_launch.cuh", "csrc/fr_f32_3d.cu",
                  "csrc/fr_f64_3d.cu", "build.py")
FWH_SOURCES = ("csrc/fwh.cu", "build.py")


def kernel_source_hash(files=KERNEL_SOURCES):
    """sha256 (first 16 hex digits) of the kernel sources and build flags,
    without blank lines and whole-line comments: counters taken on other code
    are stale and are not reported."""
    import hashlib
    h = hashlib.sha256()
    for n in files:
        with open(os.path.join(ROOT, "paper_2501_05709_gb300", n)) as f:
            for line in f:
                t = line.strip()
                if t and not t.startswith(("//", "#")) or t.startswith(("#include", "#define", "#pragma", "#if",
                                                                        "#else", "#endif", "#undef")):
                    h.update(t.encode() + b"\n")
    return h.hexdigest()[:16]


def ncu_counter(workload, precision, kernel, key):
    """A per-launch figure from profiles/ncu_counters.txt (written from one ncu
    capture of this script), or None when it was taken on other kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_counters.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    src = kernel_source_hash(FWH_SOURCES if kernel.startswith("fwh") else KERNEL_SOURCES)
    for ln in lines:
        if ln.startswith("#") or "=" not in ln:
            continue
        kv = dict(t.split("=", 1) for t in ln.split())
        if (kv.get("src") == src and kv.get("workload") == workload and kv.get("precision") == precision
                and kv.get("kernel") == kernel and key in kv):
            return float(kv[key])
    return None


# ----------------------------------------------------------------------------- GPU leg
def algorithmic_bytes(E, p, rsz, viscous=True, dim=3, curved=False):
    """Minimum HBM bytes per RK stage of each kernel: every array the kernel
    must touch, read or written once.  Metrics: one set per element (affine)
    or S and 1/|J| per solution point and a normal per flux point (curved)."""
    np_ = p + 1
    nsp, nfp, nf, nv = np_ ** dim, np_ ** (dim - 1), 2 * dim, dim + 2
    u = nv * nsp * rsz
    tr = nf * nv * nfp * rsz
    if curved:
        geo = (dim * dim + 1) * nsp * rsz + nf * nfp * dim * rsz + nf * 4
    else:
        geo = (dim * dim + 1 + nf * dim) * rsz + nf * 4
    traces = E * (u + tr)
    visc = E * (u + tr + tr + geo) if viscous else 0
    rk = (2 + 4 + 4 + 3) / 4.0 * u
    # residual: u, neighbour traces, the viscous-flux array (each face's
    # entries are read by both elements of the face, but the array need only
    # move once), metrics, RK stage arrays (stage-averaged) and the traces of
    # the updated state
    resid = E * (u + tr + (tr if viscous else 0) + geo + rk + tr)
    return {"traces": traces, "visc": visc, "resid": resid}


def reduced_bytes(orders, p, rsz, viscous=True, dim=3, curved=False):
    """Minimum HBM bytes per RK stage of the reduced-degree kernels (face and
    residual) over the elements of degree q < p: the same arrays as a
    degree-p element (state, traces, viscous fluxes and RK arrays stay at the
    degree-p points), with the metric terms taken at the (q+1)^dim points."""
    orders = np.asarray(orders)
    np_ = p + 1
    nsp, nfp, nf, nv = np_ ** dim, np_ ** (dim - 1), 2 * dim, dim + 2
    u = nv * nsp * rsz
    tr = nf * nv * nfp * rsz
    normals = (nf * nfp * dim if curved else nf * dim) * rsz + nf * 4
    rk = (2 + 4 + 4 + 3) / 4.0 * u
    total = 0.0
    for q in range(p):
        n = int((orders == q).sum())
        geo = (dim * dim + 1) * (q + 1) ** dim * rsz + normals
        face = u + tr + tr + geo if viscous else 0   # state, neighbour traces, flux write, metrics
        resid = u + tr + (tr if viscous else 0) + geo + rk + tr
        total += n * (face + resid)
    return total


WORKLOADS = {
    "tgv32_p3": "3D Taylor-Green vortex Re=1600 M=0.1, periodic 32^3 hexes, FR p=3 (2,097,152 DOF), "
                "Rusanov+BR2, RK4 dt=2.5e-4",
    "tgv32_p4": "3D Taylor-Green vortex Re=1600 M=0.1, periodic 32^3 hexes, FR p=4 (4,096,000 DOF), "
                "Rusanov+BR2, RK4 dt=1.5e-4",
    "naca100k_p3": "NACA 2412 (m=0.02, p=0.4, t=0.12) spanwise-periodic O-grid, 250x100x4 = 100,000 quadratic "
                   "hexes, span 0.2c, FR p=3 (6,400,000 DOF), Re=23000, M=0.2, AoA 3 deg, 1% seeded noise, "
                   "RK4 dt=1.37e-6 (advective+viscous CFL estimate), wall forces and an 18,840-point FW-H cylinder (r=1.5c) sampled "
                   "every step",
    "monopole125k_p3": "Appendix D.1 monopole in a quiescent box: [-5,5]^3, 50^3 = 125,000 hexes, FR p=3 "
                       "(8,000,000 DOF), Euler, characteristic far field, Gaussian energy source A=0.05, k=100, "
                       "f=0.5 at the centre (Eq. D.1), rho=1, p=1/gamma (c=1), RK4 dt=0.00625, a 1.5-radius FW-H "
                       "sphere sampled every step",
    "batch12_p3": "12 NACA 4-digit candidates (PCG64 seed 1: m~U[0,0.06], p~U[0.2,0.6], t~U[0.08,0.16], "
                  "20k-80k quadratic hexes each, 599,888 in total, 38.4M DOF) in one context, FR p=3, Re=23000, "
                  "M=0.2, AoA 3 deg, RK4 at each candidate's own stable dt (0.27e-6..2.0e-6), forces and one FW-H "
                  "cylinder per candidate every step",
}


def build_workload(name):
    """(meshes, options(prec), initial state(ctx), surfaces per candidate, curved flag)."""
    from paper_2501_05709_gb300 import cases as C
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import workloads as W
    if name.startswith("tgv32"):
        p = 3 if name.endswith("p3") else 4
        dt = 2.5e-4 if p == 3 else 1.5e-4
        nodes, conn = W.box_mesh(3, 32, 0.0, 2 * math.pi, q=1)
        p_inf = 1.0 / (GAMMA * MACH ** 2)

        def opts(prec):
            return F.options(order=p, precision=prec, viscous=True, mu=1.0 / 1600.0, p_inf=p_inf, dt=dt)

        def state(ctx):
            return np.ascontiguousarray(np.moveaxis(W.taylor_green(F.fr_sp_coords(ctx), mach=MACH), 0, 1))
        return [(nodes, conn)], opts, state, [], False, None
    if name == "monopole125k_p3":
        nodes, conn, o32, free = C.monopole_box_setup(50, 3, F.FR_FP32)
        rho, vel, pinf = free

        def opts(prec):
            return C.monopole_box_setup(50, 3, prec)[2]

        def state(ctx):
            return W.perturbed_uniform(ctx.nelem, ctx.nsp, rho, vel, pinf, amplitude=0.0)
        surf = W.sphere_surface(1.5, 30, 2 * np.pi / 45)[0]
        return [(nodes, conn)], opts, state, [surf], False, None
    if name == "naca100k_p3":
        params = [{"naca": (0.02, 0.4, 0.12), "n_theta": 250, "n_r": 100}]
    elif name == "batch12_p3":
        params = C.batch_params(12, seed=1)
    else:
        raise SystemExit(f"unknown workload {name}")
    meshes, free, dts = [], None, []
    for prm in params:
        nodes, conn, _, free = C.naca_setup(naca=prm["naca"], n_theta=prm["n_theta"], n_r=prm["n_r"])
        meshes.append((nodes, conn))
        dts.append(C.stable_dt(nodes, prm["n_theta"]))
    rho, vel, pinf = free

    def opts(prec):
        return C.naca_options(precision=prec, dt=3e-6)[0]

    def state(ctx):
        return np.concatenate([W.perturbed_uniform(len(n), ctx.nsp, rho, vel, pinf, amplitude=0.01, seed=k)
                               for k, (n, _) in enumerate(meshes)])
    surf = W.cylinder_surface(radius=1.5, center=(0.5, 0.0), spacing=0.01, span=0.2)[0]
    return meshes, opts, state, [surf] * len(meshes), True, dts


def max_over_ranks_of(x, world, device):
    """The largest x over the ranks of the default process group (the job's
    time is its slowest replica's); x itself on one rank."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, seconds_max, world):
    """Whole-job rate of N independent replicas: every rank's units over the
    slowest rank's time."""
    return world * units_per_rank / seconds_max


def ctx_viscous(o):
    return int(o.viscous)


def gpu_leg(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2501_05709_gb300 import build as B
    from paper_2501_05709_gb300 import cases as C
    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    B.build()
    meshes, opts, state_of, surfaces, curved, dts = build_workload(args.workload)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    prec = {"fp32": F.FR_FP32, "tf32": F.FR_TF32_TC, "bf16x3": F.FR_BF16X3_TC, "fp64": F.FR_FP64}[args.precision]
    rsz = 8 if prec == F.FR_FP64 else 4
    ctx = F.fr_mesh_load(meshes, opts(prec))
    for k, d in enumerate(dts or []):
        F.fr_set_cand_dt(ctx, k, d)
    if args.workload.startswith("monopole"):
        F.fr_set_source(ctx, 0, C.MONOPOLE_SOURCE, 0.0)
    orders = None
    if args.sponge:
        # far-field sponge of reduced degree on the O-grid candidates
        if not args.workload.startswith(("naca", "batch")):
            raise SystemExit("--sponge needs an O-grid workload (naca100k_p3, batch12_p3)")
        orders = np.concatenate([W.sponge_orders(n, ctx.order) for n, _ in meshes])
        F.fr_set_element_order(ctx, orders)
    viscous = bool(ctx_viscous(opts(prec)))
    p = ctx.order
    u0 = state_of(ctx)
    E, nsp = ctx.nelem, ctx.nsp
    dof = E * nsp
    F.fr_state_set(ctx, u0)
    cap = args.warmup + 3 * args.steps + 8
    for k, srf in enumerate(surfaces):
        F.fwh_register(ctx, k, srf, cap, 1)
    if args.tile > 0:
        F.fr_set_tile(ctx, args.tile)
        tile = args.tile
    else:
        tile = F.fr_autotune(ctx)
    F.fr_state_set(ctx, u0)
    F.fr_rk_step_graph(ctx, args.warmup, sh)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(x):
        return max_over_ranks_of(x, world, "cuda")

    clocks = Clocks(local_rank) if rank == 0 else None
    time.sleep(0.3)
    n0 = F.fr_launch_count(ctx)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    F.fr_rk_step_graph(ctx, args.steps, sh)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1))
    launches = F.fr_launch_count(ctx) - n0
    ck = clocks.stop() if clocks else None
    value = replica_throughput(dof * 4 * args.steps, ms / 1e3, world)

    # per-kernel durations over as many further steps, inside graph replay
    # (one step captured with an event record node around every kernel).  The
    # event nodes add a few microseconds to every kernel, so the per-kernel
    # times are also scaled to the plain graph's measured step time (the
    # shares from the instrumented replay, the total from the timed region);
    # the roofline uses the scaled times, the raw ones are reported beside.
    kms_raw, kn = F.fr_profile_step(ctx, args.steps, sh)
    ev_step = sum(kms_raw) / args.steps
    # (with reduced-degree elements the timed step runs their kernels beside
    # the degree-p ones, the instrumented replay one after the other, so the
    # two totals are not comparable and the per-kernel times stay unscaled)
    scale = min(1.0, (ms / args.steps) / ev_step) if ev_step > 0 and orders is None else 1.0
    kms = [k * scale for k in kms_raw]
    hbm, peak_kind = peaks()
    ab = algorithmic_bytes(E, p, rsz, viscous=viscous, curved=curved)
    resid_ms = kms[2] / max(kn[2], 1)
    achieved = ab["resid"] / (resid_ms / 1e3) / 1e9
    def kstat(i, key):
        avg = kms[i] / max(kn[i], 1)
        return {"avg_ms": avg, "avg_ms_event_nodes": kms_raw[i] / max(kn[i], 1), "launches": int(kn[i]),
                "gbs": (ab[key] / (avg / 1e3) / 1e9) if avg > 0 else None}

    kernels = {"traces": kstat(0, "traces"), "visc_face": kstat(1, "visc"), "residual_rk": kstat(2, "resid")}
    if orders is not None:
        # the reduced-degree elements run their own face and residual kernels:
        # their time per element and stage against that of the full-degree
        # elements (face + residual kernels)
        nred = int((orders < p).sum())
        stages = 4 * args.steps
        red_ms = kms[5] / stages
        full_ms = (kms[1] + kms[2]) / stages
        rb = reduced_bytes(orders, p, rsz, viscous=viscous, curved=curved)
        kernels["reduced_degree"] = {
            "avg_ms": kms[5] / max(kn[5], 1), "launches": int(kn[5]), "elements": nred,
            "gbs": rb / (red_ms / 1e3) / 1e9 if red_ms > 0 else None,
            "algorithmic_bytes_per_stage": rb,
            "degrees": np.bincount(orders, minlength=p + 1).tolist(),
            "dof_native": int(sum((int(q) + 1) ** 3 for q in orders)),
            "us_per_element_stage": 1e3 * red_ms / max(nred, 1),
            "full_degree_us_per_element_stage": 1e3 * full_ms / max(E - nred, 1)}
    u32 = F.fr_state_get(ctx)
    steps_done = args.warmup + 2 * args.steps
    # per-candidate wall forces accumulated over the same steps (C_L, C_D,
    # mean C_L, mean C_D, steps)
    walls = args.workload.startswith(("naca", "batch"))
    forces32 = [F.fr_forces(ctx, k) for k in range(ctx.ncand)] if walls else None

    # end to end through the C-ABI: pinned host state in, step, KE integral out
    host = torch.empty(u0.shape, dtype=torch.float64, pin_memory=True)
    host.numpy()[...] = u0
    hnp = host.numpy()
    F.fr_state_set(ctx, hnp, stream=sh)
    F.fr_rk_step_graph(ctx, 1, sh)
    F.fr_integrals(ctx)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        F.fr_state_set(ctx, hnp, stream=sh)
        F.fr_rk_step_graph(ctx, 1, sh)
        F.fr_integrals(ctx)
    torch.cuda.synchronize()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": replica_throughput(dof * 4 * args.steps, e2e_s, world), "unit": UNIT,
           "h2d_bytes_per_step": int(u0.nbytes), "d2h_bytes_per_step": int(8 * 6 * min(1024, (dof + 255) // 256))}
    ctx.close()

    # FP64 path, same workload, same number of steps
    fp64 = None
    if not args.no_fp64 and prec != F.FR_FP64:
        c64 = F.fr_mesh_load(meshes, opts(F.FR_FP64))
        for k, d in enumerate(dts or []):
            F.fr_set_cand_dt(c64, k, d)
        if args.workload.startswith("monopole"):
            F.fr_set_source(c64, 0, C.MONOPOLE_SOURCE, 0.0)
        if orders is not None:
            F.fr_set_element_order(c64, orders)
        F.fr_state_set(c64, u0)
        for k, srf in enumerate(surfaces):
            F.fwh_register(c64, k, srf, cap, 1)
        if args.tile > 0:
            F.fr_set_tile(c64, args.tile)
        else:
            F.fr_autotune(c64)
        F.fr_state_set(c64, u0)
        F.fr_rk_step_graph(c64, args.warmup, sh)
        torch.cuda.synchronize()
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        F.fr_rk_step_graph(c64, args.steps, sh)
        b.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms64 = max_over_ranks(a.elapsed_time(b))
        # per-kernel times over the same number of steps as the FP32 leg's
        # profile, which also brings the FP64 state to the FP32 state's step
        kms64, kn64 = F.fr_profile_step(c64, args.steps, sh)
        dfma_peak = F.fr_probe_fp64_peak(sh)
        u64 = F.fr_state_get(c64)
        dev = float(np.linalg.norm(u32 - u64) / np.linalg.norm(u64))
        ke = F.fr_integrals(c64)[-1]
        forces64 = [F.fr_forces(c64, k) for k in range(c64.ncand)] if forces32 is not None else None
        c64.close()
        fp64 = {"value": replica_throughput(dof * 4 * args.steps, ms64 / 1e3, world), "unit": UNIT, "ms_per_step": ms64 / args.steps,
                "fp32_state_rel_l2_vs_fp64": dev, "steps_compared": steps_done, "ke_fp64": ke}
        if forces32 is not None:
            per = [{"cl_mean_fp64": f64[2], "cl_mean_fp32": f32[2], "cd_mean_fp64": f64[3], "cd_mean_fp32": f32[3]}
                   for f32, f64 in zip(forces32, forces64)]
            fp64["per_candidate_forces"] = per
            fp64["max_abs_dev_cl_mean"] = max(abs(d["cl_mean_fp32"] - d["cl_mean_fp64"]) for d in per)
            fp64["max_abs_dev_cd_mean"] = max(abs(d["cd_mean_fp32"] - d["cd_mean_fp64"]) for d in per)
            fp64["force_steps"] = int(forces64[0][4])
        # FP64 kernels are bound by the FP64 pipe: executed FP64 flops per
        # launch (ncu: 2 DFMA + DADD + DMUL, stage average) against the DFMA
        # rate measured on this GPU
        ev64 = sum(kms64) / args.steps
        s64 = min(1.0, (ms64 / args.steps) / ev64) if ev64 > 0 else 1.0
        r64 = s64 * kms64[2] / max(kn64[2], 1)
        fl = ncu_counter(args.workload, "fp64", "k_residual", "fp64_flops_per_launch")
        ach = fl / (r64 / 1e3) / 1e9 if fl else None
        fp64["roofline"] = {"bound": "alu", "kernel": "k_residual (FR residual + RK4 stage), FP64",
                            "achieved": ach, "peak": dfma_peak, "unit": "GFLOP/s",
                            "frac": ach / dfma_peak if ach else None,
                            "peak_source": "measured: FP64 FMA throughput probe (fr_probe_fp64_peak) on this GPU",
                            "flops_per_launch": fl, "avg_launch_ms": r64,
                            "traffic": ncu_counter(args.workload, "fp64", "k_residual", "dram_bytes_per_launch")}
    roof = {"bound": "hbm", "kernel": "k_residual (FR residual + RK4 stage)", "achieved": achieved,
            "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "avg_launch_ms": resid_ms, "avg_launch_ms_event_nodes": kms_raw[2] / max(kn[2], 1),
            "timing": ("per-kernel share from a graph replay with event nodes around each kernel, scaled to the "
                       "timed graph's ms per step (factor %.4f)" % scale) if orders is None else
                      "per-kernel times from a graph replay with event nodes around each kernel, every kernel on "
                      "its own (the timed step runs the reduced-degree kernels beside the degree-p ones)",
            "traffic": ncu_counter(args.workload, args.precision, "k_residual", "dram_bytes_per_launch"),
            "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
            "algorithmic_bytes_per_launch": ab["resid"]}
    if prec == F.FR_FP64:
        # the FP64 kernels are bound by the FP64 pipe (see the fp64 leg below)
        pk = F.fr_probe_fp64_peak(sh)
        fl = ncu_counter(args.workload, "fp64", "k_residual", "fp64_flops_per_launch")
        ach = fl / (resid_ms / 1e3) / 1e9 if fl else None
        roof = {"bound": "alu", "kernel": "k_residual (FR residual + RK4 stage), FP64", "achieved": ach, "peak": pk,
                "unit": "GFLOP/s", "frac": ach / pk if ach else None,
                "traffic": roof["traffic"],
                "peak_source": "measured: FP64 FMA throughput probe (fr_probe_fp64_peak) on this GPU",
                "flops_per_launch": fl}
    return {
        "value": value, "ms": ms, "launches": launches, "clocks": ck, "kernels": kernels, "tile_epb": tile,
        "roofline": roof,
        "e2e": e2e, "fp64": fp64, "dof": dof, "elements": E,
    }


def fwh_leg():
    """FW-H post-processing at the directivity scale of Section 3.3: the
    18,840-panel cylinder of the airfoil workloads, 36 observers on the
    r = 10c circle, the surface duplicated to 3 spans, a 1000-sample record of
    a seeded moving-medium monopole field (nondimensional: |V| = 1, M = 0.2,
    AoA 3 deg); then the Welch PSD of every observer series."""
    import torch

    from paper_2501_05709_gb300 import fr as F
    from paper_2501_05709_gb300 import workloads as W
    y, n, dS = W.cylinder_surface(radius=1.5, center=(0.5, 0.0), spacing=0.01, span=0.2)
    nt, dt, c0, a = 1000, 0.002, 5.0, math.radians(3.0)
    M = [0.2 * math.cos(a), 0.2 * math.sin(a), 0.0]
    tau = dt * np.arange(nt)
    fld = W.monopole_field(y[None], tau[:, None], M, A=1e-3, omega=4 * np.pi, c0=c0, rho0=1.0)
    hist = np.concatenate([fld["rho"][..., None], fld["vel"], fld["p"][..., None]], axis=-1)
    ang = np.radians(np.arange(0, 360, 10))
    obs = np.stack([0.5 + 10.0 * np.cos(ang), 10.0 * np.sin(ang), np.full_like(ang, 0.1)], axis=1)
    d = lambda x: torch.tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")
    hd, yd, nd, sd = d(hist), d(y), d(n), d(dS)
    args = (hd, yd, nd, sd, dt, 0.0, obs, M, c0, 1.0, fld["p0"])
    F.fwh_integrate(*args, Lspan=0.2, ncopies=3)           # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p_out, nt_out, _ = F.fwh_integrate(*args, Lspan=0.2, ncopies=3)
    torch.cuda.synchronize()
    t_int = time.perf_counter() - t0
    nmin = int(nt_out.min())
    F.fwh_psd(p_out, dt, nseg=3, nt=nmin)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    F.fwh_psd(p_out, dt, nseg=3, nt=nmin)
    torch.cuda.synchronize()
    t_psd = time.perf_counter() - t0
    work = len(y) * len(obs) * 3 * nt
    # FP64-bound: executed FP64 flops of one call (ncu, all FW-H kernels)
    # against the FP64 FMA rate measured on this GPU; the time is the whole call
    fl = ncu_counter("fwh_directivity", "fp64", "fwh_integrate", "fp64_flops_per_call")
    pk = F.fr_probe_fp64_peak()
    ach = fl / t_int / 1e9 if fl else None
    return {"panels": int(len(y)), "observers": int(len(obs)), "copies": 3, "samples": nt,
            "window_samples_min": nmin, "fwh_integrate_ms": 1e3 * t_int,
            "panel_observer_copy_samples_per_s": work / t_int, "fwh_psd_ms": 1e3 * t_psd,
            "roofline": {"bound": "alu", "kernel": "fwh_integrate (k_fwh_series + k_fwh_accum + k_fwh_reduce), FP64",
                         "achieved": ach, "peak": pk, "unit": "GFLOP/s", "frac": ach / pk if ach else None,
                         "flops_per_call": fl,
                         "peak_source": "measured: FP64 FMA throughput probe (fr_probe_fp64_peak) on this GPU"},
            "note": "host wall time around each call (each call synchronises and includes its scratch set-up "
                    "and the host-side observer windows)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fwh", action="store_true", help="skip the FW-H/PSD post-processing timing")
    ap.add_argument("--no-config4", action="store_true",
                    help="skip the p=4 leg (FP32, TF32 and BF16x3 tensor-core modes) of the default run")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched 12-candidate leg (timed after the headline workload)")
    ap.add_argument("--tile", type=int, default=0, help="elements per block (0: autotune)")
    ap.add_argument("--sponge", action="store_true",
                    help="O-grid workloads: degree p near the body down to 0 at the far field (4c/6c/8c)")
    ap.add_argument("--workload", default="tgv32_p3", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tf32", "bf16x3", "fp64"],
                    help="precision of the timed path (fp32; tf32 / bf16x3: fp32 with the residual's line "
                         "operators on the tensor cores; the reduced modes also time fp64 beside them)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    config = {"workload": args.workload, "description": WORKLOADS[args.workload],
              "step": "one RK4 step = 4 residual stages (fused stage updates; forces and FW-H sampling "
                      "every step where the workload has walls/surfaces)",
              "l2": "working set larger than L2 (no flush needed)", "parallelism": f"replicas x{world}"}

    if args.impl == "reference":
        if rank != 0:
            return
        # each step: one RK4 step of the 8^3-element sample of the same workload
        # (exactly --steps timed steps after --warmup untimed ones)
        cb = run_oracle_subprocess(min_seconds=0.0, max_steps=args.steps, warmup=args.warmup)
        line = {"metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * cb["seconds"] / max(cb["steps_timed"], 1),
                "impl": "reference", "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                            "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    r = gpu_leg(args, rank, world, local_rank)
    batched = None
    if not args.no_batched and args.workload != "batch12_p3":
        bargs = argparse.Namespace(**vars(args))
        bargs.workload, bargs.sponge, bargs.tile = "batch12_p3", False, 0
        rb = gpu_leg(bargs, rank, world, local_rank)
        batched = {"workload": "batch12_p3", "description": WORKLOADS["batch12_p3"], "value": rb["value"],
                   "unit": UNIT, "ms_per_step": rb["ms"] / args.steps, "steps": args.steps, "warmup": args.warmup,
                   "dtype": {"fp32": "f32", "tf32": "f32+tf32-tc", "bf16x3": "f32+bf16x3-tc", "fp64": "f64"}[args.precision], "elements": rb["elements"],
                   "dof_per_variable": rb["dof"], "autotuned_elements_per_block": rb["tile_epb"],
                   "gpu_launches": rb["launches"], "clocks": rb["clocks"], "roofline": rb["roofline"],
                   "kernels": rb["kernels"], "e2e": rb["e2e"], "fp64": rb["fp64"],
                   "note": "the FW-H window at an observer 10c away needs ~0.6 convective times, far more than "
                           "these steps cover; OASPL mixed vs FP64 per candidate comes from the batched precision "
                           "study (cases.py batch-precision)"}
    # config 4: the TGV box at p=4 in FP32 (with its FP64 counterpart) and in
    # the two tensor-core line-operator modes
    config4 = None
    if not args.no_config4 and args.workload == "tgv32_p3" and args.precision == "fp32":
        config4 = {"workload": "tgv32_p4", "description": WORKLOADS["tgv32_p4"], "steps": args.steps,
                   "warmup": args.warmup, "modes": {}}
        for mode in ("fp32", "tf32", "bf16x3"):
            m4 = argparse.Namespace(**vars(args))
            m4.workload, m4.precision, m4.sponge, m4.tile = "tgv32_p4", mode, False, 0
            m4.no_fp64 = args.no_fp64 or mode != "fp32"
            try:
                r4 = gpu_leg(m4, rank, world, local_rank)
            except Exception as e:  # reported, not fatal: the headline line still prints
                config4["modes"][mode] = {"error": str(e)[-300:]}
                continue
            config4["modes"][mode] = {
                "value": r4["value"], "unit": UNIT, "ms_per_step": r4["ms"] / args.steps,
                "dtype": {"fp32": "f32", "tf32": "f32+tf32-tc", "bf16x3": "f32+bf16x3-tc"}[mode],
                "roofline": r4["roofline"], "kernels": r4["kernels"], "clocks": r4["clocks"], "fp64": r4["fp64"]}
    fwh = None
    if rank == 0 and not args.no_fwh:
        try:
            fwh = fwh_leg()
        except Exception as e:  # reported, not fatal
            fwh = {"error": str(e)[-300:]}
    if rank == 0:
        cb = None
        cb_all = None
        if not args.no_cpu_baseline:
            try:
                cb = run_oracle_subprocess(min_seconds=10.0)
            except Exception as e:  # reported, not fatal
                cb = {"value": None, "error": str(e)[-300:]}
            try:
                cb_all = run_oracle_all_cores(min_seconds=10.0)
            except Exception as e:
                cb_all = {"value": None, "error": str(e)[-300:]}
        if args.sponge:
            config["sponge"] = "element degree p inside 4c of (0.5, 0), then p-1, p-2, p-3 (>= 0) past 4c, 6c, 8c"
        config["autotuned_elements_per_block"] = r["tile_epb"]
        config["elements"] = r["elements"]
        config["dof_per_variable"] = r["dof"]
        line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "tf32": "f32+tf32-tc", "bf16x3": "f32+bf16x3-tc", "fp64": "f64"}[args.precision],
                "data": "synthetic", "config": config, "roofline": r["roofline"], "cpu_baseline": cb, "e2e": r["e2e"], "gpu_launches": r["launches"],
                "clocks": r["clocks"], "kernels": r["kernels"], "fp64": r["fp64"], "cpu_baseline_all_cores": cb_all,
                "batched": batched, "config4": config4, "fwh": fwh}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
