"""Drivers for the airfoil workloads on the C-ABI: one NACA 4-digit candidate
(mean lift/drag, FW-H surface samples, OASPL at a far-field observer) and a
batch of candidates advanced together in one context, as one MADS poll does
(paper Section 2.2 and Section 3.4: 2n candidates evaluated concurrently).

Everything numerical runs in libfr; this module only builds inputs, calls the
library and reduces its outputs.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import fr as F
from . import workloads as W

GAMMA = 1.4


def naca_options(span=0.2, mach=0.2, aoa_deg=3.0, reynolds=23000.0, order=3, precision=F.FR_FP32, dt=3e-6):
    """Options and free stream (rho=1, |V|=1 at the angle of attack, chord 1)."""
    rho, vel, p = W.freestream(mach, aoa_deg)
    a = math.radians(aoa_deg)
    opts = F.options(order=order, precision=precision, viscous=True, mu=rho * 1.0 * 1.0 / reynolds,
                     rho_inf=rho, p_inf=p, vel_inf=tuple(vel), dt=dt,
                     lift_dir=(-math.sin(a), math.cos(a), 0.0), drag_dir=(math.cos(a), math.sin(a), 0.0),
                     ref_area=1.0 * span)
    return opts, (rho, vel, p)


def naca_setup(naca=(0.02, 0.4, 0.12), n_theta=250, n_r=100, n_z=4, span=0.2, r_outer=10.0, first_cell=2e-3,
               mach=0.2, aoa_deg=3.0, reynolds=23000.0, order=3, precision=F.FR_FP32, dt=3e-6):
    """Mesh (quadratic O-grid), options and free stream of one candidate."""
    nodes, conn = W.ogrid_mesh(n_theta, n_r, n_z, span, r_outer=r_outer, first_cell=first_cell, body="naca",
                               naca=naca)
    opts, free = naca_options(span, mach, aoa_deg, reynolds, order, precision, dt)
    return nodes, conn, opts, free


def first_cell_thickness(nodes, n_theta):
    """Smallest wall-normal thickness of the first element ring of an O-grid
    (elements 0..n_theta-1 of the first spanwise layer, nodes at xi_2 = -1, +1)."""
    X = np.asarray(nodes)[:n_theta].reshape(n_theta, 3, 3, 3, 3)
    wall = X[:, 0, 0, :, :2]
    off = X[:, 0, 2, :, :2]
    t = wall[:, 2] - wall[:, 0]
    t /= np.linalg.norm(t, axis=1)[:, None]
    nrm = np.stack([-t[:, 1], t[:, 0]], axis=1)
    return float(np.abs(np.einsum("ij,ij->i", off[:, 1] - wall[:, 1], nrm)).min())


def stable_dt(nodes, n_theta, mach=0.2, order=3, reynolds=23000.0, cfl=0.8):
    """Explicit RK4 step estimate from the advective and viscous rates of the
    thinnest first-ring cell: dt = cfl / ((p+1)^2 (|V| + c) / h + (p+1)^4 nu / h^2)
    with |V| = 1, c = 1/M, nu = 1/Re and h the wall-normal thickness."""
    h = first_cell_thickness(nodes, n_theta)
    k = (order + 1) ** 2
    return cfl / (k * (1.0 + 1.0 / mach) / h + k * k / reynolds / (h * h))


def oaspl_from_history(hist, surface, dtau, observer, free, mach_vec, span, ncopies, stream=None):
    """FW-H (libfr fwh_integrate) of a history [nrec, npts, 5] -> (t*, p', p'_rms,
    OASPL in dB re 20 uPa with p_inf scaled to 101325 Pa), or raises FrError
    (FR_EWINDOW) when the record is too short for the observer window."""
    import torch
    rho, vel, p = free
    c0 = math.sqrt(GAMMA * p / rho)
    y, n, dS = surface
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    pout, nt, t0 = F.fwh_integrate(dev(hist), dev(y), dev(n), dev(dS), dtau, 0.0, np.asarray(observer)[None],
                                   mach_vec, c0, rho, p, Lspan=span, ncopies=ncopies, stream=stream)
    pp = pout[0, :nt[0]].cpu().numpy()
    prms = float(np.sqrt(np.mean((pp - pp.mean()) ** 2)))
    oaspl = 20.0 * math.log10(max(prms, 1e-300) * (101325.0 / p) / 2e-5)
    return t0[0] + dtau * np.arange(nt[0]), pp, prms, oaspl


def run_naca(steps=2000, precision=F.FR_FP32, sample_every=1, ncopies=1, observer=(1.0, -10.0, 0.1),
             surface_radius=1.5, seed=0, graph=True, **mesh_kw):
    """One candidate: perturbed free stream (1% seeded velocity noise), `steps`
    RK4 steps, forces every step, the FW-H surface sampled every
    `sample_every` steps, then FW-H at the observer.  Returns a dict."""
    if mesh_kw.get("dt") is None:
        mesh_kw.pop("dt", None)
        probe = W.ogrid_mesh(mesh_kw.get("n_theta", 250), 1, 1, mesh_kw.get("span", 0.2),
                             r_outer=mesh_kw.get("r_outer", 10.0), first_cell=mesh_kw.get("first_cell", 2e-3),
                             naca=mesh_kw.get("naca", (0.02, 0.4, 0.12)))[0]
        mesh_kw["dt"] = stable_dt(probe, mesh_kw.get("n_theta", 250))
    nodes, conn, opts, free = naca_setup(precision=precision, **mesh_kw)
    span = mesh_kw.get("span", 0.2)
    rho, vel, p = free
    surface = W.cylinder_surface(radius=surface_radius, center=(0.5, 0.0), spacing=0.01, span=span)
    out = {"elements": len(nodes), "steps": steps, "precision": "fp32" if precision == F.FR_FP32 else "fp64"}
    with F.fr_mesh_load((nodes, conn), opts) as ctx:
        u0 = W.perturbed_uniform(ctx.nelem, ctx.nsp, rho, vel, p, amplitude=0.01, seed=seed)
        F.fr_state_set(ctx, u0)
        cap = (steps + sample_every - 1) // sample_every
        h = F.fwh_register(ctx, 0, surface[0], cap, sample_every)
        import torch
        torch.cuda.synchronize()
        t = time.perf_counter()
        (F.fr_rk_step_graph if graph else F.fr_rk_step)(ctx, steps)
        torch.cuda.synchronize()
        out["seconds"] = time.perf_counter() - t
        out["dof_stages_per_s"] = ctx.nelem * ctx.nsp * 4 * steps / out["seconds"]
        f = F.fr_forces(ctx, 0)
        out.update(cl=f[0], cd=f[1], cl_mean=f[2], cd_mean=f[3], force_steps=int(f[4]))
        hist = F.fwh_history(ctx, h, len(surface[0]))
        out["records"] = hist.shape[0]
        final = F.fr_state_get(ctx)
        out["finite"] = bool(np.isfinite(final).all())
    c0 = math.sqrt(GAMMA * p / rho)
    mach_vec = np.asarray(vel) / c0
    try:
        _, pp, prms, oaspl = oaspl_from_history(hist, surface, opts.dt * sample_every, observer, free, mach_vec,
                                                span, ncopies)
        out.update(prms=prms, oaspl_db=oaspl, window=len(pp))
    except F.FrError as e:
        out.update(prms=None, oaspl_db=None, window=0, fwh_error=str(e))
    out["history"] = hist
    return out


def batch_params(n=12, seed=1):
    """Seeded MADS-poll candidates: camber m ~ U[0, 0.06], its position
    p ~ U[0.2, 0.6], thickness t ~ U[0.08, 0.16], element count ~ U[20k, 80k]
    realised as n_theta x n_r x 4 with n_r = 2 n_theta / 5."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        m = rng.uniform(0.0, 0.06)
        pc = rng.uniform(0.2, 0.6)
        t = rng.uniform(0.08, 0.16)
        ne = rng.uniform(20000, 80000)
        nt = int(round(math.sqrt(ne / 4 * 5 / 2)))
        nr = max(4, int(round(ne / 4 / nt)))
        out.append({"naca": (m, pc, t), "n_theta": nt, "n_r": nr})
    return out


def run_batch(params, steps, precision=F.FR_FP32, dt=None, sample_every=1, surface_radius=1.5, seed=0,
              graph=True):
    """All candidates in one context (concatenated elements; one graph-replayed
    launch sequence per RK4 step), each at its own stable time step unless dt
    is given.  Returns per-candidate mean C_L, C_D, the histories and the
    throughput."""
    import torch
    meshes, frees, opts, dts = [], None, None, []
    for k, prm in enumerate(params):
        nodes, conn, o, free = naca_setup(naca=prm["naca"], n_theta=prm["n_theta"], n_r=prm["n_r"],
                                         precision=precision, dt=dt)
        meshes.append((nodes, conn))
        frees, opts = free, o
        dts.append(stable_dt(nodes, prm["n_theta"]) if dt is None else dt)
    rho, vel, p = frees
    surface = W.cylinder_surface(radius=surface_radius, center=(0.5, 0.0), spacing=0.01, span=0.2)
    res = {"candidates": len(params), "elements": [len(n) for n, _ in meshes], "steps": steps, "dt": dts}
    with F.fr_mesh_load(meshes, opts) as ctx:
        for k, d in enumerate(dts):
            F.fr_set_cand_dt(ctx, k, d)
        us = [W.perturbed_uniform(len(n), ctx.nsp, rho, vel, p, amplitude=0.01, seed=seed + k)
              for k, (n, _) in enumerate(meshes)]
        F.fr_state_set(ctx, np.concatenate(us))
        cap = (steps + sample_every - 1) // sample_every
        hs = [F.fwh_register(ctx, k, surface[0], cap, sample_every) for k in range(len(meshes))]
        torch.cuda.synchronize()
        t = time.perf_counter()
        (F.fr_rk_step_graph if graph else F.fr_rk_step)(ctx, steps)
        torch.cuda.synchronize()
        res["seconds"] = time.perf_counter() - t
        res["dof_stages_per_s"] = ctx.nelem * ctx.nsp * 4 * steps / res["seconds"]
        res["forces"] = [F.fr_forces(ctx, k) for k in range(len(meshes))]
        res["histories"] = [F.fwh_history(ctx, h, len(surface[0])) for h in hs]
    return res


def precision_study(steps=25000, dt=4e-5, sample_every=4, n_theta=60, n_r=20, n_z=2, first_cell=2e-2):
    """Mean C_L, C_D and OASPL of one NACA 2412 candidate in FP32 and FP64 on a
    coarse O-grid run for steps*dt convective times (long enough for a
    non-empty FW-H window at the observer 10c below the trailing edge)."""
    out = {}
    for prec, name in ((F.FR_FP64, "fp64"), (F.FR_FP32, "fp32")):
        r = run_naca(steps=steps, precision=prec, sample_every=sample_every, dt=dt, n_theta=n_theta, n_r=n_r,
                     n_z=n_z, first_cell=first_cell)
        r.pop("history")
        out[name] = r
    d = {}
    for key in ("cl_mean", "cd_mean", "oaspl_db", "prms"):
        a, b = out["fp64"].get(key), out["fp32"].get(key)
        if a is not None and b is not None:
            d[key] = {"fp64": a, "fp32": b, "abs_dev": abs(b - a), "rel_dev": abs(b - a) / max(abs(a), 1e-300)}
    out["deviation"] = d
    return out


def batch_precision_study(n=12, seed=1, coarsen=4, n_z=2, first_cell=2e-2, t_end=0.8, sample_every=8,
                          spacing=0.05, ncopies=1, observer=(1.0, -10.0, 0.1)):
    """Per-candidate mean C_L, mean C_D and OASPL of a batched poll in FP32 and
    in FP64: the n seeded sections of the batched workload (``batch_params``)
    on O-grids coarsened by ``coarsen`` in both in-plane directions (uneven
    sizes kept), all candidates in one context, each at its own stable step
    (``stable_dt``), as many steps as the smallest step needs to reach t_end
    convective times (long enough for a non-empty FW-H window at the observer
    10c below the trailing edge), a cylinder surface of the given panel
    spacing sampled every ``sample_every`` steps and ``ncopies`` spanwise
    copies in the FW-H integral."""
    import torch
    params = batch_params(n, seed)
    meshes, dts = [], []
    for prm in params:
        nt, nr = max(8, round(prm["n_theta"] / coarsen)), max(6, round(prm["n_r"] / coarsen))
        nodes, conn = W.ogrid_mesh(nt, nr, n_z, 0.2, first_cell=first_cell, body="naca", naca=prm["naca"])
        meshes.append((nodes, conn))
        dts.append(stable_dt(nodes, nt))
    steps = int(math.ceil(t_end / min(dts) / sample_every)) * sample_every
    surface = W.cylinder_surface(radius=1.5, center=(0.5, 0.0), spacing=spacing, span=0.2)
    res = {"candidates": [{"naca": list(prm["naca"]), "elements": len(m[0]), "dt": d}
                          for prm, m, d in zip(params, meshes, dts)],
           "steps": steps, "t_end_min": steps * min(dts), "sample_every": sample_every, "panels": len(surface[0]),
           "ncopies": ncopies, "observer": list(observer)}
    for prec, name in ((F.FR_FP32, "fp32"), (F.FR_FP64, "fp64")):
        opts, free = naca_options(precision=prec, dt=dts[0])
        rho, vel, p = free
        with F.fr_mesh_load(meshes, opts) as ctx:
            for k, d in enumerate(dts):
                F.fr_set_cand_dt(ctx, k, d)
            us = [W.perturbed_uniform(len(nd), ctx.nsp, rho, vel, p, amplitude=0.01, seed=k)
                  for k, (nd, _) in enumerate(meshes)]
            F.fr_state_set(ctx, np.concatenate(us))
            cap = steps // sample_every + 1
            hs = [F.fwh_register(ctx, k, surface[0], cap, sample_every) for k in range(n)]
            torch.cuda.synchronize()
            t = time.perf_counter()
            F.fr_rk_step_graph(ctx, steps)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t
            forces, flagged = [], []
            for k in range(n):
                try:
                    forces.append(F.fr_forces(ctx, k))
                except F.FrError as e:
                    if e.code != F.FR_ENONFINITE:
                        raise
                    forces.append(None)
                    flagged.append(k)
            hists = [F.fwh_history(ctx, h, len(surface[0])) for h in hs]
            final = F.fr_state_get(ctx) if not flagged else None
            dof = ctx.nelem * ctx.nsp
        c0 = math.sqrt(GAMMA * p / rho)
        out = []
        for k in range(n):
            if forces[k] is None:
                out.append({"nonfinite": True})
                continue
            r = {"cl_mean": forces[k][2], "cd_mean": forces[k][3]}
            try:
                _, pp, prms, oaspl = oaspl_from_history(hists[k], surface, dts[k] * sample_every, observer, free,
                                                        np.asarray(vel) / c0, 0.2, ncopies)
                r.update(oaspl_db=oaspl, prms=prms, window=len(pp))
            except F.FrError as e:
                r.update(oaspl_db=None, prms=None, window=0, fwh_error=str(e))
            out.append(r)
        res[name] = {"per_candidate": out, "seconds": secs, "dof": dof, "dof_stages_per_s": dof * 4 * steps / secs,
                     "nonfinite_candidates": flagged}
        res[name + "_state"] = final
    a, b = res.pop("fp64_state"), res.pop("fp32_state")
    if a is not None and b is not None:
        res["fp32_state_rel_l2_vs_fp64"] = float(np.linalg.norm(b - a) / np.linalg.norm(a))
    dev = []
    for k in range(n):
        d = {}
        for key in ("cl_mean", "cd_mean", "oaspl_db"):
            x, y = res["fp64"]["per_candidate"][k].get(key), res["fp32"]["per_candidate"][k].get(key)
            if x is not None and y is not None:
                d[key] = {"fp64": x, "fp32": y, "abs_dev": abs(y - x)}
        dev.append(d)
    res["deviation"] = dev
    for key in ("cl_mean", "cd_mean", "oaspl_db"):
        v = [d[key]["abs_dev"] for d in dev if key in d]
        if v:
            res["max_abs_dev_" + key] = max(v)
    return res


def precision_modes_study(order=4, n=32, steps=200, dt=1.5e-4, mach=0.1, modes=("fp32", "tf32", "bf16x3")):
    """Taylor-Green vortex (Re 1600) on the periodic n^3 box at FR order p in
    FP64 and in each reduced mode (fp32; tf32 / bf16x3: fp32 with the
    residual's gradient and divergence line operators on the tensor cores):
    the kinetic-energy history over `steps` RK4 steps (every step), its
    dissipation rate -dKE/dt (central differences), the residual of the
    initial state and the final state, each against the FP64 run, and the
    graph-replayed time per step of every mode."""
    import torch
    nodes, conn = W.box_mesh(3, n, 0.0, 2 * math.pi, q=1)
    p_inf = 1.0 / (GAMMA * mach ** 2)
    prec = {"fp64": F.FR_FP64, "fp32": F.FR_FP32, "tf32": F.FR_TF32_TC, "bf16x3": F.FR_BF16X3_TC}
    runs = {}
    for name in ("fp64",) + tuple(modes):
        opts = F.options(order=order, precision=prec[name], viscous=True, mu=1.0 / 1600.0, p_inf=p_inf, dt=dt)
        with F.fr_mesh_load((nodes, conn), opts) as ctx:
            u0 = np.ascontiguousarray(np.moveaxis(W.taylor_green(F.fr_sp_coords(ctx), mach=mach), 0, 1))
            dtype = torch.float64 if name == "fp64" else torch.float32
            ud = torch.tensor(u0, dtype=dtype, device="cuda")
            Rd = torch.empty_like(ud)
            F.fr_residual(ctx, ud, Rd)
            torch.cuda.synchronize()
            R = Rd.double().cpu().numpy()
            del ud, Rd
            F.fr_state_set(ctx, u0)
            ke = [F.fr_integrals(ctx)[-1]]
            for _ in range(steps):
                F.fr_rk_step_graph(ctx, 1)
                ke.append(F.fr_integrals(ctx)[-1])
            final = F.fr_state_get(ctx)
            F.fr_state_set(ctx, u0)
            F.fr_rk_step_graph(ctx, 3)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            F.fr_rk_step_graph(ctx, 20)
            b.record()
            torch.cuda.synchronize()
            runs[name] = {"ke": np.array(ke), "R": R, "final": final, "ms_per_step": a.elapsed_time(b) / 20,
                          "dof": ctx.nelem * ctx.nsp}
    ref = runs["fp64"]
    eps = -np.gradient(ref["ke"], dt)
    out = {"order": order, "n": n, "steps": steps, "dt": dt, "dof": ref["dof"],
           "fp64": {"ms_per_step": ref["ms_per_step"], "ke_final": float(ref["ke"][-1]),
                    "dissipation_final": float(eps[-1])}}
    for name in modes:
        r = runs[name]
        e = -np.gradient(r["ke"], dt)
        out[name] = {
            "ms_per_step": r["ms_per_step"],
            "dof_stages_per_s": r["dof"] * 4 / (r["ms_per_step"] / 1e3),
            "residual_rel_l2_vs_fp64": float(np.linalg.norm(r["R"] - ref["R"]) / np.linalg.norm(ref["R"])),
            "final_state_rel_l2_vs_fp64": float(np.linalg.norm(r["final"] - ref["final"]) /
                                                np.linalg.norm(ref["final"])),
            "ke_max_rel_dev": float(np.max(np.abs(r["ke"] - ref["ke"]) / ref["ke"])),
            "dissipation_max_rel_dev": float(np.max(np.abs(e - eps)) / np.max(np.abs(eps))),
        }
    return out


# ---------------------------------------------------------------- Section 3.4: the optimisation loop
def design_mesh(X, n_theta=60, n_r=20, n_z=2, span=0.2, r_outer=10.0, first_cell=2e-2, pivot=(0.25, 0.0)):
    """O-grid of the design X = [c_max %, position of c_max (tenths), t_max %,
    alpha deg] (Section 3.4).  The angle of attack turns the section nose-up
    about the quarter chord, so that every candidate of a batch shares the
    free stream along x (lift along y, drag along x).  Returns the nodes,
    connectivity and the turned trailing edge."""
    m, pc, t, alpha = float(X[0]) / 100.0, float(X[1]) / 10.0, float(X[2]) / 100.0, float(X[3])
    nodes, conn = W.ogrid_mesh(n_theta, n_r, n_z, span, r_outer=r_outer, first_cell=first_cell, body="naca",
                               naca=(m, pc, t))
    a = math.radians(alpha)
    ca, sa = math.cos(a), math.sin(a)
    x0, y0 = pivot
    X3 = np.array(nodes, float)
    dx, dy = X3[..., 0] - x0, X3[..., 1] - y0
    X3[..., 0] = x0 + ca * dx + sa * dy
    X3[..., 1] = y0 - sa * dx + ca * dy
    te = (x0 + ca * (1.0 - x0), y0 - sa * (1.0 - x0))
    return np.ascontiguousarray(X3), conn, te


def evaluate_designs(designs, steps=25000, dt=4e-5, sample_every=4, precision=F.FR_FP32, mach=0.2,
                     reynolds=23000.0, order=3, ncopies=1, seed=0, **mesh_kw):
    """Mean C_L, mean C_D and the OASPL at the observer 10c below each
    candidate's trailing edge, for all designs advanced together in one
    context (the batched poll).  Returns a list of dicts."""
    import torch
    meshes, tes = [], []
    for X in designs:
        nodes, conn, te = design_mesh(X, **mesh_kw)
        meshes.append((nodes, conn))
        tes.append(te)
    span = mesh_kw.get("span", 0.2)
    opts, free = naca_options(span, mach, 0.0, reynolds, order, precision, dt)
    rho, vel, p = free
    surface = W.cylinder_surface(radius=1.5, center=(0.5, 0.0), spacing=0.01, span=span)
    out = []
    with F.fr_mesh_load(meshes, opts) as ctx:
        us = [W.perturbed_uniform(len(n), ctx.nsp, rho, vel, p, amplitude=0.01, seed=seed + k)
              for k, (n, _) in enumerate(meshes)]
        F.fr_state_set(ctx, np.concatenate(us))
        cap = (steps + sample_every - 1) // sample_every
        hs = [F.fwh_register(ctx, k, surface[0], cap, sample_every) for k in range(len(meshes))]
        F.fr_rk_step_graph(ctx, steps)
        torch.cuda.synchronize()
        forces = []
        for k in range(len(meshes)):
            # a candidate whose run diverged (device non-finite flag) has no
            # forces; the others of the batch keep theirs
            try:
                forces.append(F.fr_forces(ctx, k))
            except F.FrError as e:
                if e.code != F.FR_ENONFINITE:
                    raise
                forces.append(None)
        hists = [F.fwh_history(ctx, h, len(surface[0])) for h in hs]
    c0 = math.sqrt(GAMMA * p / rho)
    mach_vec = np.asarray(vel) / c0
    for k, X in enumerate(designs):
        if forces[k] is None:
            out.append({"design": np.asarray(X, float), "cl_mean": None, "cd_mean": None, "oaspl_db": None,
                        "prms": None, "nonfinite": True})
            continue
        r = {"design": np.asarray(X, float), "cl_mean": forces[k][2], "cd_mean": forces[k][3]}
        observer = (tes[k][0], tes[k][1] - 10.0, 0.5 * span)
        try:
            _, pp, prms, oaspl = oaspl_from_history(hists[k], surface, dt * sample_every, observer, free,
                                                    mach_vec, span, ncopies)
            r.update(oaspl_db=oaspl, prms=prms)
        except F.FrError as e:
            r.update(oaspl_db=None, prms=None, fwh_error=str(e))
        out.append(r)
    return out


def optimize_naca(baseline=(0.0, 4.0, 12.0, 6.0), l0=2, max_iter=3, log=None, **eval_kw):
    """OrthoMADS (Appendix E) on Eq. 8 from the baseline design (NACA 0012 at
    6 degrees by default), every poll evaluated as one batch on the GPU.  A
    candidate without an OASPL (empty FW-H window) counts as infeasible."""
    from . import mads as M
    base = evaluate_designs([baseline], **eval_kw)[0]
    if base["oaspl_db"] is None:
        raise RuntimeError("the baseline run is too short for an FW-H window at the observer")
    cl0, cd0 = base["cl_mean"], base["cd_mean"]
    runs = [base]

    def value(r):
        vals = (r.get("oaspl_db"), r.get("cl_mean"), r.get("cd_mean"))
        if any(v is None or not math.isfinite(v) for v in vals):
            return math.inf
        return M.objective(vals[0], vals[1], vals[2], cl0, cd0)

    def evaluate(points):
        if len(points) == 1 and np.allclose(M.to_design(points[0]), baseline):
            return [M.objective(base["oaspl_db"], cl0, cd0, cl0, cd0)]
        designs = [M.to_design(x) for x in points]
        try:
            res = evaluate_designs(designs, **eval_kw)
        except F.FrError:
            # a candidate whose mesh or run the library rejects fails alone
            res = []
            for X in designs:
                try:
                    res.extend(evaluate_designs([X], **eval_kw))
                except F.FrError as e:
                    res.append({"design": np.asarray(X, float), "error": str(e)})
        runs.extend(res)
        if log:
            log(res)
        return [value(r) for r in res]

    out = M.orthomads(evaluate, M.to_scaled(baseline), l0=l0, max_iter=max_iter)
    return {"baseline": base, "result": out, "design": M.to_design(out.x), "runs": runs}


# ---------------------------------------------------------------- Appendix D.1: monopole in a box
MONOPOLE_SOURCE = [(0.05, 100.0, (0.0, 0.0, 0.0), 0.5)]   # A, k, position, frequency (Eq. D.1)


def monopole_box_setup(n=50, order=3, precision=F.FR_FP32, half=5.0, cfl=0.5):
    """Quiescent Euler box [-half, half]^3 of n^3 hexes with characteristic
    far-field faces (the paper's Riemann-invariant boundaries), free stream at
    rest with rho = 1, p = 1/gamma (c = 1), and the explicit step
    cfl * h / ((p+1)^2 c) (RK4 with this FR discretisation: 0.6 stays stable
    on the quiescent box, 0.8 does not; 0.5 is used).  Returns (nodes, conn,
    options, free stream)."""
    nodes, conn = W.box_mesh(3, n, -half, half, q=1, periodic=[False] * 3, bc_tag=W.BC_FARFIELD)
    rho, vel, p = 1.0, np.zeros(3), 1.0 / GAMMA
    dt = cfl * (2.0 * half / n) / ((order + 1) ** 2 * 1.0)
    opts = F.options(order=order, precision=precision, viscous=False, rho_inf=rho, p_inf=p, vel_inf=(0.0, 0.0, 0.0),
                     dt=dt)
    return nodes, conn, opts, (rho, vel, p)


def run_monopole_box(order=3, n=50, t_end=8.0, precision=F.FR_FP32, observer=(0.0, 3.0, 0.0), radius=1.5,
                     graph=True):
    """Appendix D.1: a monopole (Eq. D.1) at the centre of a quiescent box;
    the acoustic pressure at the observer directly from the flow solution and
    from the FW-H integral over a sphere of the given radius (sampled every
    step).  Returns the two series on the FW-H observer times and their
    relative RMS difference."""
    import torch
    nodes, conn, opts, free = monopole_box_setup(n, order, precision)
    rho, vel, p = free
    surf = W.sphere_surface(radius, 30, 2 * np.pi / 45)
    steps = int(math.ceil(t_end / opts.dt))
    out = {"order": order, "elements": len(nodes), "steps": steps, "dt": opts.dt}
    with F.fr_mesh_load((nodes, conn), opts) as ctx:
        F.fr_state_set(ctx, W.perturbed_uniform(ctx.nelem, ctx.nsp, rho, vel, p, amplitude=0.0))
        F.fr_set_source(ctx, 0, MONOPOLE_SOURCE, 0.0)
        hs = F.fwh_register(ctx, 0, surf[0], steps, 1)
        ho = F.fwh_register(ctx, 0, np.asarray(observer, float)[None], steps, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        (F.fr_rk_step_graph if graph else F.fr_rk_step)(ctx, steps)
        torch.cuda.synchronize()
        out["seconds"] = time.perf_counter() - t0
        out["dof_stages_per_s"] = ctx.nelem * ctx.nsp * 4 * steps / out["seconds"]
        hist = F.fwh_history(ctx, hs, len(surf[0]))            # totals (rho, V, p)
        direct = F.fwh_history(ctx, ho, 1)[:, 0, 4] - p         # p' at the observer
    # sampling happens at the start of each step: record k is the state at t = k dt
    c0 = math.sqrt(GAMMA * p / rho)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    pout, nt, t0w = F.fwh_integrate(dev(hist), dev(surf[0]), dev(surf[1]), dev(surf[2]), opts.dt, 0.0,
                                    np.asarray(observer, float)[None], [0.0, 0.0, 0.0], c0, rho, p)
    hyb = pout[0, :nt[0]].cpu().numpy()
    ts = t0w[0] + opts.dt * np.arange(nt[0])
    # compare where both exist: the FW-H window runs past the last flow sample
    # by the largest surface-to-observer delay
    keep = ts <= opts.dt * (len(direct) - 1)
    ts, hyb = ts[keep], hyb[keep]
    dirp = np.interp(ts, opts.dt * np.arange(len(direct)), direct)
    rms = lambda a: float(np.sqrt(np.mean(a ** 2)))
    out.update(times=ts, direct=dirp, hybrid=hyb, window=int(keep.sum()),
               rel_rms_diff=rms(hyb - dirp) / rms(dirp),
               rel_rms_diff_mean_removed=rms((hyb - hyb.mean()) - (dirp - dirp.mean())) / rms(dirp - dirp.mean()),
               direct_rms=rms(dirp), hybrid_rms=rms(hyb))
    return out


if __name__ == "__main__":
    import json
    import sys
    if len(sys.argv) > 1 and sys.argv[1] == "naca-precision":
        print(json.dumps(precision_study(), default=float))
    elif len(sys.argv) > 1 and sys.argv[1] == "precision-modes":
        print(json.dumps(precision_modes_study(order=int(sys.argv[2]) if len(sys.argv) > 2 else 4), default=float))
    elif len(sys.argv) > 1 and sys.argv[1] == "batch-precision":
        print(json.dumps(batch_precision_study(), default=float))
    elif len(sys.argv) > 1 and sys.argv[1] == "monopole-box":
        res = {}
        for order in (1, 2, 3):
            r = run_monopole_box(order=order, t_end=12.0)
            res[f"p{order}"] = {k: v for k, v in r.items() if not isinstance(v, np.ndarray)}
        print(json.dumps(res, default=float))
    elif len(sys.argv) > 1 and sys.argv[1] == "optimize":
        r = optimize_naca(max_iter=int(sys.argv[2]) if len(sys.argv) > 2 else 3,
                          log=lambda res: print(json.dumps([{k: v for k, v in x.items()} for x in res],
                                                           default=lambda a: np.asarray(a).tolist()), flush=True))
        res = r["result"]
        print(json.dumps({"baseline": {k: v for k, v in r["baseline"].items()}, "design": r["design"].tolist(),
                          "f": res.f, "iterations": res.iterations, "evaluations": res.evaluations,
                          "history": [{k: v for k, v in h.items()} for h in res.history]},
                         default=lambda a: np.asarray(a).tolist()))
    else:
        print("usage: python -m paper_2501_05709_gb300.cases "
              "naca-precision|batch-precision|precision-modes [order]|monopole-box|optimize [iterations]")
