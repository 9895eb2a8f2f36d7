"""Benchmark: MCTDHF time steps per second on the H2 Q4 workload (one GPU per rank).

One "step" is one pass of the whole hot path: the batched Poisson solves of
all pair mean fields, the one- and two-electron integrals and RDMs, the CI
propagation, and the short-iterative Arnoldi orbital step built from the fused
matrix-free operator kernels.  Workload: H2 at R = 1.4 bohr on [-40,40]^3,
20^3 coarse cells refined 5 levels toward each nucleus, Q4 elements, 4 orbitals
(1 alpha + 1 beta electron, 16 determinants), 800 nm 3-cycle sin^2 pulse at
1e14 W/cm^2 along z, dt = 0.02, Krylov dimension 10, CG rtol 1e-10.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs an
independent replica of the workload (weak scaling, no data-path collective).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "h2_q4"
METRIC = "MCTDHF steps/s (FP32 form vs FP64 path at <=1e-6 rel. error; orbital-DoF applies/s alongside)"
UNIT = "steps/s"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def setup_state(pkg, inputs, torch, w):
    """Mesh, solver and the seeded initial state of the workload."""
    import numpy as np
    mesh = pkg.Mesh(*inputs.mesh_args(WORKLOAD))
    X, ml, _ = mesh.tables()
    interior = np.arange(mesh.N) < mesh.n_interior
    # smooth seeded orbitals: the H2 workload specifies no per-point phase noise
    phi0 = inputs.lowdin(inputs.molecular_orbitals(X, interior, w["nuclei"], w["n_orb"], phase_noise=0.0), ml)
    C0 = inputs.initial_ci(w["n_orb"], w["n_alpha"], w["n_beta"])
    solver = pkg.MCTDHF(mesh, w["n_orb"], w["n_alpha"], w["n_beta"], w["m"])
    return mesh, solver, phi0, C0


def max_over_ranks(dist, torch, value, device):
    """The largest value over the ranks (a job's time is its slowest rank's);
    the value itself without a process group."""
    if not dist:
        return float(value)
    tt = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rate(world, ms_per_step):
    """Whole-job steps/s: each of the `world` ranks advances its own replica by
    one step in ms_per_step (the max over ranks)."""
    return world * 1000.0 / ms_per_step


def _timed_form(pkg, torch, solver, state0, precision, args, field, dt, dist, stream, profile=False, t0=0.0,
                warmup=None):
    """Warm up and time K steps of one arithmetic form from a copy of state0
    (at time t0).  With profile, the library's kernel-class event timing runs
    over exactly the timed steps (classes reset after the warm-up)."""
    phi, C, W = (x.clone() for x in state0)
    solver.set_precision(precision)
    solver.set_krylov_tol(args.krylov_tol)
    t = t0
    for _ in range(args.warmup if warmup is None else warmup):
        solver.step(phi, C, W, field(t), dt, cg_rtol=1e-10, cg_max_it=20000)
        t += dt
    torch.cuda.synchronize()
    if profile:
        for c in range(pkg.PROF_COUNT):
            pkg.profile_read(c, reset=True)
        pkg.profile_enable(True)
    import ctypes
    lib = pkg.load_library()
    c0 = ctypes.c_int64(0)
    lib.afem_kernel_launch_count(ctypes.byref(c0))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    infos = []
    ev0.record(stream)
    for _ in range(args.steps):
        infos.append(solver.step(phi, C, W, field(t), dt, cg_rtol=1e-10, cg_max_it=20000))
        t += dt
    ev1.record(stream)
    torch.cuda.synchronize()
    prof = None
    if profile:
        pkg.profile_enable(False)
        prof = {c: pkg.profile_read(c, reset=True) for c in range(pkg.PROF_COUNT)}
    if dist:
        dist.barrier()
    c1 = ctypes.c_int64(0)
    lib.afem_kernel_launch_count(ctypes.byref(c1))
    ms = max_over_ranks(dist, torch, ev0.elapsed_time(ev1) / args.steps, "cuda")
    return dict(ms=ms, infos=infos, state=(phi, C, W), t=t, launches=int(c1.value - c0.value), prof=prof)


def run_batch(torch, pkg, inputs, reps=10, count=64):
    """Batching form: the complex64 orbital operator of `count` seeded uneven
    instances (DoFs log-uniform 5e4..2e6, p 2..4, 1-8 orbitals) in one
    persistent launch replayed from a CUDA graph, against the same instances
    applied one by one (FP32, then the plain FP64 form).  Inputs (~GB) are far
    larger than L2.  Returns the JSON sub-entry."""
    import numpy as np
    ins = inputs.batch_instances(count)
    t0 = time.perf_counter()
    meshes = [pkg.Mesh(*d["mesh_args"]) for d in ins]
    build_s = time.perf_counter() - t0
    rng = np.random.default_rng(inputs.BASE_SEED + 11)
    xs, ys = [], []
    for m, d in zip(meshes, ins):
        a = (rng.standard_normal((m.N, d["n_orb"])) + 1j * rng.standard_normal((m.N, d["n_orb"])))
        xs.append(torch.from_numpy(a.astype(np.complex64)).cuda())
        ys.append(torch.empty_like(xs[-1]))
    E = [d["E"] for d in ins]
    odofs = sum(m.N * d["n_orb"] for m, d in zip(meshes, ins))
    batch = pkg.Batch(meshes)
    stream = torch.cuda.current_stream()

    def timed(fn, r):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(r):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / r * 1e-3

    t_batch = timed(lambda: batch.apply(pkg.OP_H1_C64, xs, ys, E=E, graph=True), reps)
    refs = [torch.empty_like(x) for x in xs]

    def seq32():
        for m, x, y, e in zip(meshes, xs, refs, E):
            pkg.op_apply(m, pkg.OP_H1_C64, x, y, E=e)
    t_seq32 = timed(seq32, reps)
    worst = 0.0
    for y, r in zip(ys, refs):
        worst = max(worst, float(torch.linalg.norm(y - r) / torch.linalg.norm(r)))
    x64 = [x.to(torch.complex128) for x in xs]
    y64 = [torch.empty_like(x) for x in x64]

    def seq64():
        for m, x, y, e in zip(meshes, x64, y64, E):
            pkg.op_apply(m, pkg.OP_H1, x, y, E=e)
    t_seq64 = timed(seq64, max(2, reps // 3))
    tun = batch.tuning()
    batch.close()
    return {"metric": "orbital-DoF applies/s, batched complex64 orbital operator (all instances per launch)",
            "value": odofs / t_batch, "instances": count, "orbital_dofs": int(odofs),
            "dofs": int(sum(m.N for m in meshes)), "cells": int(tun["total_cells"]),
            "ms_per_batch": t_batch * 1e3,
            "one_by_one_fp32": {"value": odofs / t_seq32, "ms": t_seq32 * 1e3},
            "one_by_one_fp64_form": {"value": odofs / t_seq64, "ms": t_seq64 * 1e3},
            "speedup_vs_one_by_one_fp32": t_seq32 / t_batch, "speedup_vs_fp64_form": t_seq64 / t_batch,
            "max_rel_diff_vs_single_instance": worst,
            "tuning": {"schedule": (f"instances' own passes on {tun['grid']} parallel streams" if tun["block"] == 0
                                    else "one persistent launch over all instances' cell groups"),
                       "block": tun["block"], "grid": tun["grid"], "blocks_per_sm": tun["blocks_per_sm"],
                       "candidates_ms": [[b, g, round(t, 4)] for b, g, t in tun["candidates"]],
                       "candidates_key": "[block, grid, ms]; block 0 = per-instance passes on grid parallel streams"},
            "graph": "the chosen schedule (zero, cell pass, M_L^-1 of every instance) captured once, replayed per apply",
            "mesh_build_s": build_s,
            "recipe": "inputs.batch_instances(64): seeded, DoFs log-uniform 5e4..2e6, p in {2,3,4}, "
                      "1-3 nuclei Z 1..8 within 3 bohr, 1-8 orbitals, |E| 0.01..0.08"}


def run_batch_steps(torch, pkg, inputs, count=64, steps=1, dt=0.01, krylov_m=10):
    """Batching form at the level of the time step: one MCTDHF step of each of
    `count` seeded uneven instances (inputs.batch_instances: DoFs log-uniform
    5e4..2e6, p 2..4, 1-3 nuclei Z 1..8, 1-8 orbitals, N_e = min(sum Z, n)
    electrons, at least 2 for n >= 2) per call of afem_batch_stepper_step, precision form, multigrid
    Poisson, one Krylov step of dimension krylov_m per time step (the fixed-
    dimension step, so that every instance's cost per step is bounded).  The
    first call allocates, the next ones tune the stream count; `steps` calls on
    the tuned schedule are timed, against the same instances stepped one by one
    on one stream.  Returns the JSON sub-entry."""
    import numpy as np
    ins = inputs.batch_instances(count)
    t0 = time.perf_counter()
    meshes = [pkg.Mesh(*d["mesh_args"]) for d in ins]
    build_s = time.perf_counter() - t0
    solvers, states, Es = [], [], []
    for m, d in zip(meshes, ins):
        pkg.mesh_set_option(m, pkg.OPT_POISSON_SOLVER, pkg.POISSON_MULTIGRID)
        n = d["n_orb"]
        # N_e = min(sum Z, n), at least 2 when n >= 2: one electron in several
        # orbitals has a rank-one one-body density matrix (no gamma^-1)
        ne = max(min(int(round(sum(z for _, z, _ in d["mesh_args"][4]))), n), min(2, n))
        na, nb = (ne + 1) // 2, ne // 2
        X, ml, _ = m.tables()
        interior = np.arange(m.N) < m.n_interior
        phi = inputs.lowdin(inputs.molecular_orbitals(X, interior, d["mesh_args"][4], n, phase_noise=0.0), ml)
        sv = pkg.MCTDHF(m, n, na, nb, krylov_m)
        sv.set_precision(pkg.PREC_MIXED)
        solvers.append(sv)
        states.append((torch.from_numpy(phi).cuda(), torch.from_numpy(inputs.initial_ci(n, na, nb)).cuda(),
                       torch.zeros((m.N, n * n), dtype=torch.float64, device="cuda")))
        Es.append(d["E"])
    init = [tuple(x.clone() for x in st) for st in states]
    seq_states = [tuple(x.clone() for x in st) for st in states]
    batch = pkg.BatchStepper(solvers)
    args_ = ([st[0] for st in states], [st[1] for st in states], [st[2] for st in states], Es, dt)
    t_tune = time.perf_counter()
    while batch.tuning()["streams"] == 0:
        batch.step(*args_, cg_rtol=1e-10, cg_max_it=20000, raise_on_maxit=False)
    tune_s = time.perf_counter() - t_tune
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _ in range(steps):
        batch.step(*args_, cg_rtol=1e-10, cg_max_it=20000, raise_on_maxit=False)
    torch.cuda.synchronize()
    t_batch = (time.perf_counter() - t1) / steps
    for sv, st, e in zip(solvers, seq_states, Es):   # warm the one-by-one path's first step
        sv.step(st[0], st[1], st[2], e, dt, cg_rtol=1e-10, cg_max_it=20000, raise_on_maxit=False)
    torch.cuda.synchronize()
    first_mixed = [(st[0].clone(), st[1].clone()) for st in seq_states]   # one precision-form step from init
    t2 = time.perf_counter()
    for _ in range(steps):
        for sv, st, e in zip(solvers, seq_states, Es):
            sv.step(st[0], st[1], st[2], e, dt, cg_rtol=1e-10, cg_max_it=20000, raise_on_maxit=False)
    torch.cuda.synchronize()
    t_seq = (time.perf_counter() - t2) / steps
    # the plain FP64 path of the same instances, one by one from the initial
    # state: a first step (compared with the precision form's first step) and
    # `steps` timed ones
    del seq_states
    for sv in solvers:
        sv.set_precision(pkg.PREC_FP64)
    worst_phi = worst_ci = 0.0
    for k, (sv, st, e) in enumerate(zip(solvers, init, Es)):
        sv.step(st[0], st[1], st[2], e, dt, cg_rtol=1e-10, cg_max_it=20000, raise_on_maxit=False)
        p32, c32 = first_mixed[k]
        worst_phi = max(worst_phi, float(torch.linalg.norm(p32 - st[0]).item() / torch.linalg.norm(st[0]).item()))
        worst_ci = max(worst_ci, float(torch.linalg.norm(c32 - st[1]).item() / torch.linalg.norm(st[1]).item()))
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    for _ in range(steps):
        for sv, st, e in zip(solvers, init, Es):
            sv.step(st[0], st[1], st[2], e, dt, cg_rtol=1e-10, cg_max_it=20000, raise_on_maxit=False)
    torch.cuda.synchronize()
    t_fp64 = (time.perf_counter() - t3) / steps
    tun = batch.tuning()
    batch.close()
    for sv in solvers:
        sv.close()
    return {"metric": "MCTDHF instance-steps/s, batched whole time steps (all instances per call)",
            "value": count / t_batch, "instances": count, "dofs": int(sum(m.N for m in meshes)),
            "ms_per_batched_step": t_batch * 1e3, "one_by_one": {"value": count / t_seq, "ms": t_seq * 1e3},
            "speedup_vs_one_by_one": t_seq / t_batch,
            "one_by_one_fp64_path": {"value": count / t_fp64, "ms": t_fp64 * 1e3},
            "speedup_vs_fp64_path": t_fp64 / t_batch,
            "accuracy_vs_fp64_path": {"orbitals_rel_l2_max": worst_phi, "ci_rel_l2_max": worst_ci,
                                      "note": "one step of every instance from the same initial state, precision "
                                              "form against the FP64 path; worst instance"},
            "tuning": {"streams": tun["streams"],
                       "candidates_ms": [[c, round(ms, 2)] for c, ms in tun["candidates"]], "tuning_s": tune_s},
            "mode": f"precision form, one Krylov step of dimension {krylov_m} per time step, dt = {dt}, "
                    "multigrid Poisson to rtol 1e-10; wall-clock timed (every call ends with the GPU work done)",
            "mesh_build_s": build_s}


def run_water(torch, pkg, inputs, args):
    """The water workload at full size (O + 2 H, [-50,50]^3, 32^3 coarse, 6 / 5
    levels, Q4; 8 orbitals, 5 alpha + 5 beta electrons, 3,136 determinants,
    64 Poisson columns; 800 nm 4-cycle sin^2 at 2e14 W/cm^2, dt = 0.01,
    m = 10, Krylov threshold per substep): the plain FP64 path and the
    precision form from the same seeded state over --warmup + --steps steps,
    CUDA-event timed over the last --steps, and the precision form's
    difference from the FP64 path after them."""
    import numpy as np
    name = "water_q4"
    w = inputs.WORKLOADS[name]
    t0 = time.perf_counter()
    mesh = pkg.Mesh(*inputs.mesh_args(name))
    build_s = time.perf_counter() - t0
    if args.poisson == "multigrid":
        pkg.mesh_set_option(mesh, pkg.OPT_POISSON_SOLVER, pkg.POISSON_MULTIGRID)
    X, ML, _ = mesh.tables()
    interior = np.arange(mesh.N) < mesh.n_interior
    n = w["n_orb"]
    phi0 = inputs.lowdin(inputs.molecular_orbitals(X, interior, w["nuclei"], n, phase_noise=0.0), ML)
    C0 = inputs.initial_ci(n, w["n_alpha"], w["n_beta"])
    pulse, dt = w["pulse"], w["dt"]

    def field(tt):
        return inputs.sin2_pulse(tt, pulse["intensity"], pulse["wavelength_nm"], pulse["cycles"], pulse["pol"])

    stream = torch.cuda.current_stream()
    ml = torch.from_numpy(ML).cuda()
    res = {}
    for fname, prec in (("fp64", pkg.PREC_FP64), ("mixed", pkg.PREC_MIXED)):
        solver = pkg.MCTDHF(mesh, n, w["n_alpha"], w["n_beta"], w["m"])
        solver.set_precision(prec)
        solver.set_krylov_tol(args.krylov_tol if args.krylov_tol > 0 else 1e-10)
        phi = torch.from_numpy(phi0.copy()).cuda()
        C = torch.from_numpy(C0.copy()).cuda()
        W = torch.zeros((mesh.N, n * n), dtype=torch.float64, device="cuda")
        t = 0.0
        for _ in range(args.warmup):
            solver.step(phi, C, W, field(t), dt, cg_rtol=1e-10, cg_max_it=20000)
            t += dt
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos = []
        a.record(stream)
        for _ in range(args.steps):
            infos.append(solver.step(phi, C, W, field(t), dt, cg_rtol=1e-10, cg_max_it=20000))
            t += dt
        b.record(stream)
        torch.cuda.synchronize()
        res[fname] = dict(ms=a.elapsed_time(b) / args.steps, infos=infos, phi=phi, C=C)
        solver.close()
    p64, p32 = res["fp64"]["phi"], res["mixed"]["phi"]
    nrm = lambda ph: (torch.conj(ph) * ph).real.mul(ml[:, None]).sum(dim=0).cpu().numpy()   # noqa: E731
    i64, i32 = res["fp64"]["infos"][-1], res["mixed"]["infos"][-1]
    entry = {}
    for fname in ("fp64", "mixed"):
        inf = res[fname]["infos"]
        entry[fname] = {"ms_per_step": res[fname]["ms"], "steps_per_s": 1000.0 / res[fname]["ms"],
                        "krylov_substeps_mean": float(np.mean([i["krylov_substeps"] for i in inf])),
                        "cg_iters_mean": float(np.mean([i["cg_iters"] for i in inf])),
                        "energy_last": inf[-1]["energy"]}
    return {"workload": "water-shaped O + 2 H (1.81 bohr, 104.5 deg), [-50,50]^3, 32^3 coarse, 6 levels at O and "
                        "5 at each H, Q4; 8 orbitals, 5a+5b (3136 determinants), 64 Poisson columns; 800 nm 4-cycle "
                        "sin^2 2e14 W/cm^2, dt=0.01, m=10, Krylov threshold 1e-10 per substep, Poisson CG with the "
                        + ("multigrid" if args.poisson == "multigrid" else "Jacobi") + " preconditioner",
            "n_masters": mesh.N, "n_cells": mesh.n_cells, "n_hanging": mesh.n_hanging, "mesh_build_s": build_s,
            "warmup": args.warmup, "steps": args.steps, "fp64_path": entry["fp64"], "precision_form": entry["mixed"],
            "speedup_vs_fp64_path": res["fp64"]["ms"] / res["mixed"]["ms"],
            "accuracy_vs_fp64_path": {
                "orbital_norms_max_rel": float(np.max(np.abs(nrm(p32) - nrm(p64)) / np.abs(nrm(p64)))),
                "energy_rel": abs(i32["energy"] - i64["energy"]) / abs(i64["energy"]),
                "orbitals_rel_l2": float(torch.linalg.norm(p32 - p64).item() / torch.linalg.norm(p64).item()),
                "ci_rel_l2": float(torch.linalg.norm(res["mixed"]["C"] - res["fp64"]["C"]).item()
                                   / torch.linalg.norm(res["fp64"]["C"]).item()),
                "dipole_max_abs_diff": float(np.max(np.abs(np.subtract(i32["dipole"], i64["dipole"])))),
                "steps_compared": args.warmup + args.steps}}


def run_diff(torch, pkg, inputs, mesh, phi_col, steps=6, every=3, krylov_tol=1e-10):
    """Differentiation form on the full mesh (one-electron limit: one orbital,
    no projector or mean field): the forward pass with checkpoints, the
    adjoint sweep that gives dJ/dE_k for every step, and the tangent map, each
    timed with CUDA events on the current stream over `steps` time steps of
    the workload's dt inside the pulse.  A full-size check: the dot-product
    identity <g, J v> = <J^T g, v> between tangent and adjoint."""
    import numpy as np
    from paper_2301_02387_gb300 import adjoint as adj
    w = inputs.WORKLOADS[WORKLOAD]
    pulse, dt, m = w["pulse"], w["dt"], w["m"]
    omega = 45.5634 / pulse["wavelength_nm"]
    tau = pulse["cycles"] * 2.0 * np.pi / omega
    t0 = 0.5 * tau
    E = np.array([inputs.sin2_pulse(t0 + k * dt, pulse["intensity"], pulse["wavelength_nm"], pulse["cycles"],
                                    (0.0, 0.0, 1.0))[2] for k in range(steps)])
    e_dir = (0.0, 0.0, 1.0)
    rng = np.random.default_rng(inputs.BASE_SEED + 21)
    g = rng.standard_normal(steps + 1)
    v = rng.standard_normal(steps)
    stream = torch.cuda.current_stream()
    out = {}
    for name, prec in (("fp64", pkg.PREC_FP64), ("mixed", pkg.PREC_MIXED)):
        adj.tdse_forward(mesh, phi_col, E[:1], dt, e_dir, m, krylov_tol, prec, ckpt_every=every)   # warm-up
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        a.record(stream)
        _, _, ckpt = adj.tdse_forward(mesh, phi_col, E, dt, e_dir, m, krylov_tol, prec, ckpt_every=every)
        b.record(stream)
        grad, _ = adj.tdse_vjp(mesh, ckpt, every, E, g, dt, e_dir, m, krylov_tol, prec)
        c.record(stream)
        torch.cuda.synchronize()
        t_f, t_b = a.elapsed_time(b) / steps, b.elapsed_time(c) / steps
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        _, dd = adj.tdse_jvp(mesh, phi_col, E, v, dt, e_dir, m, krylov_tol, prec)
        d1.record(stream)
        torch.cuda.synchronize()
        lhs, rhs = float(g @ dd), float(v @ grad)
        out[name] = {"forward_ms_per_step": t_f, "adjoint_ms_per_step": t_b,
                     "tangent_ms_per_step": d0.elapsed_time(d1) / steps,
                     "gradient_over_forward": (t_f + t_b) / t_f,
                     # central differences over 256 spline samples need 2 x 256 forward passes
                     "speedup_vs_central_differences_256": 512.0 * t_f / (t_f + t_b),
                     "dot_product_rel": abs(lhs - rhs) / max(abs(lhs), abs(rhs))}
    fp = out["fp64"]
    return {"metric": "time steps/s of the gradient dJ/dE_k (forward with checkpoints + adjoint sweep)",
            "value": 1000.0 / (fp["forward_ms_per_step"] + fp["adjoint_ms_per_step"]),
            "unit": "steps/s", "steps": steps, "ckpt_every": every, "krylov_m": m, "krylov_tol": krylov_tol,
            "fp64": out["fp64"], "mixed": out["mixed"],
            "projected_2000_step_gradient_s": 2000.0 * (fp["forward_ms_per_step"] + fp["adjoint_ms_per_step"])
            * 1e-3,
            "workload": "one-electron limit on the H2 mesh (H2+ electron, orbital 0 of the seeded set), "
                        "field of the 800 nm sin^2 pulse from its peak, dt=0.02, e = z"}


def run_precision_spectrum(torch, pkg, inputs, steps=300, name=WORKLOAD, box=8.0, levels=2, nc=4):
    """The precision form against the FP64 path over a longer window on a
    reduced mesh of the same molecule and elements (box [-box,box]^3, nc^3
    coarse, `levels` levels per nucleus): both forms step from the same state
    through the pulse from its peak; the <sum r_i> traces and the spectra
    |FFT(a)|^2 of the acceleration a (second differences, Hann window) are
    compared."""
    import numpy as np
    w = inputs.WORKLOADS[name]
    args = (-box, box, nc, w["p"], [(R, Z, levels) for (R, Z, _L) in w["nuclei"]], w["c"])
    mesh = pkg.Mesh(*args)
    X, ml, _ = mesh.tables()
    interior = np.arange(mesh.N) < mesh.n_interior
    n = w["n_orb"]
    phi0 = inputs.lowdin(inputs.molecular_orbitals(X, interior, w["nuclei"], n, phase_noise=0.0), ml)
    C0 = inputs.initial_ci(n, w["n_alpha"], w["n_beta"])
    pulse, dt = w["pulse"], w["dt"]
    omega = 45.5634 / pulse["wavelength_nm"]
    t0 = 0.5 * pulse["cycles"] * 2.0 * np.pi / omega
    traces, ms = {}, {}
    for name, prec in (("fp64", pkg.PREC_FP64), ("mixed", pkg.PREC_MIXED)):
        solver = pkg.MCTDHF(mesh, n, w["n_alpha"], w["n_beta"], w["m"])
        solver.set_precision(prec)
        solver.set_krylov_tol(1e-10)
        phi = torch.from_numpy(phi0.copy()).cuda()
        C = torch.from_numpy(C0.copy()).cuda()
        W = torch.zeros((mesh.N, n * n), dtype=torch.float64, device="cuda")
        d = []
        torch.cuda.synchronize()
        tt = time.perf_counter()
        for k in range(steps):
            E = inputs.sin2_pulse(t0 + k * dt, pulse["intensity"], pulse["wavelength_nm"], pulse["cycles"],
                                  pulse["pol"])
            d.append(solver.step(phi, C, W, E, dt, cg_rtol=1e-10, cg_max_it=20000)["dipole"][2])
        torch.cuda.synchronize()
        ms[name] = 1e3 * (time.perf_counter() - tt) / steps
        traces[name] = np.array(d)
        solver.close()
    d64, d32 = traces["fp64"], traces["mixed"]
    def spectrum(dd):
        a = (dd[2:] - 2.0 * dd[1:-1] + dd[:-2]) / (dt * dt)
        return np.abs(np.fft.rfft(a * np.hanning(len(a)))) ** 2
    S64, S32 = spectrum(d64), spectrum(d32)
    freq = 2.0 * np.pi * np.arange(len(S64)) / ((len(d64) - 2) * dt) / omega
    band = freq <= 30.0
    return {"workload": f"{name} molecule, Q4, [-{box:g},{box:g}]^3, {nc}^3 coarse, {levels} levels (N={mesh.N}); "
                        f"{n} orbitals, {w['n_alpha']}a+{w['n_beta']}b; {steps} steps of dt={dt} from the "
                        f"{pulse['wavelength_nm']:g} nm pulse's peak; FP64 path vs precision form from the same state",
            "dipole_z_max_abs_diff": float(np.max(np.abs(d32 - d64))),
            "dipole_z_rel": float(np.max(np.abs(d32 - d64)) / np.max(np.abs(d64))),
            "spectrum_rel_l2_to_30_harmonics": float(np.linalg.norm(S32[band] - S64[band]) / np.linalg.norm(S64[band])),
            "spectrum": "|FFT(a)|^2, a = second differences of <sum z_i>, Hann window",
            "ms_per_step": ms}


def run_krylov_rules(torch, pkg, mesh, state0, field, dt, args, ref_state, n_orb, n_alpha, n_beta):
    """The precision form over the headline's warm-up and timed steps with
    other Krylov rules: fixed dimension 12 and 15 with the substep ladder, and
    Sec. 3.2's rule (fixed Krylov steps, dimension up to 16 grown until the
    estimate meets the threshold; the step count is 1.25 x the ladder's at
    dimension 15).  Per rule: ms per step, substeps, G applications per step
    and the orbitals' difference from the headline run."""
    import math as _m
    out = {}
    stream = torch.cuda.current_stream()
    sub15 = None
    for name, mk, adaptive in (("ladder_m12", 12, 0), ("ladder_m15", 15, 0), ("sec32_adaptive_m16", 16, -1)):
        solver = pkg.MCTDHF(mesh, n_orb, n_alpha, n_beta, mk)
        solver.set_precision(pkg.PREC_MIXED)
        solver.set_krylov_tol(args.krylov_tol if args.krylov_tol > 0 else 1e-10)
        steps_sec32 = 0
        if adaptive < 0:
            steps_sec32 = int(_m.ceil(1.25 * (sub15 or 1)))
            solver.set_krylov_adaptive(steps_sec32)
        phi, C, W = (x.clone() for x in state0)
        t = 0.0
        for _ in range(args.warmup):
            solver.step(phi, C, W, field(t), dt, cg_rtol=1e-10, cg_max_it=20000)
            t += dt
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos = []
        a.record(stream)
        for _ in range(args.steps):
            infos.append(solver.step(phi, C, W, field(t), dt, cg_rtol=1e-10, cg_max_it=20000))
            t += dt
        b.record(stream)
        torch.cuda.synchronize()
        sub = sum(i["krylov_substeps"] for i in infos) / len(infos)
        if name == "ladder_m15":
            sub15 = sub
        out[name] = {"krylov_m": mk, "ms_per_step": a.elapsed_time(b) / args.steps,
                     "substeps_per_step": sub,
                     "g_applications_per_step": sum(i["krylov_dim_sum"] for i in infos) / len(infos),
                     "largest_dimension": max(i["krylov_m_used"] for i in infos),
                     "unmet_steps": sum(i["krylov_unmet"] for i in infos),
                     "orbitals_rel_diff_vs_headline": float(torch.linalg.norm(phi - ref_state[0]).item()
                                                            / torch.linalg.norm(ref_state[0]).item())}
        if steps_sec32:
            out[name]["krylov_steps_per_time_step"] = steps_sec32
        solver.close()
    return out


def run_poisson_solvers(torch, pkg, mesh, phi, W_warm, restore, reps=3):
    """The Poisson batch of the live state (the workload's orbitals) alone,
    with the Jacobi and the multigrid preconditioner, in both forms: CUDA-event
    time per solve from the previous step's mean fields (the step's warm start)
    and from zero, and the iterations (float32 inner ones in the precision
    form)."""
    import numpy as np
    stream = torch.cuda.current_stream()
    out = {}
    for sname, sval in (("jacobi", pkg.POISSON_JACOBI), ("multigrid", pkg.POISSON_MULTIGRID)):
        pkg.mesh_set_option(mesh, pkg.OPT_POISSON_SOLVER, sval)
        for fname, prec in (("fp64", pkg.PREC_FP64), ("mixed", pkg.PREC_MIXED)):
            ent = {}
            for start in ("warm", "cold"):
                W = W_warm.clone()
                pkg.poisson_batch(mesh, phi, W, rtol=1e-10, max_it=20000, warm_start=start == "warm",
                                  precision=prec)   # first solve builds the hierarchy
                ts, its = [], []
                for _ in range(reps):
                    W.copy_(W_warm)
                    torch.cuda.synchronize()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    it, rel, rc = pkg.poisson_batch(mesh, phi, W, rtol=1e-10, max_it=20000,
                                                    warm_start=start == "warm", precision=prec)
                    b.record(stream)
                    torch.cuda.synchronize()
                    ts.append(a.elapsed_time(b))
                    its.append(it)
                ent[start] = {"ms": float(np.median(ts)), "iterations": int(np.median(its)),
                              "max_relres": float(np.max(rel))}
            out.setdefault(sname, {})[fname] = ent
    pkg.mesh_set_option(mesh, pkg.OPT_POISSON_SOLVER, restore)
    out["workload"] = ("the workload's 16 pair mean fields of its orbitals after the timed steps, rtol 1e-10; "
                       "warm: from the previous step's fields")
    return out


# Kernel classes of the library's event timing: name, bound, unit of work.
PROF_CLASSES = {
    0: ("Gram-Schmidt passes (krylov_update / project*_dots, FP64)", "alu", "flops"),
    1: ("complex64 G cell pass (gcell32b_kernel on frozen per-cell blocks; cell32v_kernel_q4<true,L4,false> when gathered)", "hbm", "bytes"),
    2: ("float32 stiffness of the CG sweeps with the p.Ap epilogue (cell32v_kernel_q4<false,L4,true>)", "hbm", "bytes"),
    3: ("float32 CG vector kernels (update_beta4 / p_update4; p.Ap in the stiffness pass)", "hbm", "bytes"),
    4: ("FP64 cell passes (g_cell_kernel / cell_op_kernel)", "alu", "flops"),
}
# DRAM bytes per bracketed call from one ncu capture of the same kernels
# (dram__bytes_read.sum + dram__bytes_write.sum, summed over a class's launches
# of one Krylov substep / CG iteration and divided by the calls); class 0 is
# captured on the reduced 16^3-coarse mesh of the molecule (N = 508,385) and
# scaled by N to the benchmark mesh (every term is a whole-vector pass); class 1
# is the G cell pass on frozen per-cell blocks (gcell32b_kernel, one launch on
# the benchmark mesh itself); None where no capture of the current kernel exists.
TRAFFIC_PER_CALL = {0: 343.9e6, 1: 300.0e6, 2: 114.9e6, 3: 341.8e6, 4: None}


def _class_rooflines(prof, total_ms, fp64_peak, hbm, peak_src):
    """Per kernel class: event time, share of the timed steps, achieved
    work rate against its roofline; the dominant class (largest time) is the
    headline entry."""
    classes = []
    for c, (ms, calls, work) in sorted(prof.items()):
        name, bound, wunit = PROF_CLASSES[c]
        if calls == 0 or ms <= 0.0:
            continue
        rate = work / (ms * 1e-3)
        if bound == "alu":
            achieved, peak, unit = rate / 1e12, fp64_peak, "TFLOP/s"
            src = "measured in this run: FP64 multiply-add throughput (afem_fma_peak, 4 x 256 threads per SM)"
        else:
            achieved, peak, unit = rate / 1e9, hbm, "GB/s"
            src = peak_src
        classes.append({"class": c, "kernel": name, "bound": bound, "achieved": achieved, "peak": peak,
                        "unit": unit, "frac": achieved / peak, "peak_source": src, "calls": calls,
                        "ms_total": ms, "share_of_step": ms / total_ms, "work_per_call": work / calls,
                        "work_unit": wunit, "traffic": TRAFFIC_PER_CALL.get(c)})
    if not classes:
        return {"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
                "classes": []}
    top = max(classes, key=lambda e: e["ms_total"])
    out = {k: top[k] for k in ("kernel", "bound", "achieved", "peak", "unit", "frac", "peak_source",
                               "share_of_step", "traffic")}
    out["classes"] = classes
    return out


def run_ours(args, rank, world, dist):
    import numpy as np
    import torch
    import paper_2301_02387_gb300 as pkg
    from paper_2301_02387_gb300 import inputs

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    w = inputs.WORKLOADS[WORKLOAD]
    mesh, solver, phi0, C0 = setup_state(pkg, inputs, torch, w)
    if args.poisson == "multigrid":
        pkg.mesh_set_option(mesh, pkg.OPT_POISSON_SOLVER, pkg.POISSON_MULTIGRID)
    n, N = w["n_orb"], mesh.N
    X, ML, _ = mesh.tables()
    state0 = (torch.from_numpy(phi0).cuda(), torch.from_numpy(C0).cuda(),
              torch.zeros((N, n * n), dtype=torch.float64, device="cuda"))
    pulse = w["pulse"]
    dt = w["dt"]
    stream = torch.cuda.current_stream()

    def field(tt):
        return inputs.sin2_pulse(tt, pulse["intensity"], pulse["wavelength_nm"], pulse["cycles"], pulse["pol"])

    # the plain FP64 path, then the precision form from the same initial state
    fp64 = fp64_prof = None
    if args.form == "both":
        fp64 = _timed_form(pkg, torch, solver, state0, pkg.PREC_FP64, args, field, dt, dist, stream)
    sampler = ClockSampler(dev)
    sampler.start()
    mixed = _timed_form(pkg, torch, solver, state0, pkg.PREC_MIXED, args, field, dt, dist, stream)
    clocks = sampler.stop()
    value = job_rate(world, mixed["ms"])
    # kernel-class event timing over K further steps continuing each form's
    # timed run (the events cost a few percent, so the headline runs without)
    mixed_prof = _timed_form(pkg, torch, solver, mixed["state"], pkg.PREC_MIXED, args, field, dt, dist, stream,
                             profile=True, t0=mixed["t"], warmup=0)
    if fp64 is not None:
        fp64_prof = _timed_form(pkg, torch, solver, fp64["state"], pkg.PREC_FP64, args, field, dt, dist, stream,
                                profile=True, t0=fp64["t"], warmup=0)
    # the same K steps with the G cell pass gathering its mean-field rows in the
    # pass instead of staging frozen per-cell blocks by bulk copies
    gcell_staging = None
    if not args.no_rules:
        def _gcell(run):
            ms_c, calls_c, _w = run["prof"][pkg.PROF_GCELL32]
            return {"ms_per_step": run["ms"], "gcell_us_per_call": 1e3 * ms_c / max(calls_c, 1),
                    "gcell_calls": calls_c}
        gcell_staging = {"blocks_bulk_copy": _gcell(mixed_prof),
                         "note": "precision form, the K steps after the timed ones, kernel-class event timing on; "
                                 "pipelined includes forming v at the hanging points"}
        for label, mode in (("rows_gathered", 0), ("blocks_pipelined", 2)):
            pkg.mesh_set_option(mesh, pkg.OPT_GCELL_BLOCKS, mode)
            try:
                run = _timed_form(pkg, torch, solver, mixed["state"], pkg.PREC_MIXED, args, field, dt, dist,
                                  stream, profile=True, t0=mixed["t"], warmup=0)
            finally:
                pkg.mesh_set_option(mesh, pkg.OPT_GCELL_BLOCKS, 1)
            gcell_staging[label] = _gcell(run)

    # accuracy of the precision form against the FP64 path after warmup + K steps
    ml = torch.from_numpy(ML).cuda()
    def norms(phi):
        return (torch.conj(phi) * phi).real.mul(ml[:, None]).sum(dim=0).cpu().numpy()
    acc = None
    if fp64 is not None:
        p64, c64, _ = fp64["state"]
        p32, c32, _ = mixed["state"]
        acc = {
            "orbital_norms_max_rel": float(np.max(np.abs(norms(p32) - norms(p64)) / np.abs(norms(p64)))),
            "energy_rel": abs(mixed["infos"][-1]["energy"] - fp64["infos"][-1]["energy"])
            / abs(fp64["infos"][-1]["energy"]),
            "orbitals_rel_l2": float(torch.linalg.norm(p32 - p64).item() / torch.linalg.norm(p64).item()),
            "ci_rel_l2": float(torch.linalg.norm(c32 - c64).item() / torch.linalg.norm(c64).item()),
            "dipole_rel": float(np.max(np.abs(np.subtract(mixed["infos"][-1]["dipole"], fp64["infos"][-1]["dipole"])))
                                / np.max(np.abs(fp64["infos"][-1]["dipole"]))),
            "steps_compared": args.warmup + args.steps,
        }

    # ---- end to end through the public API: the state lives in pinned host
    # buffers and is copied in and out every step inside the timed region;
    # the same warm-up and timed steps as the device-timed precision form
    solver.set_precision(pkg.PREC_MIXED)
    solver.set_krylov_tol(args.krylov_tol)
    phi_h, C_h, W_h = (x.cpu().pin_memory() for x in state0)
    t = 0.0

    def host_step(tt):
        phi_d = phi_h.to("cuda", non_blocking=True)
        C_d = C_h.to("cuda", non_blocking=True)
        W_d = W_h.to("cuda", non_blocking=True)
        solver.step(phi_d, C_d, W_d, field(tt), dt, cg_rtol=1e-10, cg_max_it=20000)
        phi_h.copy_(phi_d, non_blocking=True)
        C_h.copy_(C_d, non_blocking=True)
        W_h.copy_(W_d, non_blocking=True)
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        host_step(t)
        t += dt
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_e2e = time.perf_counter()
    for _ in range(args.steps):
        host_step(t)
        t += dt
    e2e_s = max_over_ranks(dist, torch, (time.perf_counter() - t_e2e) / args.steps, "cuda")
    bytes_state = phi_h.numel() * 16 + C_h.numel() * 16 + W_h.numel() * 8
    phi, W = mixed["state"][0], mixed["state"][2]
    t = mixed["t"]

    kern = measure_kernels(pkg, torch, mesh, W, phi, field(t), stream)
    integrals = measure_integrals(pkg, torch, mesh, phi, W, stream)
    psolv = None if args.no_poisson_solvers else run_poisson_solvers(
        torch, pkg, mesh, phi, W, pkg.POISSON_MULTIGRID if args.poisson == "multigrid" else pkg.POISSON_JACOBI)
    rules = None
    if not args.no_rules:
        rules = run_krylov_rules(torch, pkg, mesh, state0, field, dt, args, mixed["state"], n, w["n_alpha"],
                                 w["n_beta"])
        rules["headline_ladder_m10"] = {"krylov_m": w["m"], "ms_per_step": mixed["ms"],
                                        "substeps_per_step": float(np.mean([i["krylov_substeps"]
                                                                            for i in mixed["infos"]])),
                                        "g_applications_per_step": float(np.mean([i["krylov_dim_sum"]
                                                                                  for i in mixed["infos"]]))}
    batching = None if args.no_batch else run_batch(torch, pkg, inputs)
    batch_steps = None if args.no_batch else run_batch_steps(torch, pkg, inputs)
    spec = None if args.no_spectrum else run_precision_spectrum(torch, pkg, inputs)
    diff = None if args.no_diff else run_diff(torch, pkg, inputs, mesh, state0[0][:, 0].contiguous(),
                                              krylov_tol=args.krylov_tol if args.krylov_tol > 0 else 1e-10)
    peaks, peak_src = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    # FP64 and FP32 multiply-add peaks measured in this run on this GPU
    # (afem_fma_peak); the FP64-bound classes are reported against the FP64 one
    fp64_peak = pkg.fma_peak(pkg.PEAK_FP64, 200.0) / 1e12
    fp32_peak = pkg.fma_peak(pkg.PEAK_FP32, 200.0) / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp64_derived = sms * 4 * sm_mhz * 1e6 / 1e12
    roofline = _class_rooflines(mixed_prof["prof"], mixed_prof["ms"] * args.steps, fp64_peak, hbm, peak_src)
    roofline["measured_over"] = (f"{args.steps} precision-form steps continuing the timed ones, "
                                 f"{mixed_prof['ms']:.1f} ms/step with the event timing on")
    roofline["arith_peaks"] = {"fp64_tflops": fp64_peak, "fp32_tflops": fp32_peak,
                               "fp64_derived_tflops": fp64_derived,
                               "derived_from": f"{sms} SMs x 2 FP64 FMA/clk x 2 flop x median SM clock "
                                               f"{sm_mhz:.0f} MHz under load"}
    roofline["kernels_alone"] = {
        "stiffness_fp32": {"bound": "hbm", "achieved": kern["stiff32_gbs"], "peak": hbm, "unit": "GB/s",
                           "frac": kern["stiff32_gbs"] / hbm, "work": "8 B per DoF*RHS (read x, write y)"},
        "stiffness_fp64": {"bound": "alu", "achieved": kern["stiff_tflops"], "peak": fp64_peak, "unit": "TFLOP/s",
                           "frac": kern["stiff_tflops"] / fp64_peak, "work": "3(p+1)2+6 flops per node*RHS"}}
    if fp64 is not None:
        roofline["fp64_path_classes"] = _class_rooflines(fp64_prof["prof"], fp64_prof["ms"] * args.steps,
                                                         fp64_peak, hbm, peak_src)["classes"]
    mi = mixed["infos"]
    fp64_entry = None
    if fp64 is not None:
        fp64_entry = {"value": job_rate(world, fp64["ms"]), "unit": UNIT, "ms_per_step": fp64["ms"],
                      "cg_iters_mean": float(np.mean([i["cg_iters"] for i in fp64["infos"]])),
                      "krylov_substeps_mean": float(np.mean([i["krylov_substeps"] for i in fp64["infos"]])),
                      "gpu_launches": fp64["launches"]}
    return {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": mixed["ms"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 cell operators + f64 refinement/Gram-Schmidt/CI",
        "data": "synthetic (seeded Gaussian orbitals on the nuclei, random-phase CI vector)",
        "config": {"workload": "H2 R=1.4 bohr, [-40,40]^3, 20^3 coarse, 5 levels/nucleus, Q4, "
                               "4 orbitals (1a+1b), 800nm 3-cycle sin^2 1e14 W/cm^2, dt=0.02, m=10, rtol=1e-10, "
                               f"Krylov error threshold {args.krylov_tol:g} per substep, Poisson CG with the "
                               f"{args.poisson} preconditioner",
                   "n_masters": mesh.N, "n_cells": mesh.n_cells, "n_hanging": mesh.n_hanging,
                   "cache": "working set (Krylov basis, CG batch) larger than L2; no flush",
                   "parallelism": f"replicas x{world}"},
        "fp64_path": fp64_entry,
        "speedup_vs_fp64_path": (fp64["ms"] / mixed["ms"]) if fp64 is not None else None,
        "accuracy_vs_fp64_path": acc,
        "precision_spectrum": spec,
        "orbital_dof_applies_per_s": {"fp64": kern["h1_orbital_dof_per_s"],
                                      "fp32_in_G": kern["g32_orbital_dof_per_s"]},
        "step_detail": {"inner_cg_iters_mean": float(np.mean([i["cg_iters"] for i in mi])),
                        "krylov_m_used": mi[-1]["krylov_m_used"],
                        "krylov_substeps_mean": float(np.mean([i["krylov_substeps"] for i in mi])),
                        "krylov_tol": args.krylov_tol,
                        "arnoldi_err_max": float(max(i["arnoldi_err"] for i in mi)),
                        "energy_last": mi[-1]["energy"]},
        "roofline": roofline,
        "clocks": clocks,
        "e2e": {"value": world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": bytes_state,
                "d2h_bytes_per_step": bytes_state},
        "gpu_launches": mixed["launches"],
        "batching_form": batching,
        "batching_form_steps": batch_steps,
        "differentiation_form": diff,
        "krylov_rules": rules,
        "gcell_staging": gcell_staging,
        "tensor_core_integrals": integrals,
        "poisson_solvers": psolv,
        # the oracle solves by Jacobi-PCG: its iteration count is the FP64
        # Jacobi count (the timed steps', or the Jacobi solve of poisson_solvers)
        "_fp64_cg_iters": (fp64_entry["cg_iters_mean"] if fp64_entry and args.poisson == "jacobi"
                           else psolv["jacobi"]["fp64"]["warm"]["iterations"] if psolv else None),
        "_fp64_substeps": (float(np.mean([i["krylov_substeps"] for i in fp64["infos"]]))
                           if fp64 is not None else None),
    }


# ----------------------------------------------------------------- oracle arm
# Mean Jacobi-PCG iterations per step of the warm-started FP64 Poisson batch on
# this workload (the FP64 path's count, measured on GB300); the oracle's
# reference arm runs without a GPU and scales its per-iteration time by it.
FP64_CG_ITERS_PER_STEP = 710

_ORACLE_SAMPLE = r"""
import json, os, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
import scipy.sparse.linalg as sla
from oracle import fem, krylov, mctdhf, mesh, poisson
from paper_2301_02387_gb300 import inputs
name = %(name)r
w = inputs.WORKLOADS[name]
tb = time.perf_counter()
m = mesh.Mesh(*inputs.mesh_args(name))
op = fem.Operators(m)
tb = time.perf_counter() - tb
n = w["n_orb"]
phi = inputs.lowdin(inputs.molecular_orbitals(m.Xm, ~m.boundary, w["nuclei"], n, phase_noise=0.0), op.ML)
C = inputs.initial_ci(n, w["n_alpha"], w["n_beta"])
pl = w["pulse"]
E = inputs.sin2_pulse(%(t0)r, pl["intensity"], pl["wavelength_nm"], pl["cycles"], pl["pol"])
sim = mctdhf.MCTDHF(op, n, w["n_alpha"], w["n_beta"], poisson_method="cg", poisson_rtol=1e-10)
ps = sim.ps
# (1) the step outside its iterations: pair densities, right-hand sides and
# multipole surface data, integrals, RDMs, the CI exponential, U fields
t0 = time.perf_counter()
rho, pairs = poisson.pair_densities(op, phi)
b, g = ps.rhs_and_bc(rho)
rhs = b[ps.I] - ps.A_IB @ g
Wc = np.zeros((m.N, rho.shape[1]))
Wc[ps.B] = g
W = poisson.assemble_pair_potentials(Wc, pairs, n)
h, eri = sim.integrals(phi, W, E)
Hci = sim.ci.hamiltonian(h, eri)
g1, g2 = sim.ci.rdm1(C), sim.ci.rdm2(C)
ev, V = np.linalg.eigh(0.5 * (Hci + Hci.conj().T))
C1 = V @ (np.exp(-1j * w["dt"] * ev) * (V.conj().T @ C))
U = sim.mean_field_operator(g1, g2, W)
t_block = time.perf_counter() - t0
# (2) one Krylov substep: the Arnoldi basis of dimension m (m applications of
# G, modified Gram-Schmidt) and the substep decision; its length gives the
# oracle's own substep count per step
t0 = time.perf_counter()
_, _, _, info = krylov.arnoldi_propagate(lambda v: sim.G_apply(v, phi, U, E), phi, sim.inner, w["m"], w["dt"],
                                         %(tol)r, return_info=True, stop_after=1)
t_sub = time.perf_counter() - t0
tau1 = info["taus"][0]
# (3) Jacobi-PCG iterations on one column of the batch
d = ps.A_II.diagonal()
Minv = sla.LinearOperator(ps.A_II.shape, matvec=lambda v: v / d)
k_it = 5
t0 = time.perf_counter()
sla.cg(ps.A_II, rhs[:, 0], rtol=1e-300, atol=0.0, M=Minv, maxiter=k_it)
t_it = (time.perf_counter() - t0) / k_it
maps = open("/proc/self/maps").read() if os.path.exists("/proc/self/maps") else ""
assert "libafem" not in maps, "the oracle sample must not load the CUDA library"
print(json.dumps({"N": int(m.N), "build_s": tb, "t_block": t_block, "t_sub": t_sub, "tau1": tau1,
                  "t_cg_it_col": t_it, "cols": int(rho.shape[1]), "dt": w["dt"]}))
"""


def oracle_sample(krylov_tol=1e-10, t0=None):
    """Time the FP64 oracle (as it stands) on the benchmark mesh itself in a
    fresh process with one BLAS thread: the step's non-iterative block, one
    Krylov substep (with the oracle's own substep decision) and Jacobi-PCG
    iterations on one column.  Returns the per-unit times."""
    import math as _m
    from paper_2301_02387_gb300 import inputs
    w = inputs.WORKLOADS[WORKLOAD]
    if t0 is None:   # the pulse's peak
        t0 = 0.5 * w["pulse"]["cycles"] * 2.0 * _m.pi / (45.5634 / w["pulse"]["wavelength_nm"])
    code = _ORACLE_SAMPLE % {"root": ROOT, "name": WORKLOAD, "t0": float(t0), "tol": float(krylov_tol)}
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    t = time.perf_counter()
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    out["wall_s"] = time.perf_counter() - t
    return out


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline_entry(cg_iters=None, substeps=None, krylov_tol=1e-10):
    """The oracle's step time on the benchmark mesh from a bounded sample:
    t_step = t_block + S t_substep + cols I t_iteration, with S the substeps
    per step (given, else the oracle's own dt / tau_1) and I the Jacobi-PCG
    iterations per column and step (given, else FP64_CG_ITERS_PER_STEP)."""
    s = oracle_sample(krylov_tol)
    S_oracle = s["dt"] / s["tau1"]
    S = substeps if substeps else S_oracle
    I = cg_iters if cg_iters else FP64_CG_ITERS_PER_STEP
    t_step = s["t_block"] + S * s["t_sub"] + s["cols"] * I * s["t_cg_it_col"]
    K = _host_cores()
    return {"value": 1.0 / t_step, "unit": UNIT, "cores": 1, "host_cores": K, "kind": "oracle",
            "sample": (f"FP64 oracle (assembled SciPy CSR, one BLAS thread: 1 of {K} host cores) on the benchmark "
                       f"mesh itself (N={s['N']}; built in {s['build_s']:.0f} s, not timed), field of the pulse at "
                       f"its peak: the step's non-iterative block (pair densities, right-hand sides, multipole "
                       f"data, integrals, RDMs, CI exponential, U fields) {s['t_block']:.1f} s, one Krylov substep "
                       f"of dimension 10 with its decision {s['t_sub']:.1f} s (tau_1 = {s['tau1']:.3g}, so "
                       f"{S_oracle:.0f} substeps per step by the oracle's own controller), one Jacobi-PCG iteration "
                       f"of one column {s['t_cg_it_col'] * 1e3:.0f} ms; step = block + {S:.0f} substeps + "
                       f"{s['cols']} columns x {I:.0f} Jacobi-PCG iterations ({'this run' if cg_iters else 'FP64 path mean'}) "
                       f"= {t_step:.0f} s; sample wall time {s['wall_s']:.0f} s"),
            "t_step_s": t_step, "substeps_oracle": S_oracle, "substeps_used": S, "cg_iters_used": I}


def run_reference(args):
    # The oracle alone: the mesh size comes from the oracle's own mesh; no
    # GPU and none of the library is used.
    cb = cpu_baseline_entry(krylov_tol=args.krylov_tol if args.krylov_tol > 0 else 1e-10)
    v = cb["value"]
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "H2 Q4, as the GPU arm (the benchmark mesh itself)"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _event_time(torch, stream, fn, flush, reps):
    """Mean CUDA-event duration (s) of fn() on `stream`, L2 flushed before each launch."""
    ts = []
    for r in range(reps + 2):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        if r >= 2:
            ts.append(a.elapsed_time(b) * 1e-3)
    return sum(ts) / len(ts)


def measure_kernels(pkg, torch, mesh, W, phi, E, stream, reps=10):
    """Operator kernels timed alone on the live state: the stiffness of the
    Poisson batch (16 real columns) in FP64 and FP32, the H1 operator on the
    orbitals in complex128 and complex64."""
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    nrhs = W.shape[1]
    p1 = mesh.degree + 1
    flops = mesh.n_cells * p1 ** 3 * nrhs * (3 * p1 * 2 + 6)   # 3 line contractions + combine per node/column
    out = {}
    y = torch.empty_like(W)
    t = _event_time(torch, stream, lambda: pkg.op_apply(mesh, pkg.OP_STIFF, W, y), flush, reps)
    out["stiff_tflops"] = flops / t / 1e12
    out["stiff_gbs"] = mesh.N * nrhs * 16 / t / 1e9
    W32 = W.float().contiguous()
    y32 = torch.empty_like(W32)
    t = _event_time(torch, stream, lambda: pkg.op_apply(mesh, pkg.OP_STIFF_F32, W32, y32), flush, reps)
    out["stiff32_s"] = t
    out["stiff32_gbs"] = mesh.N * nrhs * 8 / t / 1e9          # algorithmic bytes: read x, write y (float32)
    out["stiff32_tflops"] = flops / t / 1e12
    yp = torch.empty_like(phi)
    t = _event_time(torch, stream, lambda: pkg.op_apply(mesh, pkg.OP_H1, phi, yp, E=E), flush, reps)
    out["h1_orbital_dof_per_s"] = mesh.N * phi.shape[1] / t
    p64 = phi.to(torch.complex64).contiguous()
    y64 = torch.empty_like(p64)
    t = _event_time(torch, stream, lambda: pkg.op_apply(mesh, pkg.OP_H1_C64, p64, y64, E=E), flush, reps)
    out["g32_orbital_dof_per_s"] = mesh.N * phi.shape[1] / t
    return out


def run_kernels_only(reps=3):
    """The benchmark mesh and a mean-field-shaped batch; each operator kernel runs `reps` times."""
    import numpy as np
    import torch
    import paper_2301_02387_gb300 as pkg
    from paper_2301_02387_gb300 import inputs
    torch.cuda.set_device(0)
    w = inputs.WORKLOADS[WORKLOAD]
    mesh, solver, phi0, C0 = setup_state(pkg, inputs, torch, w)
    n = w["n_orb"]
    phi = torch.from_numpy(phi0).cuda()
    # smooth mean-field-shaped columns (no solver launches before the profiled kernels)
    X, _, _ = mesh.tables()
    r = np.sqrt(np.sum(X ** 2, axis=1))
    cols = [1.0 / np.sqrt(r * r + 0.3 * (c + 1)) for c in range(n * n)]
    W = torch.from_numpy(np.ascontiguousarray(np.stack(cols, axis=1))).cuda()
    W32 = W.float().contiguous()
    y, y32 = torch.empty_like(W), torch.empty_like(W32)
    p64 = phi.to(torch.complex64).contiguous()
    yp, yp64 = torch.empty_like(phi), torch.empty_like(p64)
    E = (0.0, 0.0, 0.01)
    for _ in range(reps):
        pkg.op_apply(mesh, pkg.OP_STIFF, W, y)
        pkg.op_apply(mesh, pkg.OP_STIFF_F32, W32, y32)
        pkg.op_apply(mesh, pkg.OP_H1, phi, yp, E=E)
        pkg.op_apply(mesh, pkg.OP_H1_C64, p64, yp64, E=E)
    torch.cuda.synchronize()
    print("kernels-only done", mesh.N, float(np.abs(y32.cpu().numpy()).max()))


def run_profile_step(inner_iters=48):
    """One precision-form MCTDHF step of the workload (multigrid Poisson, inner
    CG capped at `inner_iters` iterations) with one Krylov step: every kernel of a
    step appears, in a launch count small enough for a profiler's launch list."""
    import torch
    import paper_2301_02387_gb300 as pkg
    from paper_2301_02387_gb300 import inputs
    torch.cuda.set_device(0)
    w = inputs.WORKLOADS[WORKLOAD]
    mesh, solver, phi0, C0 = setup_state(pkg, inputs, torch, w)
    pkg.mesh_set_option(mesh, pkg.OPT_POISSON_SOLVER, pkg.POISSON_MULTIGRID)
    n = w["n_orb"]
    phi = torch.from_numpy(phi0).cuda()
    C = torch.from_numpy(C0).cuda()
    W = torch.zeros((mesh.N, n * n), dtype=torch.float64, device="cuda")
    solver.set_precision(pkg.PREC_MIXED)
    solver.set_krylov_tol(0.0)
    pulse = w["pulse"]
    E = inputs.sin2_pulse(1.0, pulse["intensity"], pulse["wavelength_nm"], pulse["cycles"], pulse["pol"])
    info = solver.step(phi, C, W, E, w["dt"], cg_rtol=1e-10, cg_max_it=inner_iters, raise_on_maxit=False)
    torch.cuda.synchronize()
    print("profile-step done", info)


def run_profile_gs(nc=16, dt=1e-4):
    """The precision form's Krylov propagation on a reduced coarse grid of the
    benchmark molecule (nc^3 coarse cells, 5 levels per nucleus, Q4, 4
    orbitals: each basis vector ~20 MB, 10 of them well above L2), a few
    substeps: the small case on which the Gram-Schmidt kernels' DRAM traffic
    is captured and then scaled to the benchmark mesh by N."""
    import numpy as np
    import torch
    import paper_2301_02387_gb300 as pkg
    from paper_2301_02387_gb300 import inputs
    torch.cuda.set_device(0)
    w = inputs.WORKLOADS[WORKLOAD]
    mesh = pkg.Mesh(w["lo"], w["hi"], nc, w["p"], w["nuclei"], w["c"])
    X, ml, _ = mesh.tables()
    n = w["n_orb"]
    interior = np.arange(mesh.N) < mesh.n_interior
    phi = torch.from_numpy(inputs.lowdin(inputs.molecular_orbitals(X, interior, w["nuclei"], n, phase_noise=0.0),
                                         ml)).cuda()
    r = np.sqrt(np.sum(X ** 2, axis=1))
    U = np.zeros((mesh.N, n, n), dtype=np.complex128)
    for q in range(n):
        U[:, q, q] = 1.0 / np.sqrt(r * r + 0.3 * (q + 1))
    Ud = torch.from_numpy(U.reshape(mesh.N, n * n)).cuda()
    _, err, sub = pkg.arnoldi_propagate(mesh, phi, Ud, w["m"], dt, 1e-10, E=(0.0, 0.0, 0.01),
                                        precision=pkg.PREC_MIXED)
    torch.cuda.synchronize()
    print(json.dumps({"profile_gs": {"N": mesh.N, "n_orb": n, "substeps": sub, "err": err}}))


def measure_integrals(pkg, torch, mesh, phi, W, stream, reps=5):
    """The two-electron integrals (pq|rs) of the live orbitals and mean fields:
    the FP64 contraction against the tensor-core one (tcgen05 MMAs, TF32 hi/lo
    operands, FP64 sums of 32-point tiles), CUDA events on the launching stream
    around `reps` calls each (after one untimed call), and the largest entry
    difference relative to the largest FP64 entry."""
    n = int(phi.shape[1])
    nn = n * n
    out = {}
    res = {}
    for name, prec in (("fp64", pkg.PREC_FP64), ("tensor_cores", pkg.PREC_MIXED)):
        eri = torch.empty((nn, nn), dtype=torch.complex128, device="cuda")
        pkg.two_electron_integrals(mesh, phi, W, eri, precision=prec)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            pkg.two_electron_integrals(mesh, phi, W, eri, precision=prec)
        b.record(stream)
        torch.cuda.synchronize()
        out[name] = {"ms_per_call": a.elapsed_time(b) / reps}
        res[name] = eri
    npts = mesh.n_hanging + mesh.N
    # algorithmic work: 2 (n^2 complex = 2 n^2 real rows) x n^2 columns x support points
    flops = 2.0 * (2 * nn) * nn * npts
    for name in out:
        out[name]["tflops"] = flops / (out[name]["ms_per_call"] * 1e-3) / 1e12
    ref = res["fp64"]
    out["max_rel_diff"] = float((res["tensor_cores"] - ref).abs().max().item() / ref.abs().max().item())
    out["support_points"] = int(npts)
    out["n_orb"] = n
    return out


def run_profile_integrals(reps=5):
    """The workload's integrals alone (seeded orbitals, their Poisson mean
    fields): one untimed and `reps` timed calls of each form; small enough for a
    profiler capture of the tensor-core kernel."""
    import torch
    import paper_2301_02387_gb300 as pkg
    from paper_2301_02387_gb300 import inputs
    torch.cuda.set_device(0)
    w = inputs.WORKLOADS[WORKLOAD]
    mesh, solver, phi0, C0 = setup_state(pkg, inputs, torch, w)
    n = w["n_orb"]
    phi = torch.from_numpy(phi0).cuda()
    W = torch.zeros((mesh.N, n * n), dtype=torch.float64, device="cuda")
    pkg.mesh_set_option(mesh, pkg.OPT_POISSON_SOLVER, pkg.POISSON_MULTIGRID)
    pkg.poisson_batch(mesh, phi, W, rtol=1e-10, max_it=20000)
    torch.cuda.synchronize()
    out = measure_integrals(pkg, torch, mesh, phi, W, torch.cuda.current_stream(), reps=reps)
    print(json.dumps({"profile_integrals": out, "N": mesh.N}))


def run_profile_arnoldi(dt_short=2e-4, dt_timed=2e-3, timed=True):
    """The orbital propagator alone on the workload mesh (mean fields frozen to
    a smooth synthetic field): one short error-controlled propagation (a few
    substeps, small enough for a profiler's launch list), then a timed one per
    arithmetic form reporting ms per Krylov substep."""
    import numpy as np
    import torch
    import paper_2301_02387_gb300 as pkg
    from paper_2301_02387_gb300 import inputs
    torch.cuda.set_device(0)
    w = inputs.WORKLOADS[WORKLOAD]
    mesh, solver, phi0, C0 = setup_state(pkg, inputs, torch, w)
    n = w["n_orb"]
    phi = torch.from_numpy(phi0).cuda()
    X, _, _ = mesh.tables()
    r = np.sqrt(np.sum(X ** 2, axis=1))
    U = np.zeros((mesh.N, n, n), dtype=np.complex128)
    for p in range(n):
        U[:, p, p] = 1.0 / np.sqrt(r * r + 0.3 * (p + 1))
    U[:, 0, 1] = U[:, 1, 0] = 0.1 / np.sqrt(r * r + 1.0)
    Ud = torch.from_numpy(U.reshape(mesh.N, n * n)).cuda()
    E = (0.0, 0.0, 0.01)
    _, err, sub = pkg.arnoldi_propagate(mesh, phi, Ud, w["m"], dt_short, 1e-10, E=E, precision=pkg.PREC_MIXED)
    torch.cuda.synchronize()
    out = {"short": {"dt": dt_short, "substeps": sub, "err": err}}
    for name, prec in ((("fp64", pkg.PREC_FP64), ("mixed", pkg.PREC_MIXED)) if timed else ()):
        pkg.arnoldi_propagate(mesh, phi, Ud, w["m"], dt_short, 1e-10, E=E, precision=prec)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        _, err, sub = pkg.arnoldi_propagate(mesh, phi, Ud, w["m"], dt_timed, 1e-10, E=E, precision=prec)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        out[name] = {"dt": dt_timed, "substeps": sub, "ms": ms, "ms_per_substep": ms / max(sub, 1), "err": err}
    print(json.dumps({"profile_arnoldi": out, "N": mesh.N, "n_orb": n}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batching-form measurement (64 instances)")
    ap.add_argument("--batch-only", action="store_true",
                    help="only the batching-form measurement (its JSON sub-entry), for profiling")
    ap.add_argument("--no-diff", action="store_true", help="skip the differentiation-form measurement")
    ap.add_argument("--no-poisson-solvers", action="store_true",
                    help="skip the Poisson batch alone with the Jacobi and the multigrid preconditioner")
    ap.add_argument("--poisson", default="multigrid", choices=["jacobi", "multigrid"],
                    help="preconditioner of the Poisson batch in the timed steps (both solve to the same rtol)")
    ap.add_argument("--no-rules", action="store_true",
                    help="skip the precision form under other Krylov rules (dimension 12, 15, Sec. 3.2's rule)")
    ap.add_argument("--water", action="store_true",
                    help="only the water workload (8 orbitals, 5+5 electrons): FP64 path vs precision form over "
                         "--warmup + --steps steps (its JSON sub-entry)")
    ap.add_argument("--no-spectrum", action="store_true",
                    help="skip the precision form's dipole-trace and spectrum comparison on the reduced mesh")
    ap.add_argument("--spectrum-only", action="store_true",
                    help="only the precision form's dipole-trace and spectrum comparison (its JSON sub-entry)")
    ap.add_argument("--diff-only", action="store_true",
                    help="only the differentiation-form measurement (its JSON sub-entry)")
    ap.add_argument("--krylov-tol", type=float, default=1e-10,
                    help="Krylov error threshold per substep (0: one fixed-dimension Krylov step per time step)")
    ap.add_argument("--form", default="both", choices=["both", "mixed"],
                    help="both: time the FP64 path and the precision form; mixed: the precision form only")
    ap.add_argument("--kernels-only", action="store_true",
                    help="build the workload and run each operator kernel a few times (for profilers); no JSON")
    ap.add_argument("--profile-step", action="store_true",
                    help="one precision-form step with the inner CG capped (for a profiler's launch list); no JSON")
    ap.add_argument("--profile-integrals", action="store_true",
                    help="time the two-electron integrals (FP64 and tensor cores) on the workload mesh")
    ap.add_argument("--profile-gs", action="store_true",
                    help="a short precision-form propagation on a reduced coarse grid (the Gram-Schmidt kernels' "
                         "small capture case); one JSON line")
    ap.add_argument("--peaks", action="store_true",
                    help="only the measured FP64 and FP32 multiply-add peaks of this GPU (one JSON line)")
    ap.add_argument("--profile-arnoldi", action="store_true",
                    help="the orbital propagator alone: a short propagation, then ms per Krylov substep per form")
    args = ap.parse_args()
    if args.batch_only:
        import torch
        import paper_2301_02387_gb300 as pkg
        from paper_2301_02387_gb300 import inputs
        torch.cuda.set_device(0)
        print(json.dumps({"batching_form": run_batch(torch, pkg, inputs),
                          "batching_form_steps": run_batch_steps(torch, pkg, inputs)}))
        return
    if args.spectrum_only:
        import torch
        import paper_2301_02387_gb300 as pkg
        from paper_2301_02387_gb300 import inputs
        torch.cuda.set_device(0)
        print(json.dumps({"precision_spectrum": run_precision_spectrum(torch, pkg, inputs, steps=args.steps)}))
        return
    if args.diff_only:
        import torch
        import paper_2301_02387_gb300 as pkg
        from paper_2301_02387_gb300 import inputs
        torch.cuda.set_device(0)
        w = inputs.WORKLOADS[WORKLOAD]
        mesh, _solver, phi0, _ = setup_state(pkg, inputs, torch, w)
        phi = torch.from_numpy(phi0[:, 0].copy()).cuda()
        print(json.dumps({"differentiation_form": run_diff(torch, pkg, inputs, mesh, phi, steps=args.steps)}))
        return
    if args.water:
        import torch
        import paper_2301_02387_gb300 as pkg
        from paper_2301_02387_gb300 import inputs
        torch.cuda.set_device(0)
        out = {"water_workload": run_water(torch, pkg, inputs, args)}
        if not args.no_spectrum:
            out["water_precision_spectrum"] = run_precision_spectrum(torch, pkg, inputs, steps=300, name="water_q4",
                                                                     box=8.0, levels=2, nc=4)
        print(json.dumps(out))
        return
    if args.peaks:
        import torch
        import paper_2301_02387_gb300 as pkg
        torch.cuda.set_device(0)
        out = {k: [pkg.fma_peak(kind, 200.0) / 1e12 for _ in range(3)]
               for k, kind in (("fp64_tflops", pkg.PEAK_FP64), ("fp32_tflops", pkg.PEAK_FP32))}
        out["sms"] = torch.cuda.get_device_properties(0).multi_processor_count
        print(json.dumps({"peaks": out}))
        return
    if args.profile_arnoldi:
        run_profile_arnoldi(timed=args.steps > 0)
        return
    if args.profile_integrals:
        run_profile_integrals()
        return
    if args.profile_gs:
        run_profile_gs()
        return
    if args.kernels_only:
        run_kernels_only()
        return
    if args.profile_step:
        run_profile_step()
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
        dist = tdist
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    res = run_ours(args, rank, world, dist)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            try:
                res["cpu_baseline"] = cpu_baseline_entry(
                    cg_iters=res["_fp64_cg_iters"], substeps=res["_fp64_substeps"],
                    krylov_tol=args.krylov_tol if args.krylov_tol > 0 else 1e-10)
            except Exception as e:   # reported, never fatal
                res["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                       "sample": f"failed: {e}"}
        res.pop("_fp64_cg_iters", None)
        res.pop("_fp64_substeps", None)
        print(json.dumps(res), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
