#!/usr/bin/env python
"""Benchmark of the hot path: implicit stages of the Taylor-Green vortex, 32^3 hexahedra, P4, 3-level p-multigrid.

One step = one linearly implicit stage from the current state w (Sec. 2.2 with
gamma = 1): the stage right-hand side g = -f_h(w), the linearisation of G at w
(cached Riemann-flux Jacobian and velocities at the Gauss points), assembly of
the preconditioner (element diagonal blocks + inverses on every level,
inherited block-sparse coarse operators), FGMRES(30) on G dw = g with one
P4 -> P2 -> P1 V-cycle per iteration to a true relative residual of 1e-8, and
the state update w <- w + dw.

Prints one JSON line: value = seconds per implicit stage of the chosen form on
the 32^3 P4 mesh (device time, inputs resident in HBM, L2 flushed before every
timed stage), beside the plain FP64 form on the same mesh; the exact Jacobian
action throughput (Jv GDOF/s); the roofline of every timed kernel class against
measured peaks (HBM copy bandwidth, FP64/FP32 FMA rates measured here, BF16
tensor rate); the end-to-end time through the C ABI with host buffers over the
same stages; the SM clocks seen during the timed region; the oracle timed on the
host cores. Extra keys: the 16^3 mesh, the learned coarse correction on 24^3,
the walled channel and the batch of 64 uneven solves.

--impl reference times the FP64 CPU oracle on the same workload and metric.
Under torchrun every rank solves its own copy of the problem (replicas: the
path has no exchange step on one GPU); the reported time is the max over ranks.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402

METRIC = "Jv GDOF/s and s per implicit stage to rel-res 1e-8: chosen form vs plain FP64"
CONFIG = "tgv32_p4"
RTOL = 1e-8
def jv_flops(k, sum_factorised=True):
    """Algorithmic work (FLOP) of the exact Jacobian action per element, as the kernels compute it.

    Counted from the formulation (FMA = 2 FLOP; index arithmetic excluded):
    face pass, per face (3 per element): 2D traces 2*7*N_b, point values of the
    4 variables on both sides, linearised Riemann flux 32*N_qf, projection of the
    4 flux components, 2D viscous flux and lifting ~24*N_2. The FP64 pass takes the
    point values and the projection by sum factorisation over the face's two axes,
    8*n*(N_2 + N_qf) and 4*n*(N_qf + N_2); the FP32 pass densely, 8*N_qf*N_2 and
    4*N_qf*N_2 (sum_factorised=False).
    volume pass: corrected gradients 9*N_b*2, sum-factorised interpolation of 3
    fields 3*(N_b*n + N_2*n^2 + (k+1)*n^3), 6 products per point, sum-factorised
    projection of 6 fields 6*((k+1)*n^3 + N_2*n^2 + N_b*n), the viscous flux and
    the sparse modal derivatives ~30*N_b.
    Returns (face FLOP per element, volume FLOP per element).
    """
    n = k + 1
    nb = (k + 1) * (k + 2) * (k + 3) // 6
    n2 = (k + 1) * (k + 2) // 2
    nqf, nq = n * n, n ** 3
    if sum_factorised:
        points, proj = 8 * n * (n2 + nqf), 4 * n * (nqf + n2)
    else:
        points, proj = 8 * nqf * n2, 4 * nqf * n2
    face = 3 * 2 * (2 * 7 * nb + points + 32 * nqf + proj + 24 * n2)
    vol = 2 * (9 * nb * 2 + 3 * (nb * n + n2 * n * n + (k + 1) * nq) + 6 * nq
               + 6 * ((k + 1) * nq + n2 * n * n + nb * n) + 30 * nb)
    return float(face), float(vol)


# The dense-quadrature formulation (every contraction with the full N_q x N_b tables) needs
# about 0.52 MFLOP per element at P4; reported beside the achieved rate for reference.
DENSE_FLOP_PER_ELEMENT_P4 = 520_000.0
# Nominal FMA rates of a GB300, used only if the library's own measurement (dg_measure_peak) fails:
# FP64 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz ~ 1.26 TFLOP/s; FP32 152 x 128 lanes x 2 x 2.07 GHz.
FP64_NOMINAL_TFLOPS = 1.25
FP32_NOMINAL_TFLOPS = 80.5
BF16_FALLBACK_TFLOPS = 1900.0
# HBM peak: the measured copy bandwidth on the GB300s, else the machine's fallback.
HBM_FALLBACK_GBS = 6800.0
# DRAM bytes (read + write) per launch from Nsight Compute captures of the current kernels, by
# (profiler class, mesh n, block storage); a kernel changed since its capture has no entry.
# One-pass captures (dram__bytes_read.sum + dram__bytes_write.sum) of the chosen stage at 32^3 P4
# (FP16 blocks, 5/5/2 sweeps): the fine-level block-Jacobi apply moves 1.320 GB per sweep from
# zero and 1.357 GB per sweep with G x, one and nine of a cycle's ten fine-level sweeps, 1.353 GB
# per launch on average; the tensor-core volume pass 173.6 MB. (The FP64 face and volume passes
# changed after their capture.)
NCU_TRAFFIC = {("bj32_fine", 32, "half"): 1.353e9, ("vol_tc32", 32, "half"): 1.736e8}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def hbm_peak():
    d = measured_peaks()
    if "hbm_gbs" in d:
        return float(d["hbm_gbs"]), "measured"
    return HBM_FALLBACK_GBS, "fallback"


def bf16_peak(sustained):
    d = measured_peaks()
    key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
    if key in d:
        return float(d[key]), "measured"
    return BF16_FALLBACK_TFLOPS, "fallback"


# Fine-level operator applications (residual or Jacobian action) of one stage of the plain
# FP64 form on each workload, as counted by the library on the GPU (dg_counters): the number of
# the oracle's operator applications that the same plain algorithm makes per stage, used to scale
# the oracle's measured cost of one application to seconds per stage.
ORACLE_APPS_PER_STAGE = {"tgv4_p2": 70, "tgv16_p4": 105, "tgv24_p4": 105, "tgv32_p4": 107}


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(value, world, device):
    """The largest of the ranks' values (the job's time is its slowest replica's); the value
    itself on one rank. Collective: every rank must call it."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_seconds_per_stage(t_total, steps, world):
    """Whole-job seconds per stage: every rank runs `steps` stages of its own replica, and the
    job takes the slowest rank's total time t_total."""
    return t_total / (steps * world)


def mesh_nodes(cfg):
    n = cfg["n"]
    return S.uniform_nodes(n), S.uniform_nodes(n), S.uniform_nodes(n)


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "1", "0x1"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cores():
    """Host cores of this machine: (logical CPUs, CPU model line of lscpu or None)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return os.cpu_count() or 1, model


def oracle_jv_sample(cfg, threads, reps=1):
    """Mean seconds of one exact Jacobian action of the FP64 oracle on the full mesh of cfg (TGV
    state, the bench's direction) on `threads` host threads; and the DOF count."""
    import oracle as O
    O.threads(threads)
    xn, yn, zn = mesh_nodes(cfg)
    m = O.Mesh(xn, yn, zn, cfg["k"], S.NU_TGV, S.AC_C, S.ETA)
    w = O.project_tgv(m)
    v = S.direction(m.ne, cfg["k"], S.SEED_V)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        O.jvp(m, w, v, 1.0)
        ts.append(time.perf_counter() - t0)
    return statistics.mean(ts), m.n


def oracle_stage_sample(threads):
    """Seconds of one complete linearly implicit stage of the oracle on the 4^3 P2 Taylor-Green
    workload (residual, dense assembled G, inherited coarse operators and block inverses, FGMRES(30)
    with the 2-level V-cycle to rel-res 1e-8), on `threads` host threads; with its iterations."""
    import oracle as O
    import oracle.solvers as SV
    O.threads(threads)
    cfg = S.CONFIGS["tgv4_p2"]
    xn, yn, zn = mesh_nodes(cfg)
    m = O.Mesh(xn, yn, zn, cfg["k"], S.NU_TGV, S.AC_C, S.ETA)
    w = O.project_tgv(m)
    t0 = time.perf_counter()
    _, its, relres = SV.implicit_stage(m, w, 1.0 / S.acoustic_dt(cfg["n"], cfg["k"]), list(cfg["levels"]),
                                       rtol=RTOL)
    return time.perf_counter() - t0, its, relres


def cpu_baseline(config, apps, with_stage=True):
    """The oracle on the host cores: exact Jacobian actions on the full mesh of `config` (all
    cores), scaled by the fine-operator applications of one plain stage to s/stage; and, measured
    in full, one oracle stage of the 4^3 P2 workload on one core and on all cores."""
    ncpu, model = host_cores()
    cfg = S.CONFIGS[config]
    t_app, ndof = oracle_jv_sample(cfg, ncpu, reps=1 if cfg["n"] >= 32 else 3)
    out = {"value": t_app * apps, "unit": "s/stage", "cores": ncpu, "kind": "oracle",
           "sample": "exact Jacobian actions of the FP64 oracle on the full %d^3 P4 Taylor-Green state on %d "
                     "threads (%.2f s each), scaled by the %d fine-operator applications of one plain FP64 stage "
                     "(a lower bound: the oracle's assembly is not counted)" % (cfg["n"], ncpu, t_app, apps),
           "host": {"logical_cpus": ncpu, "model": model},
           "jv_seconds_all_cores": t_app, "jv_gdofs_all_cores": ndof / t_app / 1e9}
    if with_stage:
        stage = {}
        for nm, th in (("one_core", 1), ("all_cores", ncpu)):
            t, its, rr = oracle_stage_sample(th)
            stage[nm] = {"s_per_stage": t, "threads": th, "fgmres_its": its, "true_relres": rr}
        stage["workload"] = ("Taylor-Green 4^3 P2, levels 2-1, one linearly implicit stage to rel-res 1e-8, "
                             "measured in full (dense assembled operator)")
        out["measured_stage_tgv4_p2"] = stage
    return out


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    cfg = S.CONFIGS[args.config]
    apps = ORACLE_APPS_PER_STAGE[args.config]
    ncpu, model = host_cores()
    for _ in range(args.warmup):
        oracle_jv_sample(cfg, ncpu)
    times = []
    for _ in range(args.steps):
        t, ndof = oracle_jv_sample(cfg, ncpu)
        times.append(t)
    t_app = statistics.mean(times)
    value = t_app * apps
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s/stage", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "Taylor-Green vortex Re=1600, %d^3 periodic hexahedra, P4 (N_b=35), " % cfg["n"] +
                                   "p-levels 4-2-1, one linearly implicit stage to rel-res 1e-8",
                       "dofs": ndof, "l2": "oracle on host cores"},
            "jv": {"value": ndof / t_app / 1e9, "unit": "GDOF/s", "mode": "exact", "threads": ncpu},
            "cpu_baseline": {"value": value, "unit": "s/stage", "cores": ncpu, "kind": "oracle",
                             "sample": "one exact Jacobian action of the FP64 oracle on the full %d^3 P4 state on %d "
                                       "threads per step (%.2f s mean), scaled by the %d fine-operator applications "
                                       "of one plain FP64 stage" % (cfg["n"], ncpu, t_app, apps),
                             "host_model": model},
            "e2e": {"value": value, "unit": "s/stage", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_batch(args, P, make_opts, prec, stream, flush, world):
    """The batch workload: 64 independent periodic Taylor-Green boxes, n^3 cells with n drawn
    from 4..12 and k from {2, 3, 4} (seed 64), one linearly implicit stage each to rel-res 1e-8,
    each with its own acoustic time step. Three ways to run it:
      sequential: one handle per problem, the host-driven fgmres_solve, problem after problem;
      eager: one handle per degree holding all its boxes, the batched plan launched kernel by kernel;
      graph: the same plan captured once as one CUDA graph (the degree groups as parallel branches;
             one graph launch per restart cycle for all 64 problems)."""
    import torch
    boxes = S.batch_boxes()
    groups = {}
    for q, (n, k) in enumerate(boxes):
        groups.setdefault(k, []).append((q, n))
    hs, ws, gs, xs = [], [], [], []
    for k in sorted(groups):
        members = groups[k]
        bx = [(S.uniform_nodes(n),) * 3 for _, n in members]
        dg = P.DG(None, None, None, list(S.BATCH_LEVELS[k]), S.NU_TGV, S.AC_C, S.ETA, boxes=bx)
        if args.stb_rescale:
            dg.dg_set_stb_rescaling(True)
        dg.dg_set_problem_shifts([1.0 / S.acoustic_dt(n, k) for _, n in members])
        hs.append(dg)
        ws.append(dg.empty())
        gs.append(dg.empty())
        xs.append(dg.empty())
    singles = []
    for n, k in boxes:
        u = S.uniform_nodes(n)
        d1 = P.DG(u, u, u, list(S.BATCH_LEVELS[k]), S.NU_TGV, S.AC_C, S.ETA)
        if args.stb_rescale:
            d1.dg_set_stb_rescaling(True)
        singles.append((d1, 1.0 / S.acoustic_dt(n, k), d1.empty(), d1.empty(), d1.empty()))
    opts = make_opts()
    asm_prec = P.DG_PRECOND_FP64 if prec == P.DG_PRECOND_FP64 else P.DG_PRECOND_FP32
    ev = lambda: torch.cuda.Event(enable_timing=True)

    # every timed step is the first stage from the Taylor-Green field (at CFL 50 the 4^3 boxes
    # take steps of several time units, so the later stages of those boxes are not physical);
    # the whole stage is recomputed each time: right-hand side, linearisation, assembly, solve
    def batch_stage(plan):
        for dg, w, g in zip(hs, ws, gs):
            dg.dg_set_linearization_rhs(w, 1.0, g)
            dg.dg_assemble(precision=asm_prec)
        rc = plan.dg_plan_solve(check=False)
        if rc != P.DG_OK:
            bad = []
            for gi, k in enumerate(sorted(groups)):
                its, rr, cv = plan.dg_plan_result(gi)
                bad += ["n=%d k=%d its=%d relres=%.2e" % (n, k, its[j], rr[j])
                        for j, (q, n) in enumerate(groups[k]) if not cv[j]]
            raise RuntimeError("batched stage failed: %s: %s" % (P.load().dg_plan_error(plan.p).decode(),
                                                                  "; ".join(bad[:8])))

    def single_stage():
        its = []
        for (d1, inv, w, g, x), (n, k) in zip(singles, boxes):
            d1.dg_set_linearization_rhs(w, inv, g)
            d1.dg_assemble(precision=asm_prec)
            info, rc = d1.fgmres_solve(g, x, opts, check=False)
            if rc != P.DG_OK:
                raise RuntimeError("single stage n=%d k=%d did not converge: its %d relres %.2e"
                                   % (n, k, info.its, info.true_relres))
            its.append(info.its)
        return its

    def timed(fn, reset):
        reset()  # the stage's state; nothing below changes it
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        l0 = sum(d.dg_counters()[0] for d in hs) + sum(s[0].dg_counters()[0] for s in singles)
        times = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        l1 = sum(d.dg_counters()[0] for d in hs) + sum(s[0].dg_counters()[0] for s in singles)
        return statistics.mean(times), (l1 - l0) // max(1, args.steps)

    def reset_batch():
        for dg, w in zip(hs, ws):
            dg.dg_project_tgv(w)

    def reset_single():
        for d1, inv, w, g, x in singles:
            d1.dg_project_tgv(w)

    # first stage from the TGV field: the batch's solutions against the one-problem solves
    reset_batch()
    reset_single()
    plan_g = P.Plan(hs, gs, xs, opts, use_graph=True)
    plan_e = P.Plan(hs, gs, xs, opts, use_graph=False)
    for dg, w, g in zip(hs, ws, gs):
        dg.dg_set_linearization_rhs(w, 1.0, g)
        dg.dg_assemble(precision=asm_prec)
    plan_g.dg_plan_solve()
    first_its = single_stage()
    tuned = {}
    if args.autotune:  # every handle measured (one-box handles of the same shape share the result)
        for gi, (k, dg) in enumerate(zip(sorted(groups), hs)):
            tuned["k%d_batched" % k] = {}
            for nm, which in (("fp64_products", P.DG_TUNE_FP64), ("fp32_cycle", P.DG_TUNE_FP32)):
                dg.dg_autotune(which, use_cache=False)
                tuned["k%d_batched" % k][nm] = dg.dg_get_tuning(which).as_dict()
        for d1, *_ in singles:
            for which in (P.DG_TUNE_FP64, P.DG_TUNE_FP32):
                d1.dg_autotune(which, use_cache=True)
        plan_g.close()  # capture again with the tuned shapes
        plan_g = P.Plan(hs, gs, xs, opts, use_graph=True)
        plan_g.dg_plan_solve()
    diffs, batch_its, relres = [], [], []
    for gi, k in enumerate(sorted(groups)):
        its, rr, _ = plan_g.dg_plan_result(gi)
        es = hs[gi].elem_start
        for j, (q, n) in enumerate(groups[k]):
            xb = xs[gi].view(hs[gi].ne, -1)[es[j]:es[j + 1]].reshape(-1)
            xq = singles[q][4].reshape(-1)
            diffs.append(float((xb - xq).norm() / xq.norm()))
            batch_its.append((q, its[j]))
            relres.append(rr[j])
    its_by_q = dict(batch_its)
    t_graph, l_graph = timed(lambda: batch_stage(plan_g), reset_batch)
    t_eager, l_eager = timed(lambda: batch_stage(plan_e), reset_batch)
    t_single, l_single = timed(single_stage, reset_single)
    st = plan_g.dg_plan_stats()
    ndof = sum(d.n[0] for d in hs)
    out = {
        "workload": "64 independent Taylor-Green boxes [0,2pi]^3, n^3 periodic hexahedra with n ~ U{4..12} and "
                    "k ~ U{2,3,4} (seed 64), p-levels k-2-1 (2-1 for k=2), own acoustic dt (CFL 50) each; one "
                    "linearly implicit stage each from the Taylor-Green field to rel-res 1e-8 with the chosen "
                    "form's precision, block-Jacobi omega %.2f and sweeps %s (step = right-hand side, "
                    "linearisation, assembly and solve of all 64)" % (args.batch_omega, args.batch_sweeps),
        "problems_per_degree": {str(k): len(groups[k]) for k in sorted(groups)},
        "elements": sum(d.ne for d in hs), "dofs": ndof,
        "s_per_stage": {"graph": t_graph, "eager": t_eager, "sequential_one_handle_per_problem": t_single},
        "gdofs_per_s": {"graph": ndof / t_graph / 1e9, "sequential_one_handle_per_problem": ndof / t_single / 1e9},
        "speedup_graph_vs_sequential": t_single / t_graph, "speedup_graph_vs_eager": t_eager / t_graph,
        "kernel_launches_per_stage": {"graph": l_graph, "eager": l_eager, "sequential": l_single},
        "graph_launches_per_solve": st["cycles"], "arnoldi_steps_max": st["steps"],
        "tuning": tuned or None,
        "first_stage": {"its_batch_min_max": [min(its_by_q.values()), max(its_by_q.values())],
                        "its_sequential_min_max": [min(first_its), max(first_its)],
                        "its_equal_problems": sum(1 for q in its_by_q if its_by_q[q] == first_its[q]),
                        "max_true_relres": max(relres),
                        "max_solution_rel_diff_vs_sequential": max(diffs)},
    }
    plan_g.close()
    plan_e.close()
    for d1, *_ in singles:
        d1.close()
    for d in hs:
        d.close()
    return out


def channel_setup(args, P):
    """The channel workload's handle and fields: 24 x 12 x 12 hexahedra on 2pi x 2 x pi with
    no-slip walls at y = -1, 1 and tanh stretching (second cell 1.15 x the first), P3, p-levels
    3-2-1, viscosity for Re_tau = 180 of the laminar profile, initial field the laminar profile
    plus a 5% divergence-free perturbation (seed 180; other seeds give training states), acoustic
    CFL 50 on the smallest cell."""
    import numpy as np
    import torch
    c = S.CHANNEL
    xn, yn, zn = S.channel_nodes()
    nu = S.channel_nu(c["re_tau"])
    k = c["k"]
    dg = P.DG(xn, yn, zn, list(c["levels"]), nu, S.AC_C, S.ETA, walls=True)
    if args.stb_rescale:
        dg.dg_set_stb_rescaling(True)
    pts = dg.dg_quad_points().cpu().numpy()

    def field(seed):
        vals = np.ascontiguousarray(np.stack(S.channel_field(pts[..., 0], pts[..., 1], pts[..., 2], seed=seed),
                                             axis=1))
        w = dg.empty()
        dg.dg_project_points(torch.from_numpy(vals).cuda(), w)
        return w

    umax = 1.05
    dt = 50.0 * float(np.diff(yn).min()) / ((2 * k + 1) * (umax + math.sqrt(umax * umax + S.AC_C ** 2)))
    return {"dg": dg, "w0": field(180), "field": field, "inv": 1.0 / dt, "dt": dt, "nu": nu, "k": k}


def run_channel(args, P, ch, make_opts, plain_opts, learned_opts, stream, flush):
    """One linearly implicit stage of the channel from its initial field to rel-res 1e-8: the
    chosen form, the plain FP64 form and (when trained) the learned form. Every timed step
    recomputes the whole stage (right-hand side, linearisation, assembly, solve)."""
    import torch
    dg, w0, inv, dt, nu, k = ch["dg"], ch["w0"], ch["inv"], ch["dt"], ch["nu"], ch["k"]
    g, x = dg.empty(), dg.empty()
    asm = lambda o: P.DG_PRECOND_FP64 if o.precision == P.DG_PRECOND_FP64 else P.DG_PRECOND_FP32
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def stage(opts):
        dg.dg_set_linearization_rhs(w0, inv, g)
        dg.dg_assemble(precision=asm(opts))
        info, rc = dg.fgmres_solve(g, x, opts, check=False)
        if rc != P.DG_OK:
            raise RuntimeError("channel stage did not converge: its %d relres %.2e" % (info.its, info.true_relres))
        return info

    chosen = make_opts()
    if args.autotune:
        stage(chosen)
        for which in (P.DG_TUNE_FP64, P.DG_TUNE_FP32):
            dg.dg_autotune(which, use_cache=False)
    out = {}
    forms = [("plain_fp64", plain_opts), ("chosen", chosen)]
    if learned_opts is not None:
        forms.append(("learned", learned_opts))
    for name, opts in forms:
        for _ in range(args.warmup):
            stage(opts)
        torch.cuda.synchronize()
        times, its, rr = [], [], []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record(stream)
            info = stage(opts)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            its.append(info.its)
            rr.append(info.true_relres)
        out[name] = {"s_per_stage": statistics.mean(times), "fgmres_its": its, "true_relres": rr}
        if name == "learned":
            out[name]["fallback_at"] = info.fallback_at
    xs = {}
    for name, opts in (("plain_fp64", plain_opts), ("chosen", chosen)):
        stage(opts)
        xs[name] = x.clone()
    # the exact Jacobian action on this mesh
    v = torch.from_numpy(S.direction(dg.ne, k, S.SEED_V)).cuda()
    o = dg.empty()
    dg.dg_set_linearization(w0, inv)
    for _ in range(3):
        dg.dg_jvp(v, o)
    jt = []
    for _ in range(10):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        dg.dg_jvp(v, o)
        e1.record(stream)
        torch.cuda.synchronize()
        jt.append(e0.elapsed_time(e1) / 1e3)
    res = {
        "workload": "channel 2pi x 2 x pi, 24 x 12 x 12 hexahedra, no-slip walls at y = -1, 1 with tanh stretching "
                    "(ratio 1.15), P3 (N_b = 20), p-levels 3-2-1, Re_tau = 180 of the laminar profile "
                    "(nu = %.3e), laminar profile + 5%% divergence-free perturbation (seed 180), acoustic CFL 50 "
                    "on the smallest cell (dt = %.4f); one linearly implicit stage to rel-res 1e-8" % (nu, dt),
        "dofs": dg.n[0],
        "chosen": out["chosen"], "plain_fp64": out["plain_fp64"], "learned": out.get("learned"),
        "speedup_chosen_vs_plain": out["plain_fp64"]["s_per_stage"] / out["chosen"]["s_per_stage"],
        "first_stage_solution_rel_diff": float((xs["chosen"] - xs["plain_fp64"]).norm() / xs["plain_fp64"].norm()),
        "jv": {"value": dg.n[0] / statistics.median(jt) / 1e9, "unit": "GDOF/s", "mode": "exact (tangent), FP64",
               "ms": 1e3 * statistics.median(jt)},
        "tuning": {"fp64_products": dg.dg_get_tuning(P.DG_TUNE_FP64).as_dict(),
                   "fp32_cycle": dg.dg_get_tuning(P.DG_TUNE_FP32).as_dict()} if args.autotune else None,
    }
    if "learned" in out:
        res["learned"]["vs_chosen_without_network"] = out["chosen"]["s_per_stage"] / out["learned"]["s_per_stage"]
        res["learned"]["what"] = ("the chosen cycle with the network trained on Taylor-Green and channel states "
                                  "(seeds other than the timed field's) replacing the coarsest solve")
    dg.close()
    return res


FORM_NAMES = ("fp64", "fp32", "h16", "bf16", "h16tc", "bf16tc")


def form_precision(P, form):
    return {"fp32": P.DG_PRECOND_FP32, "fp64": P.DG_PRECOND_FP64, "h16": P.DG_PRECOND_FP32_H16,
            "bf16": P.DG_PRECOND_FP32_BF16, "h16tc": P.DG_PRECOND_FP32_H16_TC,
            "bf16tc": P.DG_PRECOND_FP32_BF16_TC}[form]


def form_dtype(form):
    base = "f64 (FGMRES, products with G, stage RHS) + f32 (preconditioner cycle)"
    return {"fp64": "f64", "fp32": base, "h16": base + " with f16 block storage",
            "bf16": base + " with bf16 block storage",
            "h16tc": base + " with f16 block storage and f16 tensor-core volume contractions (f32 accumulation)",
            "bf16tc": base + " with bf16 block storage and bf16 tensor-core volume contractions (f32 accumulation)"}[form]


class TgvCase:
    """One Taylor-Green mesh of the benchmark: its handle, state vectors and stage helpers."""

    def __init__(self, P, config, args, flush, world=1):
        import torch
        self.P, self.args, self.flush, self.world = P, args, flush, world
        self.config = config
        self.cfg = cfg = S.CONFIGS[config]
        self.k, self.levels = cfg["k"], list(cfg["levels"])
        xn, yn, zn = mesh_nodes(cfg)
        self.dg = P.DG(xn, yn, zn, self.levels, S.NU_TGV, S.AC_C, S.ETA)
        if args.stb_rescale:
            self.dg.dg_set_stb_rescaling(True)  # rescaled-inherited coarse operators (Appendix A)
        self.n0 = self.dg.n[0]
        self.dt = S.acoustic_dt(cfg["n"], self.k)
        self.inv = 1.0 / self.dt
        self.w, self.f, self.dw = self.dg.empty(), self.dg.empty(), self.dg.empty()
        self.st = torch.cuda.current_stream()
        self.plans = {}
        self.smoother = P.DG_SMOOTH_GMRES if args.smoother == "gmres" else P.DG_SMOOTH_JACOBI

    def opts(self, precision, omega, sweeps, **kw):
        a, b, c = (int(x) for x in sweeps.split(","))
        return self.P.solve_opts(restart=30, maxit=300, rtol=RTOL, precond=self.P.DG_PREC_VCYCLE, pre_sweeps=a,
                                 post_sweeps=b, coarse_sweeps=c, omega=omega, smoother=self.smoother,
                                 precision=precision, **kw)

    def ev(self):
        import torch
        return torch.cuda.Event(enable_timing=True)

    def solve(self, opts, krylov=None):
        """FGMRES on G dw = f: the device-driven plan (restart cycle as one CUDA graph) when
        --krylov plan and the options allow it, else the host-driven fgmres_solve."""
        P, dg = self.P, self.dg
        if (krylov or self.args.krylov) == "plan" and opts.fallback_its == 0:
            key = tuple(getattr(opts, fld) for fld, _ in opts._fields_)
            if key not in self.plans:
                self.plans[key] = P.Plan([dg], [self.f], [self.dw], opts, use_graph=True)
            pl = self.plans[key]
            rc = pl.dg_plan_solve(check=False)
            its, rr, _ = pl.dg_plan_result(0)
            return rc, its[0], rr[0], -1
        info, rc = dg.fgmres_solve(self.f, self.dw, opts)
        return rc, info.its, info.true_relres, info.fallback_at

    def stage(self, w, opts, log, phases=None, assemble=True, krylov=None):
        """One linearly implicit stage from w, all in the library: g = -f_h(w) and the
        linearisation, the assembly (or the lagged one), the solve, w <- w + dw."""
        dg, st = self.dg, self.st
        e = [self.ev() for _ in range(4)] if phases is not None else None
        if e: e[0].record(st)
        dg.dg_set_linearization_rhs(w, self.inv, self.f)
        if e: e[1].record(st)
        if assemble:
            dg.dg_assemble(precision=opts.precision)
        else:
            dg.dg_reuse_assembly()
        if e: e[2].record(st)
        rc, its, relres, fb = self.solve(opts, krylov)
        if rc != self.P.DG_OK:
            raise RuntimeError("stage did not converge: rc %d relres %.3e" % (rc, relres))
        dg.dg_stage_update(w, self.dw)
        if e:
            e[3].record(st)
            phases.append(e)
        log["its"].append(its)
        log["relres"].append(relres)
        log.setdefault("fallback_at", []).append(fb)

    def run_form(self, opts, steps, warmup, lag=1):
        """`warmup` untimed stages from the Taylor-Green field, then `steps` timed ones (L2 flushed
        before each); seconds per stage over the whole job (max over ranks)."""
        import torch
        dg = self.dg
        dg.dg_project_tgv(self.w)
        count = 0
        for _ in range(warmup):
            self.stage(self.w, opts, {"its": [], "relres": []}, assemble=count % lag == 0)
            count += 1
        torch.cuda.synchronize()
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()
        log = {"its": [], "relres": []}
        l0, a0 = dg.dg_counters()
        times, phases = [], []
        for _ in range(steps):
            self.flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = self.ev(), self.ev()
            e0.record(self.st)
            self.stage(self.w, opts, log, phases, assemble=count % lag == 0)
            count += 1
            e1.record(self.st)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        l1, a1 = dg.dg_counters()
        t_total = max_over_ranks(sum(times), self.world, "cuda")
        names = ["rhs_and_linearize", "assemble", "solve"]
        breakdown = {nm: statistics.mean(ph[i].elapsed_time(ph[i + 1]) for ph in phases) / 1e3
                     for i, nm in enumerate(names)}
        return {"s_per_stage": job_seconds_per_stage(t_total, steps, self.world), "t_total": t_total,
                "steps": steps, "warmup": warmup, "breakdown_s": breakdown,
                "fgmres_its": log["its"], "true_relres": log["relres"], "fallback_at": log.get("fallback_at"),
                "operator_applications": (a1 - a0) / max(1, steps),
                "gpu_launches": (l1 - l0) // max(1, steps)}

    def autotune(self, opts):
        """Launch shapes of the hot kernels measured on this handle (untimed setup): the first
        stage's linearisation and assembly, one cycle to make the 16-bit block copies, the tuner."""
        P, dg = self.P, self.dg
        dg.dg_project_tgv(self.w)
        dg.dg_set_linearization_rhs(self.w, self.inv, self.f)
        dg.dg_assemble(precision=opts.precision)
        dg.pmg_vcycle(self.f, self.dw, opts)
        tuning = {}
        for nm, which in (("fp64_products", P.DG_TUNE_FP64), ("fp32_cycle", P.DG_TUNE_FP32)):
            rep = dg.dg_autotune(which, use_cache=False)
            tuning[nm] = {"chosen": dg.dg_get_tuning(which).as_dict(), "device_ms_default_vs_chosen": rep}
        return tuning

    def first_stage_error(self, plain_opts, chosen_opts):
        """The chosen form's first-stage correction against the plain FP64 form's."""
        dg = self.dg
        dg.dg_project_tgv(self.w)
        dg.dg_set_linearization_rhs(self.w, self.inv, self.f)
        dg.dg_assemble(precision=plain_opts.precision)
        d64, d32 = dg.empty(), dg.empty()
        dg.fgmres_solve(self.f, d64, plain_opts)
        dg.dg_assemble(precision=chosen_opts.precision)
        dg.fgmres_solve(self.f, d32, chosen_opts)
        return float((d32 - d64).norm() / d64.norm())

    def close(self):
        for pl in self.plans.values():
            pl.close()
        self.dg.close()


def fp32_operator_times(case, opts_by_name):
    """Device ms per launch of the FP32 cycle's operator passes (face pass, volume pass on CUDA
    cores or on the tensor cores), timed inside five V-cycles of each form (L2 flushed)."""
    import torch
    P, dg = case.P, case.dg
    dg.dg_set_linearization(case.w, case.inv)
    dg.dg_assemble(precision=P.DG_PRECOND_FP32)
    g32 = torch.from_numpy(S.direction(dg.ne, case.k, S.SEED_V + 1)).cuda()
    z32 = dg.empty()
    out = {}
    for nm, o in opts_by_name.items():
        dg.pmg_vcycle(g32, z32, o)
        dg.dg_profile(True)
        dg.dg_profile_read()
        for _ in range(5):
            case.flush.zero_()
            dg.pmg_vcycle(g32, z32, o)
        prof = dg.dg_profile_read()
        dg.dg_profile(False)
        ent = {}
        for cls in ("face_tan32", "vol_tan32", "vol_tc32"):
            ms_k, cnt = prof[cls]
            if cnt:
                ent[cls] = {"ms_per_launch": ms_k / cnt, "launches": cnt}
        out[nm] = ent
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1809_00866_gb300 as P
    if rank == 0:
        P.build()
    if world > 1:
        dist.barrier()
    P.build()
    # measured arithmetic peaks of this device (the ALU rooflines' denominators)
    try:
        fp64_peak, fp64_src = P.dg_measure_peak(P.DG_PEAK_FP64_FMA), "measured (dg_measure_peak, FP64 FMA chains)"
        fp32_peak, fp32_src = P.dg_measure_peak(P.DG_PEAK_FP32_FMA), "measured (dg_measure_peak, FP32 FMA chains)"
    except P.DgError:
        fp64_peak, fp64_src = FP64_NOMINAL_TFLOPS, "nominal (measurement failed)"
        fp32_peak, fp32_src = FP32_NOMINAL_TFLOPS, "nominal (measurement failed)"
    try:  # read-only streaming bandwidth: context for the read-dominated block products
        hbm_read = P.dg_measure_peak(P.DG_PEAK_HBM_READ)
    except P.DgError:
        hbm_read = None
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device="cuda")  # 512 MB > L2
    K, W = args.steps, args.warmup
    case = TgvCase(P, args.config, args, flush, world)
    dg, k, n0 = case.dg, case.k, case.n0
    chosen_prec = form_precision(P, args.form)
    chosen_opts = case.opts(chosen_prec, args.omega, args.sweeps)
    # the plain form at its own best measured setting (undamped, 2/2/2 sweeps)
    plain_opts = case.opts(P.DG_PRECOND_FP64, 1.0, args.plain_sweeps)
    tuning = case.autotune(chosen_opts) if args.autotune else None
    chan = channel_setup(args, P) if args.channel else None

    clk = Clocks(local)
    clk.start()
    chosen = case.run_form(chosen_opts, K, W)
    plain = case.run_form(plain_opts, min(K, args.plain_steps), min(W, 3))
    lagged = case.run_form(chosen_opts, min(K, 10), 3, lag=args.lag) if args.lag > 1 else None
    clocks = clk.stop()
    chosen_err = case.first_stage_error(plain_opts, chosen_opts)

    # --- exact Jacobian action throughput and the roofline of its kernels (L2 flushed each time)
    st = case.st
    v = torch.from_numpy(S.direction(dg.ne, k, S.SEED_V)).cuda()
    out = dg.empty()
    dg.dg_project_tgv(case.w)
    dg.dg_set_linearization(case.w, case.inv)
    for _ in range(5):
        dg.dg_jvp(v, out)
    jv_times = []
    dg.dg_profile(True)
    dg.dg_profile_read()
    for _ in range(args.jv_reps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = case.ev(), case.ev()
        e0.record(st)
        dg.dg_jvp(v, out)
        e1.record(st)
        torch.cuda.synchronize()
        jv_times.append(e0.elapsed_time(e1) / 1e3)
    prof = dg.dg_profile_read()
    dg.dg_profile(False)
    t_jv = statistics.median(jv_times)
    jv_gdofs = n0 / t_jv / 1e9
    face_ms = prof["face_tan"][0] / max(1, prof["face_tan"][1])
    vol_ms = prof["vol_tan"][0] / max(1, prof["vol_tan"][1])
    ff, fv = jv_flops(k)
    if face_ms >= vol_ms:
        kname, kms, kflop = "face_kernel<%d,tangent,double>" % k, face_ms, ff * dg.ne
    else:
        kname, kms, kflop = "vol_kernel<%d,tangent,double>" % k, vol_ms, fv * dg.ne
    achieved = kflop / (kms / 1e3) / 1e12
    storage_jv = {"fp32": "float", "h16": "half", "bf16": "bfloat16", "h16tc": "half", "bf16tc": "bfloat16"}.get(args.form)
    traffic_jv = NCU_TRAFFIC.get(("face_tan" if kname.startswith("face") else "vol_tan", case.cfg["n"], storage_jv))
    roofline_jv = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": fp64_peak,
                   "unit": "TFLOP/s", "frac": achieved / fp64_peak, "traffic": traffic_jv, "peak_source": fp64_src,
                   "frac_of": "of measured" if fp64_src.startswith("measured") else "of nominal",
                   "flop_per_element": {"face": ff, "vol": fv},
                   "kernel_ms": {"face_tan": face_ms, "vol_tan": vol_ms},
                   "face_frac": ff * dg.ne / (face_ms / 1e3) / 1e12 / fp64_peak,
                   "vol_frac": fv * dg.ne / (vol_ms / 1e3) / 1e12 / fp64_peak,
                   "jv_tflops_of_implemented_work": (ff + fv) * dg.ne / t_jv / 1e12,
                   "jv_dense_equivalent_tflops": DENSE_FLOP_PER_ELEMENT_P4 * dg.ne / t_jv / 1e12}

    # --- the FP32 cycle's operator passes: CUDA-core volume pass against the tensor-core one
    op32 = fp32_operator_times(case, {
        "cuda_core_h16": case.opts(P.DG_PRECOND_FP32_H16, args.omega, args.sweeps),
        "tensor_core_h16": case.opts(P.DG_PRECOND_FP32_H16_TC, args.omega, args.sweeps)})

    # --- the chosen stage's kernels, timed live with CUDA events on the launching stream
    dg.dg_project_tgv(case.w)
    dg.dg_profile(True)
    dg.dg_profile_read_bytes()
    flush.zero_()
    case.stage(case.w, chosen_opts, {"its": [], "relres": []}, krylov="host")  # eager: events bracket each launch
    kp = dg.dg_profile_read_bytes()
    dg.dg_profile(False)
    hbm, hbm_src = hbm_peak()
    bf16, bf16_src = bf16_peak(sustained=False)
    kernels = {}
    for nm, (ms_k, cnt, by) in kp.items():
        if cnt:
            kernels[nm] = {"launches": cnt, "ms_per_launch": ms_k / cnt, "total_ms": ms_k}
            if by > 0:
                kernels[nm]["gbs"] = by / (ms_k / 1e3) / 1e9
    storage = {"fp32": "float", "h16": "half", "bf16": "bfloat16", "h16tc": "half", "bf16tc": "bfloat16"}.get(args.form)
    names = {"bj32_fine": "staged_jacobi_kernel<float, %s> (fine level)" % storage,
             "bj64_fine": "bj_update_kernel<double> (fine level)",
             "bsr32_l1": ("direct_apply_kernel<float, 7, float> (P2 level)" if args.form == "fp32" else
                          "direct7_vec_kernel<%s> (P2 level)" % storage),
             "bsr64_l1": "direct_apply_kernel<double, 7, double> (P2 level)",
             "face_tan32": "face_kernel<%d, tangent, float>" % k, "vol_tan32": "vol_kernel<%d, tangent, float>" % k,
             "vol_tc32": "tc_vol_kernel<%d, %s> (tcgen05)" % (k, "bf16" if args.form == "bf16tc" else "f16"),
             "face_tan": "face_kernel<%d, tangent, double>" % k, "vol_tan": "vol_kernel<%d, tangent, double>" % k}
    hbm_note = ("measured HBM copy bandwidth (hbm_gbs of the measured-peaks file)" if hbm_src == "measured"
                else "fallback HBM bandwidth 6.8 TB/s")
    nb = (k + 1) * (k + 2) * (k + 3) // 6
    nq, n2 = (k + 1) ** 3, (k + 1) * (k + 2) // 2
    by_kernel = {}
    for nm, (ms_k, cnt, by) in kp.items():
        if not cnt or nm not in names:
            continue
        t = ms_k / cnt / 1e3
        if nm == "vol_tc32":
            # algorithmic bytes per element: the input and output coefficients, the linearisation
            # velocity at the points, the face-slot contributions and liftings (FP32, read once)
            b_el = 4.0 * (2 * 4 * nb + 3 * nq + 6 * 4 * n2 + 6 * 3 * n2)
            ach = b_el * dg.ne / t / 1e9
            tflop = 2.0 * nq * nb * 9 * dg.ne / t / 1e12  # the two dense contractions' useful FLOP
            ent = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                   "algorithmic_bytes_per_launch": b_el * dg.ne, "peak_source": hbm_note, "frac_of": "of " + hbm_src,
                   "tensor": {"achieved_tflops": tflop, "peak_tflops": bf16, "frac": tflop / bf16,
                              "peak_source": "bf16 dense burst of the measured-peaks file (f16 the same nominal rate)"
                              if bf16_src == "measured" else "fallback 1.9 PFLOP/s"}}
        elif by > 0:
            ach = by / cnt / t / 1e9
            ent = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                   "algorithmic_bytes_per_launch": by / cnt, "peak_source": hbm_note, "frac_of": "of " + hbm_src,
                   "frac_of_read_stream": ach / hbm_read if hbm_read else None}
        else:
            f32 = nm.endswith("32")
            flop = ((jv_flops(k, sum_factorised=False)[0] if f32 else ff) if nm.startswith("face") else fv) * dg.ne
            peak = fp32_peak if f32 else fp64_peak
            ach = flop / t / 1e12
            ent = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                   "algorithmic_flop_per_launch": flop, "peak_source": fp32_src if f32 else fp64_src}
        ent.update({"kernel": names[nm], "ms_per_launch": t * 1e3, "launches": cnt, "total_ms": ms_k,
                    "traffic": NCU_TRAFFIC.get((nm, case.cfg["n"], storage))})
        by_kernel[nm] = ent
    if by_kernel:
        top = max(by_kernel, key=lambda n: by_kernel[n]["total_ms"])
        roofline = dict(by_kernel[top], profiler_class=top)
    else:
        roofline = roofline_jv

    # --- end to end through the C ABI: the same warm-up and timed stages as `value`, each with its
    # state copied in from pinned host memory and the updated state copied back
    dg.dg_project_tgv(case.w)
    host_w = case.w.detach().cpu().pin_memory()
    wd = dg.empty()
    e2e_times = []
    for step in range(W + K):
        timed = step >= W
        if timed:
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = case.ev(), case.ev()
            e0.record(st)
        wd.copy_(host_w, non_blocking=True)
        case.stage(wd, chosen_opts, {"its": [], "relres": []})
        host_w.copy_(wd, non_blocking=True)
        if timed:
            e1.record(st)
        torch.cuda.synchronize()
        if timed:
            e2e_times.append(e0.elapsed_time(e1) / 1e3)
    e2e_total = max_over_ranks(sum(e2e_times), world, "cuda")
    e2e = {"value": job_seconds_per_stage(e2e_total, K, world), "unit": "s/stage", "h2d_bytes_per_step": n0 * 8,
           "d2h_bytes_per_step": n0 * 8, "stages": K,
           "what": "the same %d warm-up and %d timed stages from the Taylor-Green field as value; each stage "
                   "copies the state from pinned host memory to the device and the updated state back" % (W, K)}

    line = {"metric": METRIC, "value": chosen["s_per_stage"], "unit": "s/stage", "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * chosen["t_total"] / K,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": form_dtype(args.form), "data": "synthetic",
            "config": {"workload": "Taylor-Green vortex Re=1600, %d^3 periodic hexahedra, P4 (N_b=35), " % case.cfg["n"] +
                                   "p-levels 4-2-1, one linearly implicit stage to rel-res 1e-8",
                       "dofs": n0, "dt": case.dt,
                       "solver": "FGMRES(30) + MG_V, %s smoother, pre/post/coarse %s (plain form %s)%s; %s"
                                 % (args.smoother, args.sweeps, args.plain_sweeps,
                                    ", rescaled-inherited coarse operators" if args.stb_rescale else "",
                                    "device-driven FGMRES, restart cycle (V-cycle included) as one CUDA graph"
                                    if args.krylov == "plan" else "host-driven FGMRES"),
                       "l2": "flushed (512 MB write) before every timed stage and Jacobian action",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "jv": {"value": jv_gdofs, "unit": "GDOF/s", "mode": "exact (tangent), FP64", "ms": 1e3 * t_jv},
            "form": "chosen: %s preconditioner cycle, block-Jacobi omega %.2f, sweeps %s, inside FP64 FGMRES; "
                    "plain: FP64 cycle, omega 1, sweeps %s" % (args.form.upper(), args.omega, args.sweeps,
                                                              args.plain_sweeps),
            "stage": chosen, "plain_fp64": plain,
            "chosen_vs_plain": {"speedup": plain["s_per_stage"] / chosen["s_per_stage"],
                                "first_stage_solution_rel_diff": chosen_err},
            "roofline": roofline, "roofline_by_kernel": by_kernel, "roofline_jv": roofline_jv,
            "fp32_operator_passes": op32,
            "peaks": {"fp64_fma_tflops": fp64_peak, "fp32_fma_tflops": fp32_peak, "hbm_gbs": hbm,
                      "hbm_read_stream_gbs": hbm_read, "bf16_tflops": bf16},
            "stage_kernels": kernels,
            "clocks": clocks, "e2e": e2e, "gpu_launches": chosen["gpu_launches"], "tuning": tuning}
    if lagged is not None:
        line["lagged_form"] = {
            "lag": args.lag, "what": "the chosen form with the preconditioner (element blocks, factors, coarse "
                                    "block-sparse operators) assembled every %d stages and reused in between" % args.lag,
            "s_per_stage": lagged["s_per_stage"], "fgmres_its": lagged["fgmres_its"],
            "breakdown_s": lagged["breakdown_s"], "vs_plain_fp64": plain["s_per_stage"] / lagged["s_per_stage"]}
    # --- the other Taylor-Green meshes
    if args.extra_meshes:
        for cname in [c for c in ("tgv16_p4",) if c != args.config]:
            c2 = TgvCase(P, cname, args, flush, world)
            o2 = c2.opts(chosen_prec, args.omega, args.sweeps)
            p2 = c2.opts(P.DG_PRECOND_FP64, 1.0, args.plain_sweeps)
            if args.autotune:
                c2.autotune(o2)
            r_ch = c2.run_form(o2, min(K, 10), 3)
            r_pl = c2.run_form(p2, min(K, 5), 3)
            line[cname + "_form"] = {"s_per_stage": r_ch["s_per_stage"], "fgmres_its": r_ch["fgmres_its"],
                                     "plain_fp64": {"s_per_stage": r_pl["s_per_stage"],
                                                    "fgmres_its": r_pl["fgmres_its"]},
                                     "speedup_chosen_vs_plain": r_pl["s_per_stage"] / r_ch["s_per_stage"],
                                     "dofs": c2.n0}
            c2.close()
    if args.learned:
        line["learned_form"] = run_learned(args, P, flush, world, chosen_prec, chan)
    if chan is not None:
        ch_opts = lambda: case.opts(chosen_prec, args.omega, args.sweeps)
        line["channel_form"] = run_channel(args, P, chan, ch_opts, plain_opts,
                                           line.get("learned_form", {}).pop("_opts", None), st, flush)
    elif "learned_form" in line:
        line["learned_form"].pop("_opts", None)
    if args.batch:
        line["batch_form"] = run_batch(args, P, lambda: case.opts(chosen_prec, args.batch_omega, args.batch_sweeps),
                                       chosen_prec, st, flush, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.config, ORACLE_APPS_PER_STAGE[args.config])
        line["cpu_baseline"]["gpu_plain_fp64_operator_applications_per_stage"] = plain["operator_applications"]
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    case.close()
    return 0


def run_learned(args, P, flush, world, chosen_prec, chan):
    """The learned coarse correction on its own workload, the 24^3 P4 Taylor-Green mesh: the network
    is trained here (untimed setup) by the library's BF16 kernels on the coarse right-hand sides the
    chosen cycle produces in the first stages (and on channel states of other seeds than the timed
    channel field), then the chosen form is timed with and without it on the same stages."""
    import torch
    import paper_1809_00866_gb300.learned as Lrn
    c = TgvCase(P, "tgv24_p4", args, flush, world)
    dg = c.dg
    pre, post, coarse = (int(x) for x in args.sweeps.split(","))
    base = c.opts(chosen_prec, args.omega, args.sweeps)
    if args.autotune:
        c.autotune(base)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dg.dg_project_tgv(c.w)
    states = [c.w.clone()]
    for _ in range(3):
        c.stage(c.w, base, {"its": [], "relres": []})
        states.append(c.w.clone())
    D = Lrn.collect_rhs(dg, states, c.inv, base, per_state=40)
    extra = []
    if chan is not None:  # channel states of other seeds than the timed field
        chan_states = [chan["field"](sd) for sd in (181, 182, 183)]
        Dc = Lrn.collect_rhs(chan["dg"], chan_states, chan["inv"], base, per_state=40)
        extra.append((chan["dg"], Dc))
    torch.cuda.synchronize()
    t_collect = time.perf_counter() - t0
    dg.dg_set_linearization(states[-1], c.inv)
    dg.dg_assemble()
    theta, rep = Lrn.train_residual(dg, D, steps=args.learn_steps, lr=1e-3, seed=0, extra=extra)
    r_net = Lrn.residual_ratio(dg, D[-8:])
    lc = len(c.levels) - 1
    yj, rj = dg.empty(lc), dg.empty(lc)
    r_jac = []
    for d in D[-8:]:
        yj.zero_()
        dg.block_jacobi_smooth(lc, d, yj, max(1, coarse), args.omega)
        rj.copy_(d)
        dg.bsr_spmv(lc, -1.0, yj, 1.0, rj)
        r_jac.append(float(rj.norm().item()) / float(d.norm().item()))
    learned_opts = c.opts(chosen_prec, args.omega, args.sweeps, coarse_solver=P.DG_COARSE_LEARNED, fallback_its=5,
                          fallback_rho=0.8)
    steps = min(args.steps, 10)
    without = c.run_form(base, steps, 3)
    with_net = c.run_form(learned_opts, steps, 3)
    out = {"workload": "Taylor-Green vortex Re=1600, 24^3 periodic hexahedra, P4, p-levels 4-2-1 (the learned "
                       "form's own configuration)", "dofs": c.n0,
           "collect_s": t_collect, "train_s": rep["train_s"], "train_steps": rep["steps"],
           "coarse_vectors": rep["vectors"],
           "coarse_residual_ratio": {"network": r_net,
                                     "block_jacobi_%d_sweeps" % max(1, coarse): statistics.mean(r_jac)},
           "cycle": "the chosen cycle with its coarsest (P1) solve replaced by the BF16 network followed by "
                    "%d block-Jacobi sweeps; fallback to the plain coarse solve if the residual estimate is "
                    "above 0.8^its after 5 iterations" % coarse,
           "with_network": {"s_per_stage": with_net["s_per_stage"], "fgmres_its": with_net["fgmres_its"],
                            "fallback_at": with_net["fallback_at"]},
           "without_network": {"s_per_stage": without["s_per_stage"], "fgmres_its": without["fgmres_its"]},
           "gain": without["s_per_stage"] / with_net["s_per_stage"],
           "_opts": learned_opts}
    c.close()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default=CONFIG, choices=sorted(S.CONFIGS))
    ap.add_argument("--jv-reps", type=int, default=30)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--smoother", choices=["jacobi", "gmres"], default="jacobi")
    ap.add_argument("--sweeps", default="5,5,2", help="pre,post,coarse smoothing iterations of the chosen form")
    ap.add_argument("--plain-sweeps", default="2,2,2", help="pre,post,coarse smoothing iterations of the plain form")
    ap.add_argument("--plain-steps", type=int, default=5, help="timed stages of the plain FP64 form (at most --steps)")
    ap.add_argument("--form", choices=FORM_NAMES, default="h16tc",
                    help="precision of the chosen form's cycle (h16 / bf16: FP32 cycle with 16-bit block storage; "
                         "h16tc / bf16tc: the same with the volume contractions on the tensor cores)")
    ap.add_argument("--omega", type=float, default=0.95, help="block-Jacobi damping of the chosen form")
    ap.add_argument("--batch-sweeps", default="3,3,2",
                    help="pre,post,coarse smoothing iterations of the batch of uneven solves (its small meshes "
                         "converge best with fewer sweeps)")
    ap.add_argument("--batch-omega", type=float, default=0.9, help="block-Jacobi damping of the batch")
    ap.add_argument("--no-learned", dest="learned", action="store_false",
                    help="skip the learned coarse correction (trained and timed on the 24^3 mesh)")
    ap.add_argument("--learn-steps", type=int, default=2000)
    ap.add_argument("--no-stb-rescale", dest="stb_rescale", action="store_false",
                    help="keep the plain inherited coarse operators (default: rescale their stabilisation "
                         "part, Appendix A)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default launch shapes (no dg_autotune)")
    ap.add_argument("--krylov", choices=["host", "plan"], default="plan",
                    help="FGMRES of the stages: host-driven fgmres_solve, or the device-driven plan whose restart "
                         "cycle is one CUDA graph (forms without the learned form's fallback)")
    ap.add_argument("--no-extra-meshes", dest="extra_meshes", action="store_false",
                    help="skip the 16^3 Taylor-Green mesh")
    ap.add_argument("--no-channel", dest="channel", action="store_false",
                    help="skip the walled channel workload")
    ap.add_argument("--no-batch", dest="batch", action="store_false",
                    help="skip the batch of 64 uneven independent solves")
    ap.add_argument("--lag", type=int, default=2, help="also time the chosen form with the preconditioner "
                                                       "assembled every LAG stages (1: skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
