"""Small, fixed workloads for profiling the library's kernels (e.g. under Nsight Compute).

    python profile_workloads.py jv [--n 16] [--reps 3]
        TGV n^3 P4 handle (levels 4-2-1), linearisation at the TGV field, `reps` exact
        Jacobian actions (face_kernel + vol_kernel per action) after a warm-up one, between
        cudaProfilerStart/Stop.
    python profile_workloads.py assemble [--n 16] [--form fp32|fp64]
        one preconditioner assembly after a warm-up one, between cudaProfilerStart/Stop.
    python profile_workloads.py stage [--n 16] [--form fp32|fp64|h16|bf16|h16tc|bf16tc] [--learned]
        one implicit stage to rel-res 1e-8 after two warm-up solves; only the timed FGMRES solve
        lies between cudaProfilerStart and cudaProfilerStop (ncu --profile-from-start off).

Prints the wall time of the profiled region. Inputs are the synthetic Taylor-Green states.
"""
import argparse
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("what", choices=["jv", "stage", "assemble"])
    ap.add_argument("--n", type=int, default=16)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--form", choices=["fp32", "fp64", "h16", "bf16", "h16tc", "bf16tc"], default="fp32")
    ap.add_argument("--learned", action="store_true", help="train the coarse network first and use it")
    ap.add_argument("--no-stb-rescale", dest="stb", action="store_false",
                    help="plain inherited coarse operators (the bench rescales their stabilisation part)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="default launch shapes (the bench measures them with dg_autotune)")
    a = ap.parse_args(argv)
    import torch

    import synthetic as S
    from paper_1809_00866_gb300 import (DG, DG_COARSE_LEARNED, DG_PRECOND_FP32, DG_PRECOND_FP32_BF16,
                                        DG_PRECOND_FP32_BF16_TC, DG_PRECOND_FP32_H16, DG_PRECOND_FP32_H16_TC,
                                        DG_PRECOND_FP64, DG_TUNE_FP32, DG_TUNE_FP64, build, solve_opts)
    build()
    un = S.uniform_nodes(a.n)
    levels = [4, 2, 1]
    dg = DG(un, un, un, levels, S.NU_TGV, S.AC_C, S.ETA)
    if a.stb:
        dg.dg_set_stb_rescaling(True)
    inv = 1.0 / S.acoustic_dt(a.n, levels[0])
    w = dg.empty()
    dg.dg_project_tgv(w)
    if a.what == "jv":
        dg.dg_set_linearization(w, inv)
        v = torch.from_numpy(S.direction(dg.ne, levels[0], S.SEED_V)).cuda()
        out = dg.empty()
        dg.dg_jvp(v, out)  # warm-up, outside the profiled window
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        t0 = time.perf_counter()
        for _ in range(a.reps):
            dg.dg_jvp(v, out)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        torch.cuda.profiler.stop()
        print("jv: %d actions, %.3f ms each" % (a.reps, 1e3 * t / a.reps))
        return 0
    if a.what == "assemble":
        prec = DG_PRECOND_FP64 if a.form == "fp64" else DG_PRECOND_FP32
        g = dg.empty()
        dg.dg_set_linearization_rhs(w, inv, g)
        dg.dg_assemble(precision=prec)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        t0 = time.perf_counter()
        dg.dg_assemble(precision=prec)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        torch.cuda.profiler.stop()
        print("assemble (%s): %.4f s" % (a.form, t))
        return 0
    # the settings of the benchmark's forms: reduced-precision cycles damped 0.95 with 5/5/2
    # sweeps, the FP64 cycle undamped with 2/2/2
    prec = {"fp32": DG_PRECOND_FP32, "fp64": DG_PRECOND_FP64, "h16": DG_PRECOND_FP32_H16,
            "bf16": DG_PRECOND_FP32_BF16, "h16tc": DG_PRECOND_FP32_H16_TC, "bf16tc": DG_PRECOND_FP32_BF16_TC}[a.form]
    low = prec != DG_PRECOND_FP64
    o = solve_opts(restart=30, maxit=300, rtol=1e-8, omega=0.95 if low else 1.0, pre_sweeps=5 if low else 2,
                   post_sweeps=5 if low else 2, coarse_sweeps=2, precision=prec)
    if a.learned:
        from paper_1809_00866_gb300 import learned as Lrn
        states = [w.clone()]
        for _ in range(3):
            g = dg.empty()
            dg.dg_set_linearization_rhs(states[-1], inv, g)
            dg.dg_assemble()
            x = dg.empty()
            dg.fgmres_solve(g, x, o)
            states.append((states[-1] + x).contiguous())
        D = Lrn.collect_rhs(dg, states, inv, o, per_state=40)
        dg.dg_set_linearization(states[-1], inv)
        dg.dg_assemble()
        Lrn.train_residual(dg, D, steps=2000, lr=1e-3, seed=0)
        o.coarse_solver = DG_COARSE_LEARNED
    g = dg.empty()
    dg.dg_set_linearization_rhs(w, inv, g)
    dg.dg_assemble(precision=o.precision)
    x = dg.empty()
    for _ in range(2):
        dg.fgmres_solve(g, x, o)
    if a.autotune:  # the bench's launch shapes
        for which in (DG_TUNE_FP64, DG_TUNE_FP32):
            dg.dg_autotune(which, use_cache=False)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    t0 = time.perf_counter()
    info, rc = dg.fgmres_solve(g, x, o)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    torch.cuda.profiler.stop()
    print("stage solve: %d iterations, %.4f s (%.3f ms per iteration), rc %d" % (info.its, t, 1e3 * t / max(1, info.its),
                                                                               rc))
    return 0


if __name__ == "__main__":
    sys.exit(main())
