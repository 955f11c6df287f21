"""Benchmark: time-to-RCS at a 1e-4 relative residual and MLFMM matvec GB/s,
chosen form (mixed precision, ILU(0)-preconditioned FGMRES) vs plain FP64 form.

Workload: two-layer coated dielectric sphere (core radius 1.0 lambda0, eps_r 4;
shell radius 1.5 lambda0, eps_r 2.56) in free space, geodesic meshes of
frequency 30 (outer) and 20 (inner), 78 000 unknowns, 5-level MLFMM, one
x-polarised plane wave along -z, bistatic RCS at 361 angles.  Synthetic
geometry (the paper's meshes are not published).

One step = plane-wave excitation + FGMRES(50) with ILU(0) to 1e-4 + bistatic
RCS.  Under torchrun each rank solves its own incidence angle (independent
replicas, weak scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-RCS at 1e-4 residual & MLFMM matvec GB/s: chosen vs plain FP64 form"
WORKLOAD = "coated_c2"
LEVELS = 5
DIGITS = 3.0
TOL = 1e-4
RESTART = 50
NANO_LEVELS = 4
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes (read + write) of one k_near_spmv<float> launch on this workload, from one
# ncu capture of that kernel; valid while the kernel is unchanged
NEAR_SPMV_TRAFFIC_BYTES = 508421888 + 521984
# DRAM bytes (read + write) of one single-RHS FP32 ILU(0) apply (15 k_ilu_sweep<float, 512>
# launches) on this workload, from one ncu capture of those launches; valid while the kernel
# is unchanged (None otherwise)
ILU_APPLY_TRAFFIC_BYTES = 566045184 + 139520


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """Samples nvidia-smi SM clocks and throttle reasons while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.n0 = 0
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            # the timed region starts once nvidia-smi is sampling; only later samples count
            t0 = time.time()
            while not self.rows and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.n0 = len(self.rows)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if len(self.rows) > self.n0:
            self.rows = self.rows[self.n0:]
        sm = [float(r[0]) for r in self.rows if len(r) >= 7 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 7 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 7 for i in range(4) if "Active" in r[3 + i]
                          and "Not" not in r[3 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_incidence(rank):
    """Each rank solves its own incidence (replicas): theta_i = 0.05 rad x rank,
    phi_i = 0, theta-polarised, unit amplitude."""
    return np.array([[0.05 * rank, 0.0, 0.0, 1.0]])


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (the job's time) on every rank."""
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- CPU oracle timing
def oracle_sample(mesh, rng_seed=0, nrows=4):
    """Time the oracle on a bounded sample of the workload and extrapolate its
    time-to-RCS: dense rows of the JMCFIE matrix (all media), a dense LU of a
    smaller complex system scaled by N^3, and a few far-field angles."""
    from oracle import farfield, fill
    from oracle.rwg import Mesh
    t0 = time.perf_counter()
    m = Mesh(**mesh)
    t_mesh = time.perf_counter() - t0
    rows = np.random.default_rng(rng_seed).choice(m.ne, nrows, replace=False)
    t0 = time.perf_counter()
    fill.assemble(m, rows=rows)
    t_rows = time.perf_counter() - t0
    n_lu = 2000
    A = np.random.default_rng(1).standard_normal((n_lu, n_lu)) + 1j * np.eye(n_lu) * n_lu
    t0 = time.perf_counter()
    np.linalg.solve(A, np.ones(n_lu, complex))
    t_lu = time.perf_counter() - t0
    N = 2 * m.ne
    x = np.zeros((1, N), complex)
    obs = np.array([[0.3, 0.0], [1.0, 0.0]])
    t0 = time.perf_counter()
    farfield.rcs(m, x, obs)
    t_ff = time.perf_counter() - t0
    est = t_mesh + t_rows / nrows * m.ne + t_lu * (N / n_lu) ** 3 + t_ff / len(obs) * 361
    sample = (f"oracle on host: {nrows} dense JMCFIE edge rows of {m.ne} ({t_rows:.1f} s), dense LU n={n_lu} "
              f"({t_lu:.2f} s, scaled by N^3 to N={N}), far field at {len(obs)} of 361 angles; extrapolated")
    return est, sample, t_mesh + t_rows + t_lu + t_ff, N


def arm_config(unknowns, ws):
    """The workload keys both arms report."""
    return {"workload": WORKLOAD, "unknowns": unknowns, "levels": LEVELS, "digits": DIGITS, "tol": TOL,
            "restart": RESTART, "nrhs_per_gpu": 1, "parallelism": f"replicas{ws}"}


def oracle_c1_full():
    """The oracle end to end, nothing extrapolated, on the small workload it
    can finish (homogeneous sphere, 3 840 unknowns): dense JMCFIE fill, dense
    LU, bistatic RCS at 361 angles."""
    from oracle import farfield, fill, solvers
    from oracle.rwg import Mesh
    from paper_1704_06862_gb300 import geometry as geo
    t0 = time.perf_counter()
    m = Mesh(**geo.workload("sphere_c1"))
    Z = fill.assemble(m)
    t1 = time.perf_counter()
    x = solvers.lu_solve(Z, fill.rhs(m, [[0.0, 0.0, 0.0, 1.0]])[0])
    t2 = time.perf_counter()
    farfield.rcs(m, x[None], geo.bistatic_angles(361))
    t3 = time.perf_counter()
    return {"workload": "sphere_c1", "unknowns": 2 * m.ne, "s_to_rcs": t3 - t0, "fill_s": t1 - t0, "lu_s": t2 - t1,
            "rcs_s": t3 - t2, "cores": os.cpu_count()}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    from paper_1704_06862_gb300 import geometry as geo
    mesh = geo.workload(WORKLOAD)
    vals = []
    for i in range(args.warmup + args.steps):
        est, sample, spent, unknowns = oracle_sample(mesh, rng_seed=i, nrows=2)
        if i >= args.warmup:
            vals.append(est)
    v = float(np.mean(vals))
    c1 = None if args.no_c1 else oracle_c1_full()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config(unknowns, ws),
            "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "sample": sample, "value": v, "unit": "s"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "oracle_c1_end_to_end": c1}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-nn", action="store_true")
    ap.add_argument("--batch", type=int, default=16, help="right-hand sides of the batched monostatic leg")
    ap.add_argument("--no-graphs", action="store_true", help="launch every Krylov step eagerly (for profilers)")
    ap.add_argument("--no-solvers", action="store_true", help="skip the solver comparison leg")
    ap.add_argument("--no-forms", action="store_true", help="skip the formulation comparison leg")
    ap.add_argument("--no-nano", action="store_true", help="skip the plasmonic nanoparticle leg")
    ap.add_argument("--no-mie-refinement", action="store_true", help="skip the RCS-vs-Mie mesh refinement leg")
    ap.add_argument("--cube-sweep", type=int, default=256,
                    help="incidences of the cube's monostatic sweep (0: skip the leg)")
    ap.add_argument("--cube-block", type=int, default=64, help="right-hand sides per block of the cube sweep")
    ap.add_argument("--tuning-file", default=None, help="where the cube leg's autotuner writes its choice (JSON)")
    ap.add_argument("--no-c1", action="store_true",
                    help="skip the small homogeneous-sphere leg (GPU arm) / its full oracle run (reference arm)")
    ap.add_argument("--ellipsoid", action="store_true",
                    help="add the ellipsoid leg (355 488 unknowns, learned preconditioner on 32 incidences)")
    ap.add_argument("--lens", action="store_true",
                    help="add the lens-on-slab leg (1 189 264 unknowns, junction edges): one incidence in the "
                         "mixed and the plain FP64 forms, a monostatic sweep in blocks, the learned preconditioner")
    ap.add_argument("--lens-sweep", type=int, default=64, help="incidences of the lens's monostatic sweep (0: skip)")
    ap.add_argument("--lens-block", type=int, default=16, help="right-hand sides per block of the lens sweep")
    ap.add_argument("--formulation-study", action="store_true",
                    help="add the iterations-versus-unknowns study of the formulations on the two-layer sphere")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    import torch.distributed as dist

    import __graft_entry__ as g
    g.build()
    import paper_1704_06862_gb300 as sie
    from paper_1704_06862_gb300 import geometry as geo

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    mesh = geo.workload(WORKLOAD)
    t0 = time.perf_counter()
    s = sie.Solver(mesh, levels=LEVELS, digits=DIGITS, stream=stream)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    ne = s.ne
    obs = geo.bistatic_angles(361)
    # each rank its own incidence (replicas)
    inc = rank_incidence(rank)
    theta_i = float(inc[0, 0])
    b_dev = s.vec(1)
    x = s.vec(1)
    sie.sie_plane_wave_rhs(s.ctx, inc, b_dev)

    def solve(prec, e2e, precond=1):
        if e2e:                       # host incidence -> device excitation
            sie.sie_plane_wave_rhs(s.ctx, inc, b_dev)
        x.zero_()
        st = sie.gmres_solve(s.ctx, b_dev, x, 1, restart=RESTART, max_iters=3000, tol=TOL, prec=prec,
                             precond=precond, check=False, graphs=not args.no_graphs)
        rcs = sie.rcs_farfield_prec(s.ctx, x, 1, obs, prec)  # device -> host
        return st[0], rcs

    def timed(prec, steps, e2e, precond=1):
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = None
        for _ in range(steps):
            out = solve(prec, e2e, precond)
        e1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        ms = e0.elapsed_time(e1) / steps
        if ws > 1:
            ms = max_over_ranks(ms, dist, "cuda")
        return ms, out

    for _ in range(args.warmup):
        solve(sie.SIE_PREC_MIXED, False)
    launches0 = sie.sie_query(s.ctx, 8)
    clk = Clocks(local)
    clk.start()
    ms, (st, rcs) = timed(sie.SIE_PREC_MIXED, args.steps, False)
    clocks = clk.stop()
    launches = (sie.sie_query(s.ctx, 8) - launches0) // args.steps
    ms_e2e, _ = timed(sie.SIE_PREC_MIXED, 1, True)
    # the chosen form's currents against the whole FP64 operator (outside the timed region)
    y64 = s.vec(1)
    sie.mlfmm_matvec(s.ctx, x, y64, 1, sie.SIE_PREC_FP64)
    fp64_resid = float(torch.linalg.vector_norm(b_dev - y64) / torch.linalg.vector_norm(b_dev))
    del y64
    plain = None
    if not args.no_plain:
        ms64, (st64, rcs64) = timed(sie.SIE_PREC_FP64, 1, False)
        db = 10 * np.log10(np.maximum(rcs[:, :, 0], 1e-30)) - 10 * np.log10(np.maximum(rcs64[:, :, 0], 1e-30))
        plain = {"ms_per_solve": ms64, "iters": st64["iters"], "rel_residual": st64["rel_residual"],
                 "speedup_chosen_vs_plain": ms64 / ms, "rcs_max_abs_db_diff_vs_plain": float(np.max(np.abs(db)))}
    # learned preconditioner: trained on solver-recorded pairs of seeded random incidences
    learned = None
    if not args.no_nn:
        rng = np.random.default_rng(2017)
        nt = 8
        train = np.stack([np.arccos(rng.uniform(-1, 1, nt)), rng.uniform(0, 2 * np.pi, nt), np.zeros(nt),
                          np.ones(nt)], axis=1)
        tst = sie.nnprec_train(s.ctx, train, record_restart=5, max_pairs=96, epochs=12, batch=4096, lr=1e-3, seed=7)
        solve(sie.SIE_PREC_MIXED, False, 2)
        ms_nn, (st_nn, rcs_nn) = timed(sie.SIE_PREC_MIXED, args.steps, False, 2)
        dbn = 10 * np.log10(np.maximum(rcs_nn[:, :, 0], 1e-30)) - 10 * np.log10(np.maximum(rcs[:, :, 0], 1e-30))
        learned = {"train": tst, "ms_per_solve": ms_nn, "iters": st_nn["iters"], "rel_residual": st_nn["rel_residual"],
                   "converged": st_nn["converged"],
                   "ilu_only_ms_per_solve": ms, "ilu_only_iters": st["iters"], "speedup_vs_ilu_only": ms / ms_nn,
                   "rcs_max_abs_db_diff_vs_ilu_only": float(np.max(np.abs(dbn)))}
    # batched monostatic sweep: nb incidence angles theta in [0, 180] deg (phi = 0, theta-pol)
    # solved as one block of right-hand sides (block-RHS products and ILU sweeps)
    batched = None
    if args.batch > 1:
        nb = args.batch
        incb = geo.monostatic_incidences(nb)
        bb = s.vec(nb)
        xb = s.vec(nb)

        def solve_b():
            sie.sie_plane_wave_rhs(s.ctx, incb, bb)
            xb.zero_()
            stb = sie.gmres_solve(s.ctx, bb, xb, nb, restart=RESTART, max_iters=3000, tol=TOL,
                                  prec=sie.SIE_PREC_MIXED, precond=1, check=False,
                                  graphs=not args.no_graphs)
            obs_b = np.stack([incb[:, 0], incb[:, 1]], axis=1)
            mono = sie.rcs_farfield_prec(s.ctx, xb, nb, obs_b, sie.SIE_PREC_MIXED)
            return stb, mono[np.arange(nb), np.arange(nb), 0]

        solve_b()
        torch.cuda.synchronize()
        eb0 = torch.cuda.Event(enable_timing=True)
        eb1 = torch.cuda.Event(enable_timing=True)
        eb0.record(stream)
        stb, mono = solve_b()
        eb1.record(stream)
        torch.cuda.synchronize()
        msb = eb0.elapsed_time(eb1)
        batched = {"nrhs": nb, "ms_per_block": msb, "rhs_per_s": nb / (msb / 1e3),
                   "ms_per_rhs": msb / nb, "single_rhs_ms": ms, "speedup_per_rhs_vs_single": ms / (msb / nb),
                   "iters_max": max(t["iters"] for t in stb), "all_converged": all(t["converged"] for t in stb),
                   "monostatic_rcs_dbsm": [round(float(10 * np.log10(v)), 3) for v in mono]}
        del bb, xb
    # the paper's solver comparison on the same operator (mixed form): FGMRES(50),
    # BiCGStab and CGS, with ILU(0) and without a preconditioner
    solvers_cmp = None
    if not args.no_solvers:
        solvers_cmp = {}
        for label, method, pc in (("fgmres_ilu", 0, 1), ("bicgstab_ilu", 1, 1), ("cgs_ilu", 2, 1),
                                  ("fgmres_none", 0, 0), ("bicgstab_none", 1, 0)):
            def one():
                x.zero_()
                stc = sie.gmres_solve(s.ctx, b_dev, x, 1, restart=RESTART, max_iters=3000, tol=TOL,
                                      prec=sie.SIE_PREC_MIXED, precond=pc, check=False, method=method,
                                      graphs=not args.no_graphs)
                return stc[0], sie.rcs_farfield_prec(s.ctx, x, 1, obs, sie.SIE_PREC_MIXED)
            one()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stc, rcsc = one()
            e1.record(stream)
            torch.cuda.synchronize()
            dbc = 10 * np.log10(np.maximum(rcsc[:, :, 0], 1e-30)) - 10 * np.log10(np.maximum(rcs[:, :, 0], 1e-30))
            solvers_cmp[label] = {"ms_to_rcs": e0.elapsed_time(e1), "iters": stc["iters"],
                                  "products": stc["iters"] * (1 if method == 0 else 2),
                                  "converged": stc["converged"], "rel_residual": stc["rel_residual"],
                                  "rcs_max_abs_db_vs_chosen": float(np.max(np.abs(dbc)))}
    # Mie check of the chosen form
    # (stored Mie series of the coated sphere, written by tests/golden/make_golden.py)
    mie_db = None
    mie_ref = None
    mie_path = os.path.join(ROOT, "tests", "golden", "mie_coated_c2.npz")
    if theta_i == 0.0 and os.path.exists(mie_path):
        mie_ref = np.load(mie_path)["mie"]
        d = 10 * np.log10(rcs[0, :, 0]) - 10 * np.log10(mie_ref)
        mie_db = {"mean_abs_db": float(np.mean(np.abs(d))), "max_abs_db": float(np.max(np.abs(d)))}
    # the formulations the paper compares JMCFIE with, on the same mesh and tree
    # (each its own context: fill, patterns and ILU(0) of that formulation)
    forms_cmp = None
    if not args.no_forms:
        forms_cmp = {"jmcfie": {"ms_to_rcs": ms, "iters": st["iters"], "converged": st["converged"],
                                "rcs_vs_mie_mean_db": mie_db["mean_abs_db"] if mie_db else None}}
        for fname, form in (("ctf", sie.FORM_CTF), ("cnf", sie.FORM_CNF), ("pmchwt", sie.FORM_PMCHWT),
                            ("ictf", sie.FORM_ICTF)):
            sf = sie.Solver(mesh, levels=LEVELS, digits=DIGITS, stream=stream, formulation=form)
            bf = sf.vec(1)
            xf = sf.vec(1)
            sie.sie_plane_wave_rhs(sf.ctx, inc, bf)

            def one():
                xf.zero_()
                stf = sie.gmres_solve(sf.ctx, bf, xf, 1, restart=RESTART, max_iters=1000, tol=TOL,
                                      prec=sie.SIE_PREC_MIXED, precond=1, check=False, graphs=not args.no_graphs)
                return stf[0], sie.rcs_farfield_prec(sf.ctx, xf, 1, obs, sie.SIE_PREC_MIXED)
            one()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stf, rcsf = one()
            e1.record(stream)
            torch.cuda.synchronize()
            row = {"ms_to_rcs": e0.elapsed_time(e1), "iters": stf["iters"], "converged": stf["converged"],
                   "rel_residual": stf["rel_residual"], "rcs_vs_mie_mean_db": None}
            if mie_ref is not None:
                row["rcs_vs_mie_mean_db"] = float(np.mean(np.abs(10 * np.log10(rcsf[0, :, 0]) - 10 * np.log10(mie_ref))))
            forms_cmp[fname] = row
            del bf, xf
            sf.close()

    # plasmonic coated nanoparticle (negative-permittivity, lossy media; its own
    # mesh and tree): time to RCS with ILU(0) FGMRES(50) and BiCGStab in the mixed
    # form, and FGMRES(50) in the plain FP64 form
    nano = None
    if not args.no_nano:
        t0 = time.perf_counter()
        sn = sie.Solver(geo.workload("nanoparticle"), levels=NANO_LEVELS, digits=DIGITS, stream=stream)
        torch.cuda.synchronize()
        nano = {"unknowns": 2 * sn.ne, "levels": NANO_LEVELS, "setup_s": time.perf_counter() - t0}
        bn = sn.vec(1)
        xn = sn.vec(1)
        sie.sie_plane_wave_rhs(sn.ctx, inc, bn)
        nano_path = os.path.join(ROOT, "tests", "golden", "nanoparticle.npz")
        mie_n = np.load(nano_path)["mie"] if theta_i == 0.0 and os.path.exists(nano_path) else None
        for label, method, pr in (("fgmres_ilu", 0, sie.SIE_PREC_MIXED), ("bicgstab_ilu", 1, sie.SIE_PREC_MIXED),
                                  ("fgmres_ilu_plain_fp64", 0, sie.SIE_PREC_FP64)):
            def one():
                xn.zero_()
                stn = sie.gmres_solve(sn.ctx, bn, xn, 1, restart=RESTART, max_iters=3000, tol=TOL,
                                      prec=pr, precond=1, check=False, method=method,
                                      graphs=not args.no_graphs)
                return stn[0], sie.rcs_farfield_prec(sn.ctx, xn, 1, obs, pr)
            one()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stn, rcsn = one()
            e1.record(stream)
            torch.cuda.synchronize()
            row = {"ms_to_rcs": e0.elapsed_time(e1), "iters": stn["iters"], "converged": stn["converged"],
                   "rel_residual": stn["rel_residual"], "rcs_vs_mie_mean_db": None, "rcs_vs_mie_max_db": None}
            if mie_n is not None:
                dn = np.abs(10 * np.log10(rcsn[0, :, 0]) - 10 * np.log10(mie_n))
                row["rcs_vs_mie_mean_db"] = float(dn.mean())
                row["rcs_vs_mie_max_db"] = float(dn.max())
            nano[label] = row
        nano["matvec_fp32_ms"] = sie.sie_stage_timing(sn.ctx, 3, 1, sie.SIE_PREC_MIXED, 20)
        del bn, xn
        sn.close()

    # the small homogeneous-sphere workload (3 840 unknowns) end to end on the
    # GPU, beside the oracle's end-to-end time on the same case (reference arm)
    c1 = None
    if not args.no_c1:
        t0 = time.perf_counter()
        s1 = sie.Solver(geo.workload("sphere_c1"), levels=3, digits=DIGITS, stream=stream)
        torch.cuda.synchronize()
        c1 = {"workload": "sphere_c1", "unknowns": 2 * s1.ne, "levels": 3, "setup_s": time.perf_counter() - t0}
        b1 = s1.vec(1)
        x1 = s1.vec(1)
        for rep in range(2):                     # the first solve captures the step graphs
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sie.sie_plane_wave_rhs(s1.ctx, inc, b1)
            x1.zero_()
            st1 = sie.gmres_solve(s1.ctx, b1, x1, 1, restart=RESTART, max_iters=3000, tol=TOL,
                                  prec=sie.SIE_PREC_MIXED, precond=1, check=False, graphs=not args.no_graphs)[0]
            sie.rcs_farfield_prec(s1.ctx, x1, 1, obs, sie.SIE_PREC_MIXED)
            e1.record(stream)
            torch.cuda.synchronize()
        c1.update({"ms_to_rcs": e0.elapsed_time(e1), "iters": st1["iters"], "converged": st1["converged"]})
        del b1, x1
        s1.close()

    # RCS against the Mie series under mesh refinement (the discretisation error
    # of the flat-facet RWG model falls as h^2): the homogeneous sphere of the
    # small workload and the two-layer sphere at finer meshes than the timed one;
    # mixed form, ILU(0) FGMRES(50) to 1e-4, all 361 angles (nulls included)
    mie_ref = None
    if not args.no_mie_refinement and theta_i == 0.0:
        # Mie series at the same 361 angles, stored by tests/golden/make_golden.py
        mie_sph = np.load(os.path.join(ROOT, "tests", "golden", "sphere_c1.npz"))["mie"]
        mie_coat = np.load(os.path.join(ROOT, "tests", "golden", "mie_coated_c2.npz"))["mie"]
        mie_ref = {"solver": "mixed form, ILU(0) FGMRES(50), tol 1e-4; |dB error| over 361 phi=0 angles",
                   "rows": []}
        cases = [("sphere", 8, None, 3), ("sphere", 16, None, 4), ("coated", 30, 20, LEVELS),
                 ("coated", 36, 24, LEVELS), ("coated", 42, 28, LEVELS)]
        for kind, nu_o, nu_i, lv in cases:
            if kind == "sphere":
                mesh_r = geo.homogeneous_sphere(nu=nu_o, radius=0.5, eps_r=4.0)
                ref_r = mie_sph
            else:
                mesh_r = geo.coated_sphere(nu_o, nu_i)
                ref_r = mie_coat
            t0 = time.perf_counter()
            sr = sie.Solver(mesh_r, levels=lv, digits=DIGITS, stream=stream)
            torch.cuda.synchronize()
            t_set = time.perf_counter() - t0
            br = sr.vec(1)
            xr = sr.vec(1)
            sie.sie_plane_wave_rhs(sr.ctx, inc, br)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            str_ = sie.gmres_solve(sr.ctx, br, xr, 1, restart=RESTART, max_iters=3000, tol=TOL,
                                   prec=sie.SIE_PREC_MIXED, precond=1, check=False, graphs=not args.no_graphs)[0]
            rr = sie.rcs_farfield_prec(sr.ctx, xr, 1, obs, sie.SIE_PREC_MIXED)
            e1.record(stream)
            torch.cuda.synchronize()
            dd = np.abs(10 * np.log10(rr[0, :, 0]) - 10 * np.log10(ref_r))
            mie_ref["rows"].append({"body": kind, "nu_outer": nu_o, "nu_inner": nu_i, "unknowns": 2 * sr.ne,
                                    "levels": lv, "iters": str_["iters"], "converged": str_["converged"],
                                    "setup_s": t_set, "ms_to_rcs": e0.elapsed_time(e1),
                                    "mean_abs_db": float(dd.mean()), "max_abs_db": float(dd.max())})
            del br, xr
            sr.close()

    # monostatic RCS sweep of the lossy dielectric cube (3 lambda0, eps 6 - 0.6j,
    # 104 976 unknowns): the incidences solved as blocks of right-hand sides
    # (block products, block ILU sweeps, FGMRES in lockstep), mixed form,
    # ILU(0) FGMRES(50) to 1e-4, theta-theta RCS of each incidence
    cube = None
    if args.cube_sweep > 0:
        t0 = time.perf_counter()
        sc = sie.Solver(geo.workload("cube_c3"), levels=LEVELS, digits=DIGITS, stream=stream)
        torch.cuda.synchronize()
        cube = {"workload": "cube_c3", "unknowns": 2 * sc.ne, "levels": LEVELS, "incidences": args.cube_sweep,
                "block": args.cube_block, "setup_s": time.perf_counter() - t0}
        inc_c = geo.monostatic_incidences(args.cube_sweep)
        B = min(args.cube_block, args.cube_sweep)
        # tile shapes of the block kernels for this block size, chosen by the autotuner
        far_default = sie.sie_stage_timing(sc.ctx, 1, B, sie.SIE_PREC_MIXED, 3)
        cube["tuning"] = sie.sie_autotune(sc.ctx, B, reps=2, path=args.tuning_file)
        cube["far_ms_per_block_default_tiles"] = far_default
        bc = sc.vec(B)
        xc = sc.vec(B)
        # untimed: work buffers of the block size and the first captured steps
        sie.sie_plane_wave_rhs(sc.ctx, inc_c[:B], bc)
        sie.gmres_solve(sc.ctx, bc, xc, B, restart=RESTART, max_iters=2, tol=TOL, prec=sie.SIE_PREC_MIXED,
                        precond=1, check=False, graphs=not args.no_graphs)
        torch.cuda.synchronize()
        mono_c = np.zeros(args.cube_sweep)
        iters_c = []
        conv_c = True
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i0 in range(0, args.cube_sweep, B):
            nb_ = min(B, args.cube_sweep - i0)
            sie.sie_plane_wave_rhs(sc.ctx, inc_c[i0:i0 + nb_], bc[:nb_])
            xc.zero_()
            stc = sie.gmres_solve(sc.ctx, bc[:nb_], xc[:nb_], nb_, restart=RESTART, max_iters=3000, tol=TOL,
                                  prec=sie.SIE_PREC_MIXED, precond=1, check=False, graphs=not args.no_graphs)
            obs_c = np.stack([inc_c[i0:i0 + nb_, 0], inc_c[i0:i0 + nb_, 1]], axis=1)
            rc = sie.rcs_farfield_prec(sc.ctx, xc[:nb_], nb_, obs_c, sie.SIE_PREC_MIXED)
            mono_c[i0:i0 + nb_] = rc[np.arange(nb_), np.arange(nb_), 0]
            iters_c += [t["iters"] for t in stc]
            conv_c = conv_c and all(t["converged"] for t in stc)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_c = e0.elapsed_time(e1)
        db_c = 10 * np.log10(mono_c)
        cube.update({"ms_sweep": ms_c, "rhs_per_s": args.cube_sweep / (ms_c / 1e3),
                     "ms_per_rhs": ms_c / args.cube_sweep, "iters_max": max(iters_c), "iters_mean": float(np.mean(iters_c)),
                     "all_converged": conv_c, "mirror_symmetry_max_db": float(np.max(np.abs(db_c - db_c[::-1]))),
                     "far_ms_per_rhs_at_block": sie.sie_stage_timing(sc.ctx, 1, B, sie.SIE_PREC_MIXED, 3) / B,
                     "far_ms_per_rhs_single": sie.sie_stage_timing(sc.ctx, 1, 1, sie.SIE_PREC_MIXED, 10),
                     "monostatic_rcs_dbsm": [round(float(v), 3) for v in db_c]})
        del bc, xc
        sc.close()

    # lossy dielectric ellipsoid (semi-axes 4 x 2 x 1 lambda0, eps 3 - 0.2j,
    # 355 488 unknowns, 7 levels): the learned preconditioner trained on
    # solver-generated pairs of 32 random incidences (uniform on the sphere,
    # seed 2017), then ILU(0) FGMRES against ILU(0) + network FGMRES on held-out
    # incidences (seed 2018), mixed form, tol 1e-4
    ell = None
    if args.ellipsoid:
        t0 = time.perf_counter()
        se = sie.Solver(geo.workload("ellipsoid_c4"), levels=7, digits=DIGITS, stream=stream)
        torch.cuda.synchronize()
        ell = {"workload": "ellipsoid_c4", "unknowns": 2 * se.ne, "levels": 7, "setup_s": time.perf_counter() - t0}

        def uniform_incidences(n, seed):
            rng = np.random.default_rng(seed)
            return np.stack([np.arccos(rng.uniform(-1, 1, n)), rng.uniform(0, 2 * np.pi, n), np.zeros(n),
                             np.ones(n)], axis=1)

        ell["train"] = sie.nnprec_train(se.ctx, uniform_incidences(32, 2017), record_restart=5, max_pairs=256,
                                        epochs=12, batch=4096, lr=1e-3, seed=7)
        test_inc = uniform_incidences(4, 2018)
        be = se.vec(1)
        xe = se.vec(1)
        rows = []
        for i in range(len(test_inc)):
            sie.sie_plane_wave_rhs(se.ctx, test_inc[i:i + 1], be)
            row = {"theta": float(test_inc[i, 0]), "phi": float(test_inc[i, 1])}
            for label, pc in (("ilu", 1), ("ilu_nn", 2)):
                if pc == 2 and not ell["train"]["enabled"]:
                    continue
                xe.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ste = sie.gmres_solve(se.ctx, be, xe, 1, restart=RESTART, max_iters=3000, tol=TOL,
                                      prec=sie.SIE_PREC_MIXED, precond=pc, check=False, graphs=not args.no_graphs)[0]
                e1.record(stream)
                torch.cuda.synchronize()
                row[label] = {"iters": ste["iters"], "converged": ste["converged"], "ms": e0.elapsed_time(e1)}
            rows.append(row)
        ell["held_out"] = rows
        ell["far_ms"] = sie.sie_stage_timing(se.ctx, 1, 1, sie.SIE_PREC_MIXED, 5)
        ell["matvec_ms"] = sie.sie_stage_timing(se.ctx, 3, 1, sie.SIE_PREC_MIXED, 5)
        ell["ilu_ms"] = sie.sie_stage_timing(se.ctx, 2, 1, sie.SIE_PREC_MIXED, 5)
        del be, xe
        se.close()

    # three-layer hemispherical lens (radii 1.5 / 3 / 6 lambda0, eps 10.2 / 4.5
    # / 2.2) on a 14 x 14 x 0.5 lambda0 slab of eps 2.2 (Eq. 16's multilayer
    # body, five media, junction edges on the three base circles; 1 189 264
    # unknowns, 7 levels): setup, one normal incidence to RCS, mixed form, ILU(0)
    # FGMRES(50), tol 1e-4, and the stage times of one product and one ILU apply;
    # the same incidence in the plain FP64 form (its RCS the check of the mixed
    # one); a monostatic sweep (theta_i uniform in [0, 180] degrees, phi = 0) in
    # blocks of right-hand sides; the learned preconditioner trained on 8
    # incidences (uniform on the sphere, seed 2017), one held out (seed 2018)
    lens = None
    if args.lens:
        t0 = time.perf_counter()
        g = geo.workload("lens_c5")
        t_mesh = time.perf_counter() - t0
        sl = sie.Solver(g, levels=7, digits=DIGITS, stream=stream)
        torch.cuda.synchronize()
        lens = {"workload": "lens_c5", "unknowns": 2 * sl.ne, "triangles": int(len(g["tris"])), "levels": 7,
                "mesh_s": t_mesh, "setup_s": time.perf_counter() - t0 - t_mesh,
                "device_bytes": sie.sie_query(sl.ctx, 7), "near_blocks": sie.sie_query(sl.ctx, 1)}
        del g
        bl = sl.vec(1)
        xl = sl.vec(1)
        sie.sie_plane_wave_rhs(sl.ctx, [[0.0, 0.0, 0.0, 1.0]], bl)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stl = sie.gmres_solve(sl.ctx, bl, xl, 1, restart=RESTART, max_iters=3000, tol=TOL,
                              prec=sie.SIE_PREC_MIXED, precond=1, check=False, graphs=not args.no_graphs)[0]
        rl = sie.rcs_farfield(sl.ctx, xl, 1, geo.bistatic_angles(361))
        e1.record(stream)
        torch.cuda.synchronize()
        lens.update(iters=stl["iters"], converged=stl["converged"], rel_residual=stl["rel_residual"],
                    ms_to_rcs=e0.elapsed_time(e1), rcs_finite=bool(np.isfinite(rl).all()))
        lens["far_ms"] = sie.sie_stage_timing(sl.ctx, 1, 1, sie.SIE_PREC_MIXED, 5)
        lens["matvec_ms"] = sie.sie_stage_timing(sl.ctx, 3, 1, sie.SIE_PREC_MIXED, 5)
        lens["ilu_ms"] = sie.sie_stage_timing(sl.ctx, 2, 1, sie.SIE_PREC_MIXED, 5)
        lens["far_fp64_ms"] = sie.sie_stage_timing(sl.ctx, 1, 1, sie.SIE_PREC_FP64, 2)
        # plain FP64 form of the same incidence: its RCS is the mixed form's check
        xl.zero_()
        e0.record(stream)
        st64 = sie.gmres_solve(sl.ctx, bl, xl, 1, restart=RESTART, max_iters=3000, tol=TOL,
                               prec=sie.SIE_PREC_FP64, precond=1, check=False, graphs=not args.no_graphs)[0]
        r64 = sie.rcs_farfield(sl.ctx, xl, 1, geo.bistatic_angles(361))
        e1.record(stream)
        torch.cuda.synchronize()
        ok = r64[0, :, 0] > r64[0, :, 0].max() * 1e-3
        dbl = np.abs(10 * np.log10(rl[0, ok, 0]) - 10 * np.log10(r64[0, ok, 0]))
        lens["fp64"] = {"iters": st64["iters"], "converged": st64["converged"], "ms_to_rcs": e0.elapsed_time(e1)}
        lens.update(rcs_vs_fp64_mean_db=float(dbl.mean()), rcs_vs_fp64_max_db=float(dbl.max()))
        del bl, xl
        if args.lens_sweep > 0:
            inc_l = geo.monostatic_incidences(args.lens_sweep)
            B = min(args.lens_block, args.lens_sweep)
            bs = sl.vec(B)
            xs = sl.vec(B)
            sie.sie_plane_wave_rhs(sl.ctx, inc_l[:B], bs)      # untimed: work buffers of the block size
            sie.gmres_solve(sl.ctx, bs, xs, B, restart=RESTART, max_iters=2, tol=TOL, prec=sie.SIE_PREC_MIXED,
                            precond=1, check=False, graphs=not args.no_graphs)
            torch.cuda.synchronize()
            mono_l = np.zeros(args.lens_sweep)
            iters_l, conv_l = [], True
            e0.record(stream)
            for i0 in range(0, args.lens_sweep, B):
                nb_ = min(B, args.lens_sweep - i0)
                sie.sie_plane_wave_rhs(sl.ctx, inc_l[i0:i0 + nb_], bs[:nb_])
                xs.zero_()
                stb = sie.gmres_solve(sl.ctx, bs[:nb_], xs[:nb_], nb_, restart=RESTART, max_iters=3000, tol=TOL,
                                      prec=sie.SIE_PREC_MIXED, precond=1, check=False, graphs=not args.no_graphs)
                obs_l = np.stack([inc_l[i0:i0 + nb_, 0], inc_l[i0:i0 + nb_, 1]], axis=1)
                rb = sie.rcs_farfield_prec(sl.ctx, xs[:nb_], nb_, obs_l, sie.SIE_PREC_MIXED)
                mono_l[i0:i0 + nb_] = rb[np.arange(nb_), np.arange(nb_), 0]
                iters_l += [t["iters"] for t in stb]
                conv_l = conv_l and all(t["converged"] for t in stb)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_l = e0.elapsed_time(e1)
            lens["sweep"] = {"incidences": args.lens_sweep, "block": B, "ms_sweep": ms_l,
                             "rhs_per_s": args.lens_sweep / (ms_l / 1e3), "ms_per_rhs": ms_l / args.lens_sweep,
                             "iters_mean": float(np.mean(iters_l)), "iters_max": max(iters_l),
                             "all_converged": conv_l, "device_bytes": sie.sie_query(sl.ctx, 7),
                             "monostatic_rcs_dbsm": [round(float(v), 3) for v in 10 * np.log10(mono_l)]}
            del bs, xs

        def uniform_incidences_l(n, seed):
            rng = np.random.default_rng(seed)
            return np.stack([np.arccos(rng.uniform(-1, 1, n)), rng.uniform(0, 2 * np.pi, n), np.zeros(n),
                             np.ones(n)], axis=1)

        try:
            lens["train"] = sie.nnprec_train(sl.ctx, uniform_incidences_l(8, 2017), record_restart=5, max_pairs=256,
                                             epochs=12, batch=4096, lr=1e-3, seed=7)
        except sie.SieError as e:            # reported in the line, the rest of the bench still runs
            lens["train"] = {"enabled": False, "error": str(e)}
        bh = sl.vec(1)
        xh = sl.vec(1)
        sie.sie_plane_wave_rhs(sl.ctx, uniform_incidences_l(1, 2018), bh)
        held = {}
        for label, pc in (("ilu", 1), ("ilu_nn", 2)):
            if pc == 2 and not lens["train"]["enabled"]:
                continue
            xh.zero_()
            e0.record(stream)
            sth = sie.gmres_solve(sl.ctx, bh, xh, 1, restart=RESTART, max_iters=3000, tol=TOL,
                                  prec=sie.SIE_PREC_MIXED, precond=pc, check=False, graphs=not args.no_graphs)[0]
            e1.record(stream)
            torch.cuda.synchronize()
            held[label] = {"iters": sth["iters"], "converged": sth["converged"], "ms": e0.elapsed_time(e1)}
        lens["held_out"] = held
        del bh, xh
        sl.close()

    # iterations versus unknowns per formulation (the comparison of Fig. 6) on the
    # two-layer sphere at four mesh densities: FGMRES(50) with ILU(0) and without
    # a preconditioner, mixed form, tol 1e-4, at most 1000 iterations
    study = None
    if args.formulation_study:
        study = {"solver": "FGMRES(50), ILU(0) ('ilu') or none ('none'), mixed form, tol 1e-4, max 1000 iterations",
                 "rows": []}
        for nu_o, nu_i in ((12, 8), (18, 12), (24, 16), (30, 20)):
            mesh_s = geo.coated_sphere(nu_o, nu_i)
            row = {"nu_outer": nu_o, "nu_inner": nu_i}
            for fname, form in (("jmcfie", sie.FORM_JMCFIE), ("ctf", sie.FORM_CTF), ("cnf", sie.FORM_CNF),
                                ("pmchwt", sie.FORM_PMCHWT), ("ictf", sie.FORM_ICTF)):
                sf = sie.Solver(mesh_s, levels=LEVELS, digits=DIGITS, stream=stream, formulation=form)
                row["unknowns"] = 2 * sf.ne
                bf = sf.vec(1)
                xf = sf.vec(1)
                sie.sie_plane_wave_rhs(sf.ctx, inc, bf)
                row[fname] = {}
                for pname, pc in (("ilu", 1), ("none", 0)):
                    xf.zero_()
                    stf = sie.gmres_solve(sf.ctx, bf, xf, 1, restart=RESTART, max_iters=1000, tol=TOL,
                                          prec=sie.SIE_PREC_MIXED, precond=pc, check=False,
                                          graphs=not args.no_graphs)
                    row[fname][pname] = {"iters": stf[0]["iters"], "converged": stf[0]["converged"],
                                         "rel_residual": stf[0]["rel_residual"]}
                del bf, xf
                sf.close()
            study["rows"].append(row)

    # stage timings (CUDA events on the library stream) and the roofline of the dominant kernel
    graphs_state = sie.sie_query(s.ctx, 10)
    stages = {}
    for name, stg in (("near_spmv", 0), ("far_mlfmm", 1), ("ilu_sweeps", 2), ("matvec", 3)):
        stages[name] = {"fp32_ms": sie.sie_stage_timing(s.ctx, stg, 1, sie.SIE_PREC_MIXED, 20),
                        "fp64_ms": sie.sie_stage_timing(s.ctx, stg, 1, sie.SIE_PREC_FP64, 10)}
    # the same ILU(0) apply as one persistent cooperative launch (grid barriers between the steps)
    sie.sie_set_param(s.ctx, 1, 0)
    stages["ilu_sweeps_persistent"] = {
        "fp32_ms": sie.sie_stage_timing(s.ctx, 2, 1, sie.SIE_PREC_MIXED, 20),
        "fp64_ms": sie.sie_stage_timing(s.ctx, 2, 1, sie.SIE_PREC_FP64, 10)}
    sie.sie_set_param(s.ctx, 1, 1)
    sie.sie_device_status(s.ctx)
    # the far field with the M2L by sibling groups split over warps (the alternative form)
    sie.sie_set_param(s.ctx, 7, 2)
    stages["far_mlfmm_m2l_split_groups"] = {"fp32_ms": sie.sie_stage_timing(s.ctx, 1, 1, sie.SIE_PREC_MIXED, 20)}
    sie.sie_set_param(s.ctx, 7, -1)
    nnzb = sie.sie_query(s.ctx, 1)
    near_bytes_fp32 = nnzb * (4 * 8 + 4) + (ne + 1) * 4 + 2 * (2 * ne * 8)
    near_bytes_fp64 = nnzb * (4 * 16 + 4) + (ne + 1) * 4 + 2 * (2 * ne * 16)
    peak, peak_src = measured_peaks()
    # the kernel with the largest share of the solve's time: the ILU(0) sweeps
    # (one apply = 15 dependent k_ilu_sweep launches; bytes and time per apply)
    ilu_bytes = sie.sie_query(s.ctx, 9)
    ach_ilu = ilu_bytes / (stages["ilu_sweeps"]["fp32_ms"] * 1e-3) / 1e9
    roofline = {"kernel": "k_ilu_sweep<float, 512> (ILU(0) apply: 15 colour sweep steps)", "bound": "hbm",
                "achieved": ach_ilu, "peak": peak, "peak_source": peak_src, "unit": "GB/s", "frac": ach_ilu / peak,
                "traffic": ILU_APPLY_TRAFFIC_BYTES if WORKLOAD == "coated_c2" else None,
                "algorithmic_bytes_per_apply": ilu_bytes, "launches_per_apply": 15}
    ach = near_bytes_fp32 / (stages["near_spmv"]["fp32_ms"] * 1e-3) / 1e9
    roofline_near = {"kernel": "k_near_spmv<float> (near-field 2x2 block-sparse product)", "bound": "hbm",
                     "achieved": ach, "peak": peak, "peak_source": peak_src, "unit": "GB/s", "frac": ach / peak,
                     "traffic": NEAR_SPMV_TRAFFIC_BYTES if WORKLOAD == "coated_c2" else None,
                     "algorithmic_bytes_per_launch": near_bytes_fp32,
                     "fp64_achieved": near_bytes_fp64 / (stages["near_spmv"]["fp64_ms"] * 1e-3) / 1e9}
    pat_bytes = sie.sie_query(s.ctx, 6)
    mv_bytes32 = near_bytes_fp32 + pat_bytes // 2
    matvec = {"fp32_ms": stages["matvec"]["fp32_ms"], "fp64_ms": stages["matvec"]["fp64_ms"],
              "true_residual_product_ms": sie.sie_stage_timing(s.ctx, 3, 1, sie.SIE_PREC_NEAR64, 10),
              "fp32_algorithmic_GBs": mv_bytes32 / (stages["matvec"]["fp32_ms"] * 1e-3) / 1e9,
              "fp64_algorithmic_GBs": (near_bytes_fp64 + pat_bytes) / (stages["matvec"]["fp64_ms"] * 1e-3) / 1e9}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        est, sample, spent, _ = oracle_sample(mesh)
        cpu = {"value": est, "unit": "s", "cores": os.cpu_count(), "kind": "oracle", "sample": sample,
               "sample_wall_s": spent}
    line = {
        "metric": METRIC, "value": ms / 1e3 * 1.0, "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "precision": "FP32 complex operator, ILU(0) and RCS; FP64 Arnoldi, Givens and true-residual vectors, "
                     "true residual with the FP64 near field and the FP32 far field", "data": "synthetic",
        "config": dict(arm_config(2 * ne, ws),
                       l2=f"operator data {(near_bytes_fp32 + pat_bytes // 2) / 1e6:.0f} MB > 129 MB L2 (no flush)"),
        "iters": st["iters"], "rel_residual": st["rel_residual"], "fp64_operator_rel_residual": fp64_resid,
        "setup_s": t_setup,
        "e2e": {"value": ms_e2e / 1e3, "unit": "s", "h2d_bytes_per_step": int(inc.nbytes),
                "d2h_bytes_per_step": int(rcs.nbytes)},
        "plain_fp64": plain, "learned_precond": learned, "batched_monostatic": batched, "solvers": solvers_cmp, "formulations": forms_cmp,
        "nanoparticle": nano, "formulation_study": study, "rcs_vs_mie": mie_db, "mie_refinement": mie_ref, "sphere_c1": c1, "cube_monostatic": cube, "ellipsoid": ell, "lens": lens, "stages_ms": stages, "matvec": matvec,
        "roofline": roofline, "roofline_near_spmv": roofline_near, "cpu_baseline": cpu, "clocks": clocks, "gpu_launches": int(launches), "krylov_step_graphs": graphs_state,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
