"""Benchmark: IPCS steps/s of the GB300 path on a seeded synthetic workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload tg3d_64|tg2d_32|channel|stress128_rcm|stress128_random]

One "step" is one full IPCS time step (assembly + Algorithm 2, d-RHS BiCGStab,
pressure CG, normalisation, lumped update) on the device, every solve to the
same relative residual (1e-8).  Default workload: the unstructured-stress cube,
128^3 cells x 6 tetrahedra (2,146,689 dofs, 12,582,912 cells), interior vertices
jittered by up to 20 % of the spacing, dofs in reverse Cuthill-McKee order, 3D
Taylor-Green data; mixed precision, the three velocity components in one 3-RHS
solve, the multigrid-preconditioned pressure CG started from the learned guess,
the step captured in one CUDA graph.  Beside it: the same form with the previous
correction as the guess, the same form in float64, and the plain float64 form
(one solve per component, eager launches, Jacobi, zero guess).

Prints one JSON line.  Under torchrun (N > 1) every rank runs an independent
replica of the workload on its own GPU (the single-GPU method has no exchange
step); the whole-job value is the steps of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IPCS steps/s at matched residual, mixed+learned vs FP64; SpMV HBM GB/s"
RTOL = 1e-8


def workload(name, scalars=0):
    pb = _workload(name)
    if scalars:
        from workloads import problems as WP
        WP.with_scalars(pb, ns=scalars)
    return pb


def _workload(name):
    from workloads import problems as WP
    if name == "tg3d_64":
        return WP.taylor_green_3d(64, n_steps=200, rtol=RTOL)
    if name == "tg2d_32":
        return WP.taylor_green_2d(32)
    if name == "channel":
        return WP.channel()
    if name.startswith("stress"):
        # stress<n>[_<ordering>], e.g. stress128_rcm (the 128^3 configuration) or a smaller cube
        head, _, order = name.partition("_")
        return WP.stress_cube(int(head[len("stress"):] or 128), ordering=order or "natural")
    raise ValueError(name)


def workload_config(name, pb, precision, gpu=True):
    """The workload (and, for the GPU arm, the solver form) a line was measured on."""
    c = {"workload": name, "n_dofs": int(pb.mesh.n_dofs), "n_cells": int(pb.mesh.n_cells),
         "dt": pb.dt, "nu": pb.nu, "rtol": RTOL, "precision": precision}
    if gpu:
        c |= {"batch_rhs": True, "cuda_graph": True, "l2": "flushed between steps (256 MiB write)"}
    else:
        c |= {"solver": "scipy BiCGStab (velocity, one solve per component) and CG (pressure), Jacobi, "
                        "sparse matrices assembled per step, host cores"}
    return c


# ---------------------------------------------------------------------- rooflines
# DRAM bytes per launch of a family's kernel from an ncu capture (cold caches),
# per workload and layout, with the profile summary it comes from; valid for the
# kernels as they stand (an entry is removed when its kernel changes)
_S112 = "profiles/dram_traffic_products_stress112_rcm.md (stress112_rcm capture, scaled by algorithmic bytes)"
MEASURED_TRAFFIC = {("stress128_rcm", "pcg_spmv@sell"): (215.0e6, _S112),
                    ("stress128_rcm", "pcg_spmv@pairs"): (229.8e6, _S112),
                    ("stress128_rcm", "amg_fine@pairs"): (163.3e6, _S112),
                    ("stress128_rcm", "bicg_spmm@rows"): (332.4e6, _S112),
                    ("stress128_rcm", "bicg_spmm@rows16"): (263.6e6, _S112)}


def family_bytes(pb, nnz, args, tuning, amg):
    """Algorithmic bytes per launch of every timed kernel family (float32 values,
    int32 indices unless stated; N dofs, Z pattern entries, T cells, D dims; each
    array counted once per launch, gathered operands once per row):
      pcg_spmv     multigrid CG product w = K u on SELL-32 + 3 dots: K values and
                   columns (16-bit offsets where the mesh has them), u gathered, r read,
                   w written, slice pointers/lengths
      bicg_spmm    d-RHS product of the BiCGStab: A values + columns (int32, or 16-bit
                   offsets for a col16 shape), row pointers, x gathered, y written, the
                   dot operand read
      amg_fine     finest-level smoothing sweep (pre or post, SELL-32): K values as
                   bfloat16 + columns, 4 vectors of N, slice pointers/lengths
      amg_transfer restriction/prolongation (bfloat16 values), averaged over the 2(L-1)
                   launches of a V-cycle: per level 12 nnz(P) + 16 n_l + 12 n_(l+1) in CSR
                   form; 8 nnz(P) + 12.5 n_l + 8.5 n_(l+1) with both pair-packed (16-bit
                   offsets, 16-byte slice headers; 6 bytes per entry where a packed copy
                   keeps 32-bit columns)
      amg_coarse   coarser-level sweeps (bfloat16 values) and the dense coarsest product,
                   averaged over their 2(L-2)+1 launches: per sweep 6 nnz_l + 20 n_l (CSR)
                   or 4 nnz_l + 16.5 n_l (pair-packed); dense 4 nc ld + 8 nc
      bicg_vec     BiCGStab vector kernels, averaged over dir (64 N), s (52 N), and
                   the solution/residual update with its dots (96 N), for D = 3
      assemble     convecting velocity per dof (u^{n-1}, u^{n-2} read, ubar written: 60 N),
                   convection cell terms (80 T + 12 N) and the fused row pass (incidence and
                   cell terms 48 T, per entry 28 Z, per row 132 N), once per step
      outer        float64-quality residuals of the sweeps, averaged over the tentative
                   solve's (A + columns 8 Z; r0, Delta gathered, r, rh, p, v, dl: 112 N)
                   and the pressure's (K as float-float + columns 12 Z; 56 N)
      pcg_update   multigrid CG vector update: u, w, p, s, increment, r read, p, s,
                   increment, r written (40 N)
    Returns {family: (kernel, bytes per launch, formula)}."""
    N, Z, T, D = pb.mesh.n_dofs, nnz, pb.mesh.n_cells, pb.mesh.dim
    n_slices = (N + 31) // 32
    out = {}
    if amg:
        have16 = any(c["col16"] and c["us"] > 0 for c in tuning["candidates"])
        chosen = tuning["candidates"][tuning.get("chosen", 1) - 1]
        cb = 2 if have16 else 4
        pcg = ("k_amg_cg_spmv_pairs<Mixed> (multigrid CG: w = K u on the pair-packed SELL-32 copy + 3 dots)"
               if chosen["col16"] == 2 else "k_amg_cg_spmv<Mixed> (multigrid CG: w = K u on SELL-32 + 3 dots)")
        out["pcg_spmv"] = (pcg, (4 + cb) * Z + 12 * N + 8 * n_slices, f"(4+{cb}) Z + 12 N + 8 N/32")
        fine = ("k_amg_fine_pairs (finest-level damped-Jacobi sweep, pair-packed SELL-32, bfloat16 K)" if have16
                else "k_amg_fine<float> (finest-level damped-Jacobi sweep on SELL-32, bfloat16 K)")
        out["amg_fine"] = (fine, (2 + cb) * Z + 16 * N + 8 * n_slices, f"(2+{cb}) Z + 16 N + 8 N/32")
        rows, nz, pn = amg["rows"], amg["nnz"], amg["p_nnz"]
        packed = amg.get("packed") or [0] * len(pn)
        L = amg["levels"]
        if pn:
            # restriction: entries, R's row pointers (CSR) or slice headers (packed), the
            # fine residual gathered, the coarse vector written; prolongation: entries,
            # P's row pointers or slice headers, the coarse vector gathered, the fine
            # iterate read and written
            # (a packed copy with 32-bit columns reads 6 bytes per entry, as CSR does)
            def restrict_b(l):
                eb = 6 if packed[l] & 16 else 4
                return (eb * pn[l] + 4 * rows[l] + 4.5 * rows[l + 1] if packed[l] & 2
                        else 6 * pn[l] + 4 * rows[l] + 8 * rows[l + 1])

            def prolong_b(l):
                eb = 6 if packed[l] & 32 else 4
                return (eb * pn[l] + 8.5 * rows[l] + 4 * rows[l + 1] if packed[l] & 4
                        else 6 * pn[l] + 12 * rows[l] + 4 * rows[l + 1])
            tb = sum(restrict_b(l) + prolong_b(l) for l in range(len(pn)))
            out["amg_transfer"] = ("k_amg_restrict / k_amg_prolong (CSR) and k_amg_sellp (pair-packed SELL-32), "
                                   "bfloat16 values, every level", tb / (2 * len(pn)),
                                   "per V-cycle sum_l: restriction 6 nnz(P_l) + 4 n_l + 8 n_(l+1) (CSR) or "
                                   "4 nnz(P_l) + 4 n_l + 4.5 n_(l+1) (packed); prolongation 6 nnz(P_l) + 12 n_l "
                                   "+ 4 n_(l+1) or 4 nnz(P_l) + 8.5 n_l + 4 n_(l+1); over 2(L-1) launches")
        nc = rows[L - 1]
        ld = (nc + 3) // 4 * 4

        def sweep_b(l):
            eb = 6 if packed[l] & 8 else 4
            return eb * nz[l] + 16.5 * rows[l] if packed[l] & 1 else 6 * nz[l] + 20 * rows[l]
        cbytes = sum(2 * sweep_b(l) for l in range(1, L - 1)) + 4 * nc * ld + 8 * nc
        out["amg_coarse"] = ("k_amg_pre / k_amg_post (CSR) and k_amg_sellp (pair-packed SELL-32), bfloat16 values, "
                             "levels >= 1, and k_amg_dense",
                             cbytes / (2 * (L - 2) + 1), "per V-cycle sum_l 2 (6 nnz_l + 20 n_l) (CSR) or "
                                                         "2 (4 nnz_l + 16.5 n_l) (packed) + 4 nc ld + 8 nc, "
                                                         "over 2(L-2)+1 launches")
    bcs = tuning.get("bicg_candidates")
    bc = bcs[tuning["bicg_chosen"] - 1] if bcs else {"lanes": 0}
    c16 = bool(bc.get("col16"))
    if bc["lanes"]:
        spmm = (f"k_bicg_spmm_rows<Mixed,{D},{D}> (tentative BiCGStab: {D}-RHS product A x + dots; "
                f"{bc['lanes']} lanes per row, {bc['rows']} rows in flight, registers for {bc['min_blocks']} "
                f"blocks per SM{', 16-bit column offsets' if c16 else ''})")
    else:
        spmm = f"k_bicg_spmm<Mixed,{D},{D}> (tentative BiCGStab: {D}-RHS product A x + dots, row tiles)"
    zb = 6 if c16 else 8
    out["bicg_spmm"] = (spmm, zb * Z + 4 * (N + 1) + 12 * D * N, f"{zb} Z + 4 N + 12 D N")
    out["bicg_vec"] = ("k_bicg_dir / k_bicg_s / k_bicg_xr (BiCGStab vector updates + dots)",
                       (64 + 52 + 96) * N * D / 3 / 3, "(64 + 52 + 96) N / 3 per launch (D = 3)")
    out["assemble"] = ("k_ubar + k_cell_beta + k_assemble (convection assembly + Algorithm 2, once per step)",
                       60 * N + 80 * T + 12 * N + 48 * T + 28 * Z + 132 * N, "128 T + 28 Z + 204 N per step")
    out["outer"] = ("k_bicg_outer(_rows) / k_pcg_outer_sell (float-float residuals of the sweeps)",
                    10 * Z + 84 * N, "(8 Z + 112 N + 12 Z + 56 N) / 2 per launch")
    if amg:
        out["pcg_update"] = ("k_amg_cg_update (multigrid CG vector update + ||r||^2)", 40 * N, "40 N")
    return out


# ---------------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            # the timed region is short: start it only once the sampler is running
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                self.fh.flush()
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------- ranks
def max_over_ranks(ms, world, device):
    """The slowest rank's time: every rank times its own replica of the workload."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(steps, world, ms_max):
    """Steps of all ranks over the slowest rank's time (weak scaling: one replica per GPU)."""
    return world * steps / (ms_max / 1e3)


# ---------------------------------------------------------------------- ours
def run_ours(args, rank, world):
    import numpy as np
    import torch
    from paper_1602_03643_gb300 import build, capi
    from paper_1602_03643_gb300.driver import IPCSRun

    build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    pb = workload(args.workload, args.scalars)
    N = pb.mesh.n_dofs
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    pc = capi.OASIS_PC_AMG if args.pc == "amg" else capi.OASIS_PC_JACOBI

    def make(precision, graph=1, guess=capi.OASIS_GUESS_PREV_PHI, batch=1, pressure_pc=None):
        return IPCSRun(pb, precision=precision, rtol_u=RTOL, rtol_p=RTOL, max_it_u=5000, max_it_p=200000,
                       inner_rtol=args.inner_rtol, use_graph=graph, guess=guess, batch_rhs=batch,
                       pressure_pc=pc if pressure_pc is None else pressure_pc, inner_iters=args.inner_iters,
                       convection=1 if args.convection == "abe" else 0,
                       velocity_update=capi.OASIS_UPDATE_CONSISTENT if args.velocity_update == "consistent"
                       else capi.OASIS_UPDATE_LUMPED, stream=stream,
                       bicg_variant=args.bicg_variant if batch else 0)

    def timed_steps(run, k):
        evs = []
        stats = []
        with torch.cuda.stream(stream):
            for _ in range(k):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                capi.oasis_step(run.solver, stream, want_stats=False)
                e1.record(stream)
                evs.append((e0, e1))
                stats.append(capi.oasis_last_stats(run.solver).as_dict())
        torch.cuda.synchronize(dev)
        return sum(a.elapsed_time(b) for a, b in evs), stats

    def timed_form(run):
        """W untimed steps, barrier, then K timed steps (max over ranks)."""
        for _ in range(args.warmup):
            capi.oasis_step(run.solver, stream, want_stats=False)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        with Clocks(local) as clk:
            ms, stats = timed_steps(run, args.steps)
        torch.cuda.synchronize(dev)
        return max_over_ranks(ms, world, dev), stats, clk.summary()

    # ---- the headline form: mixed precision + batched + graph + learned guess
    # (the network is trained first, untimed, on samples the solver records
    # during the first steps of the same run)
    learned = args.guess == "learned"
    run = make(capi.OASIS_MIXED, graph=0 if args.eager else 1,
               guess=capi.OASIS_GUESS_LEARNED if learned else capi.OASIS_GUESS_PREV_PHI)
    run.set_dirichlet_for_next_step()
    train_info = None
    if learned:
        from paper_1602_03643_gb300.guess import GuessNet
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            run.record_guess(True)
            samples = []
            for k in range(args.train_steps):
                capi.oasis_step(run.solver, stream, want_stats=False)
                if k >= 2:
                    samples.append(run.guess_sample())
            run.record_guess(False)
            net = GuessNet(run.mesh, run.n, seed=1)
            losses = net.fit(samples, epochs=args.train_epochs, lr=2e-3)
            run.attach_guess_net(net)
        torch.cuda.synchronize(dev)
        train_info = {"samples": len(samples), "epochs": args.train_epochs,
                      "adam_updates": len(samples) * args.train_epochs,
                      "loss_first_epoch": float(losses[0]), "loss_last_epoch": float(losses[-1]),
                      "setup_s": time.perf_counter() - t0}
        del samples
    ms, stats, clocks = timed_form(run)
    tuning = capi.oasis_get_tuning(run.solver)
    if args.minimal:
        return {"minimal": True, "ms_per_step": ms / args.steps, "stats_last": stats[-1]}
    bad = [s for s in stats if s["status"] != 0]
    ms_per_step = ms / args.steps
    value = whole_job_value(args.steps, world, ms)

    # ---- e2e: the same step through the public API with host buffers each step
    g_host = torch.empty((pb.mesh.dim, max(1, len(pb.dirichlet))), dtype=torch.float64).pin_memory()
    g_host.numpy()[:] = pb.g(0.0) if len(pb.dirichlet) else 0.0
    u_host = torch.empty((pb.mesh.dim, N), dtype=torch.float64).pin_memory()
    p_host = torch.empty(N, dtype=torch.float64).pin_memory()
    k_e2e = max(3, args.steps // 2)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        if len(pb.dirichlet):
            capi.oasis_set_dirichlet(run.solver, g_host.numpy(), False, stream)
        capi.oasis_step(run.solver, stream, want_stats=False)
        capi.oasis_get_fields(run.solver, pb.mesh.dim, N, False, u=u_host.numpy(), p=p_host.numpy(),
                              phi=None, stream=stream)
    torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(1e3 * (time.perf_counter() - t0), world, dev) / 1e3
    h2d = len(pb.dirichlet) * pb.mesh.dim * 8
    d2h = (pb.mesh.dim + 1) * N * 8

    # ---- every kernel family, timed live with CUDA events (eager steps of the same
    # configuration; the library records events around each launch of a family)
    run_e = make(capi.OASIS_MIXED, graph=0,
                 guess=capi.OASIS_GUESS_LEARNED if learned else capi.OASIS_GUESS_PREV_PHI)
    net_e = None
    if learned:
        net_e = GuessNet(run_e.mesh, run_e.n, params=net.get_params())
        run_e.attach_guess_net(net_e)
    run_e.set_dirichlet_for_next_step()
    capi.oasis_step(run_e.solver, stream, want_stats=False)
    capi.oasis_profile(run_e.solver, True)
    n_prof = 2
    for _ in range(n_prof):
        flush.fill_(1.0)
        capi.oasis_step(run_e.solver, stream, want_stats=False)
    torch.cuda.synchronize(dev)
    fam = {f: capi.oasis_profile_read(run_e.solver, f) for f in capi.PROF_FAMILIES}
    tun_e = capi.oasis_get_tuning(run_e.solver)
    amg_info = capi.oasis_get_amg_info(run_e.solver) if pc == capi.OASIS_PC_AMG else None
    run_e.close()
    if net_e is not None:
        net_e.close()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    fams = family_bytes(pb, run.nnz, args, tun_e, amg_info)
    table = {}
    bc = tun_e["bicg_candidates"][tun_e["bicg_chosen"] - 1]
    pc_chosen = tun_e["candidates"][tun_e["chosen"] - 1] if tun_e["candidates"] else {"col16": 0}
    pairs16 = any(c["col16"] and c["us"] > 0 for c in tun_e["candidates"])
    # the layout a measured traffic figure belongs to (every shape of one layout
    # reads the same arrays once per launch)
    shape = {"bicg_spmm": ("@rows16" if bc.get("col16") else "@rows") if bc["lanes"] else "@tile",
             "pcg_spmv": "@pairs" if pc_chosen["col16"] == 2 else "@sell",
             "amg_fine": "@pairs" if pairs16 else "@sell"}
    for f, (kernel, nbytes, per) in fams.items():
        n_l, ms_l = fam.get(f, (0, 0.0))
        if not n_l:
            continue
        ach = nbytes / (ms_l / n_l / 1e3) / 1e9
        table[f] = {"kernel": kernel, "bound": "hbm", "algorithmic_bytes_per_launch": nbytes,
                    "bytes_counted": per, "launches": n_l, "avg_launch_us": ms_l / n_l * 1e3,
                    "ms_per_step": ms_l / n_prof, "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak,
                    "traffic": MEASURED_TRAFFIC.get((args.workload, f + shape.get(f, "")), (None,))[0],
                    "traffic_source": MEASURED_TRAFFIC.get((args.workload, f + shape.get(f, "")), (None, None))[1]}
    # the dominant kernel: the single-kernel family (one kernel, one launch shape)
    # that takes the most time in the step
    single = [f for f in ("pcg_spmv", "bicg_spmm", "amg_fine") if f in table]
    dominant = max(single, key=lambda f: table[f]["ms_per_step"])
    roofline = dict(table[dominant])
    roofline["family"] = dominant
    roofline["peak_source"] = ("of measured (MEASURED_PEAKS.json hbm_gbs, burst copy)" if "hbm_gbs" in peaks
                               else "of fallback 6.8 TB/s")
    roofline["note"] = ("working set larger than L2" if table[dominant]["algorithmic_bytes_per_launch"] > 129e6
                        else "algorithmic bytes below the 129 MB L2: the operands stay L2-resident across "
                             "iterations; an L2 figure")
    kernel_share = {f: {"launches": n, "ms": m} for f, (n, m) in fam.items()}

    # ---- float64 forms at the same 1e-8 residual (comparison arms)
    def short_form(run_, k):
        for _ in range(max(1, args.warmup // 2)):
            capi.oasis_step(run_.solver, stream, want_stats=False)
        ms_, st_ = timed_steps(run_, k)
        return ms_, st_

    fp64 = fp64_matched = None
    if not args.skip_fp64:
        # the same form as the headline but float64 throughout (graph, batched,
        # multigrid, previous-phi guess): isolates what the precision buys
        runm = make(capi.OASIS_FP64, graph=0 if args.eager else 1, guess=capi.OASIS_GUESS_PREV_PHI)
        runm.set_dirichlet_for_next_step()
        km = max(3, args.steps // 4)
        msm, stm = short_form(runm, km)
        runm.close()
        fp64_matched = {"form": "float64, batched, graph, multigrid, previous-phi guess",
                        "steps_per_s": km / (msm / 1e3), "ms_per_step": msm / km,
                        "it_u_mean": float(np.mean([max(s["it_u"]) for s in stm])),
                        "it_p_mean": float(np.mean([s["it_p"] for s in stm])),
                        "failed_steps": sum(s["status"] != 0 for s in stm)}
        # the plain float64 GPU form: float64, one solve per velocity component,
        # eager launches, pressure guess p = p*, Jacobi-PCG
        run64 = make(capi.OASIS_FP64, graph=0, guess=capi.OASIS_GUESS_ZERO, batch=0,
                     pressure_pc=capi.OASIS_PC_JACOBI)
        run64.set_dirichlet_for_next_step()
        k64 = max(3, args.steps // 10)
        ms64, st64 = short_form(run64, k64)
        run64.close()
        fp64 = {"form": "float64, unbatched, eager, guess p*, Jacobi-PCG",
                "steps_per_s": k64 / (ms64 / 1e3), "ms_per_step": ms64 / k64,
                "it_u_mean": float(np.mean([max(s["it_u"]) for s in st64])),
                "it_p_mean": float(np.mean([s["it_p"] for s in st64])),
                "failed_steps": sum(s["status"] != 0 for s in st64)}

    prev_form = None
    if learned and not args.skip_compare:
        runp = make(capi.OASIS_MIXED, graph=0 if args.eager else 1, guess=capi.OASIS_GUESS_PREV_PHI)

        runp.set_dirichlet_for_next_step()
        msp, stp, _ = timed_form(runp)
        runp.close()
        prev_form = {"form": "mixed, batched, graph, multigrid, previous-phi guess (no network)",
                     "steps_per_s": world * args.steps / (msp / 1e3), "ms_per_step": msp / args.steps,
                     "it_p_mean": float(np.mean([s["it_p"] for s in stp]))}
    per_rank = value / world
    ratios = {}
    if fp64_matched:
        ratios["headline_over_fp64_matched"] = per_rank / fp64_matched["steps_per_s"]
    if fp64:
        ratios["headline_over_fp64_plain"] = per_rank / fp64["steps_per_s"]
    if prev_form:
        ratios["learned_over_previous_phi"] = per_rank / (prev_form["steps_per_s"] / world)
        if fp64_matched:
            ratios["mixed_over_fp64_matched_previous_phi"] = (prev_form["steps_per_s"] / world) / \
                fp64_matched["steps_per_s"]
    if learned:
        gr = np.array([s["guess_res"] for s in stats])
        train_info |= {"used_fraction": float(np.mean([s["guess_used"] == capi.OASIS_GUESS_LEARNED
                                                       for s in stats])),
                       "residual_ratio_mean": float(np.mean(gr[:, 0] / np.maximum(gr[:, 1], 1e-300)))}

    it_u = float(np.mean([max(s["it_u"]) for s in stats]))
    it_p = float(np.mean([s["it_p"] for s in stats]))
    sw_u = float(np.mean([s["sweeps_u"] for s in stats]))
    sw_p = float(np.mean([s["sweeps_p"] for s in stats]))
    it_m = float(np.mean([s["it_m"] for s in stats]))
    it_c = float(np.mean([s["it_c"] for s in stats]))
    # kernels per step in the graph: ubar + beta + assembly 3 (explicit convection:
    # beta + assembly 2); velocity: per sweep a residual
    # and (all but the last) a correction, 5 per BiCGStab iteration; pressure: rhs
    # and guess 2, per sweep residual + CG start + (all but the last) correction,
    # 1 per CG iteration; update 1
    # learned guess: input scales, inputs, two network layers, judge.  Multigrid:
    # a V-cycle is 4 kernels per operator level + the dense coarsest solve; per
    # sweep residual, start, V-cycle, product, update (and all but the last a
    # correction); per further iteration of an inner solve (every sweep but the
    # last runs one) V-cycle, product, update.  Inner iterations
    # (Algorithm 1; the statistics describe the last repetition): per repetition
    # after the first a pressure advance, the assembly and both solves again.
    # Consistent-mass update: start 2, 2 per CG iteration, then the update.
    # Scalars (approximate: the statistics give the largest iteration count):
    # assembly, two residual sweeps and a correction, 5 per BiCGStab iteration,
    # the final update.
    if amg_info:
        vk = 4 * (amg_info["levels"] - 1) + 1
        p_kernels = sw_p * (5 + vk) + max(0, it_p - (sw_p - 1)) * (2 + vk)
    else:
        p_kernels = 3 * sw_p + it_p
    ni = max(1, args.inner_iters)
    upd_kernels = 3 + 2 * it_m if args.velocity_update == "consistent" else 1
    upd_kernels += args.scalars * (5 + 5 * it_c)
    n_asm = 2 if args.convection == "abe" else 3
    n_asm += 1   # the tentative velocity u^I formed once per dof for the pressure right-hand side
    launches = int(round(args.steps * (ni * (n_asm + 2 * sw_u + 5 * it_u + p_kernels) + (ni - 1)
                                       + (5 if learned else 0) + upd_kernels)))
    run.close()

    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed: f32 inner Krylov, f64 residual)"
                 + ("; bf16 network weights, f32 accumulation" if learned else ""),
        "data": "synthetic (seeded Taylor-Green initial field on a jittered Kuhn tetrahedral mesh)"
                if args.workload.startswith("stress") else
                "synthetic (seeded perturbed Poiseuille flow in the channel)" if args.workload == "channel" else
                "synthetic (Taylor-Green initial field on a Kuhn simplex mesh)",
        "config": workload_config(args.workload, pb, "mixed") | {
            "parallelism": f"replicas x{world}",
            "pressure_guess": "learned (judged against previous phi)" if learned else "previous phi",
            "pressure_pc": args.pc, "inner_iters": args.inner_iters, "convection": args.convection,
            "velocity_update": args.velocity_update, "scalars": args.scalars},
        "e2e": {"value": world * k_e2e / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": roofline,
        "roofline_families": table,
        "solver": {"it_u_mean": it_u, "it_p_mean": it_p, "sweeps_u_mean": sw_u, "sweeps_p_mean": sw_p,
                   "it_mass_mean": it_m, "it_scalar_max_mean": it_c,
                   "failed_steps": len(bad), "res_p_last": stats[-1]["res_p"]},
        "fp64_gpu": fp64,
        "fp64_matched": fp64_matched,
        "mixed_prev_phi": prev_form,
        "ratios": ratios,
        "learned_guess": train_info,
        "cg_autotune": tuning,
        "multigrid": amg_info,
        "kernel_time_eager_2steps": kernel_share,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, pb, budget_s=args.cpu_budget)
    return line


# ---------------------------------------------------------------------- oracle (CPU)
def run_guess_study(args):
    """The learned-guess experiment on the channel (held-out seed): the network is
    trained on samples that the plain solver records in runs from other seeds,
    then the held-out run is stepped with the zero, previous-phi and learned
    guesses; every pressure solve ends at the same 1e-8 residual.  Reported:
    mean CG iterations and device steps/s of each form (one GPU)."""
    import ctypes
    import numpy as np
    import torch
    from paper_1602_03643_gb300 import build, capi
    from paper_1602_03643_gb300.driver import IPCSRun
    from paper_1602_03643_gb300.guess import GuessNet
    from workloads import problems as WP
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)

    def make(seed, guess):
        pb = WP.channel(seed=seed)
        run = IPCSRun(pb, precision=capi.OASIS_MIXED, rtol_u=RTOL, rtol_p=RTOL, max_it_u=20000,
                      max_it_p=200000, inner_rtol=args.inner_rtol, use_graph=1, guess=guess,
                      pressure_pc=capi.OASIS_PC_AMG, stream=stream)
        run.set_dirichlet_for_next_step()
        return run

    t0 = time.perf_counter()
    samples = []
    train_seeds = list(range(100, 100 + args.study_seeds))
    stopped = {}
    with torch.cuda.stream(stream):
        for sd in train_seeds:
            run = make(sd, capi.OASIS_GUESS_PREV_PHI)
            run.record_guess(True)
            for k in range(args.study_steps):
                capi.oasis_step(run.solver, stream, want_stats=False)
                # a run that has left the scheme's stable range (a failed solve,
                # non-finite fields) gives no further training samples
                st = capi.oasis_step_stats()
                capi.lib().oasis_last_stats(run.solver, ctypes.byref(st))
                if st.status != 0:
                    stopped[sd] = k
                    break
                if k >= 2:
                    feat, target = run.guess_sample()
                    if bool(torch.isfinite(feat).all()) and bool(torch.isfinite(target).all()):
                        samples.append((feat, target))
            run.record_guess(False)
            torch.cuda.synchronize(dev)
            run.close()
    t_collect = time.perf_counter() - t0
    test = {}
    for form, guess in (("zero", capi.OASIS_GUESS_ZERO), ("previous_phi", capi.OASIS_GUESS_PREV_PHI),
                        ("learned", capi.OASIS_GUESS_LEARNED)):
        run = make(110, guess)
        net = None
        if form == "learned":
            with torch.cuda.stream(stream):
                # the records and the network live on the mesh of the run that uses them
                net = GuessNet(run.mesh, run.n, seed=1)
                t1 = time.perf_counter()
                losses = net.fit(samples, epochs=args.train_epochs, lr=2e-3)
                torch.cuda.synchronize(dev)
                t_fit = time.perf_counter() - t1
                run.attach_guess_net(net)
        for _ in range(args.warmup):
            capi.oasis_step(run.solver, stream, want_stats=False)
        torch.cuda.synchronize(dev)
        evs, stats = [], []
        with torch.cuda.stream(stream):
            for _ in range(args.study_test_steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                capi.oasis_step(run.solver, stream, want_stats=False)
                e1.record(stream)
                evs.append((e0, e1))
                # a failed solve is counted, not raised (its stats are still filled)
                st = capi.oasis_step_stats()
                capi.lib().oasis_last_stats(run.solver, ctypes.byref(st))
                stats.append(st.as_dict())
        torch.cuda.synchronize(dev)
        ms = sum(a.elapsed_time(b) for a, b in evs)
        it_p = [st["it_p"] for st in stats]
        entry = {"steps_per_s": 1e3 * len(evs) / ms, "ms_per_step": ms / len(evs),
                 "it_p_mean": float(np.mean(it_p)), "it_u_mean": float(np.mean([max(st["it_u"]) for st in stats])),
                 "failed_steps": sum(st["status"] != 0 for st in stats),
                 "first_failed_step": next((k for k, st in enumerate(stats) if st["status"] != 0), None),
                 "statuses": sorted({st["status"] for st in stats})}
        if form == "learned":
            gr = np.array([st["guess_res"] for st in stats])
            entry |= {"used_fraction": float(np.mean([st["guess_used"] == capi.OASIS_GUESS_LEARNED
                                                      for st in stats])),
                      "residual_ratio_mean": float(np.mean(gr[:, 0] / np.maximum(gr[:, 1], 1e-300))),
                      "loss_first_epoch": float(losses[0]), "loss_last_epoch": float(losses[-1]),
                      "fit_s": t_fit}
            net.close()
        run.close()
        test[form] = entry
    return {"study": "learned pressure guess, channel 128x96x96, held-out seed 110",
            "train": {"seeds": train_seeds, "steps_per_seed": args.study_steps, "samples": len(samples),
                      "runs_stopped_at_failed_step": stopped,
                      "epochs": args.train_epochs, "collect_s": t_collect},
            "test": {"seed": 110, "warmup": args.warmup, "steps": args.study_test_steps} | test,
            "solver": "mixed, 3-RHS BiCGStab, multigrid CG, CUDA graph, every solve to 1e-8",
            "data": "synthetic (seeded perturbed Poiseuille flow in the channel)"}


def oracle_options(args):
    """The scheme options of the run, in the oracle's terms."""
    return {"inner_iters": max(1, getattr(args, "inner_iters", 1)),
            "convection": getattr(args, "convection", "abcn"),
            "velocity_update": getattr(args, "velocity_update", "lumped")}


def cpu_baseline(args, pb, budget_s=20.0):
    """The CPU float64 oracle, as it stands, on this host (iterative solves at 1e-8)."""
    import numpy as np  # noqa: F401
    from oracle.ipcs import IPCS
    t0 = time.perf_counter()
    o = IPCS(pb, iterative=True, rtol=RTOL, **oracle_options(args))
    setup = time.perf_counter() - t0
    s = o.initial_state()
    n = 0
    t1 = time.perf_counter()
    while True:
        s = o.step(s)
        n += 1
        if time.perf_counter() - t1 > budget_s or n >= args.steps:
            break
    el = time.perf_counter() - t1
    return {"value": n / el, "unit": "steps/s", "cores": _threads(), "kind": "oracle",
            "sample": f"{n} full steps of the same workload (float64, scipy BiCGStab/CG + Jacobi at rtol 1e-8, "
                      f"setup {setup:.1f} s excluded)"}


def _threads():
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, rank, world):
    if rank != 0:
        return None
    pb = workload(args.workload, getattr(args, "scalars", 0))
    from oracle.ipcs import IPCS
    o = IPCS(pb, iterative=True, rtol=RTOL, **oracle_options(args))
    s = o.initial_state()
    for _ in range(min(args.warmup, 1)):
        s = o.step(s)
    n, t0 = 0, time.perf_counter()
    while n < args.steps and time.perf_counter() - t0 < args.cpu_budget * 4:
        s = o.step(s)
        n += 1
    el = time.perf_counter() - t0
    v = n / el
    cores = _threads()
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": world,
            "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 * el / n, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, pb, "fp64 (CPU oracle)", gpu=False),
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} full steps (iterative float64 oracle, rtol 1e-8)"},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="stress128_rcm")
    ap.add_argument("--inner-rtol", type=float, default=1e-4)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-compare", action="store_true",
                    help="do not time the previous-phi form beside the learned one")
    ap.add_argument("--guess", default="learned", choices=["learned", "prev"])
    ap.add_argument("--convection", default="abcn", choices=["abcn", "abe"],
                    help="convection form: ubar.grad u~ (Eq. 22) or explicit Adams-Bashforth (Eq. 21)")
    ap.add_argument("--velocity-update", default="lumped", choices=["lumped", "consistent"],
                    help="velocity update of the projection: lumped mass or a CG on the consistent mass "
                         "matrix (Sec. 5)")
    ap.add_argument("--scalars", type=int, default=0,
                    help="passive scalars transported with the flow (Sec. 3 scalar equation)")
    ap.add_argument("--inner-iters", type=int, default=1,
                    help="inner velocity/pressure iterations per step (Algorithm 1)")
    ap.add_argument("--bicg-variant", type=int, default=0,
                    help="shape of the batched BiCGStab product: 0 = autotuned at solver creation, k >= 1 = "
                         "candidate k of the tuning report (bicg_variant of the solver parameters)")
    ap.add_argument("--pc", default="amg", choices=["amg", "jacobi"],
                    help="pressure-CG preconditioner (multigrid V-cycle or Jacobi)")
    ap.add_argument("--train-steps", type=int, default=14)
    ap.add_argument("--train-epochs", type=int, default=60)
    ap.add_argument("--minimal", action="store_true",
                    help="only the warm-up and timed steps (for profiler captures)")
    ap.add_argument("--eager", action="store_true",
                    help="run the headline form as eager launches (profilers cannot see kernels "
                         "inside graphs with conditional nodes)")
    ap.add_argument("--guess-study", action="store_true",
                    help="the learned-guess experiment on the channel with a held-out seed (one GPU)")
    ap.add_argument("--study-seeds", type=int, default=6)
    ap.add_argument("--study-steps", type=int, default=40)
    ap.add_argument("--study-test-steps", type=int, default=40)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.guess_study:
        print(json.dumps(run_guess_study(args)), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    line = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
