"""Benchmark: batched RKS B3LYP/STO-3G SCF, molecules/s on one GB300.

Workload (default): 4096 seeded synthetic molecules with 9-11 heavy atoms
(C/N/O/F + H, the paper's QM1B shape), mixed precision, 20 SCF iterations plus
the final step (FP64 recompute of the largest quartets, exact fixed-point
sums).  One "step" = the whole method for the whole batch: integrals, Schwarz
screening and packing, ERIs, grid, 20 iterations of J/K + XC + FP64
DIIS/eigh, final step.

The mixed path runs with the recheck: molecules whose DIIS error is still
above 1e-4 after the 20 iterations run again from the initial guess with
every Fock build at the final step's precision, and the unconverged ones
(DIIS error above 3e-4) are redone on the FP64 path.

Printed JSON line (rank 0):
  value       molecules within the accuracy gate per second, inputs resident
              in HBM (CUDA events on the library's stream around K steps)
  gate        every molecule of the run against the plain FP64 GPU path
              (itself pinned to the FP64 oracle by the parity tests): counts
              over |dE| 1e-5 Ha and |d gap| 1e-4 Ha; a molecule outside the
              gate does not count in value
  e2e         the same metric through the serving API (rks_submit / rks_wait /
              rks_result) with host buffers: H2D, every kernel and D2H inside
  latency_s   p50 / p99 of a short Poisson trace through the serving API
  roofline    the dominant kernel's achieved rate vs the peak, measured by the
              library's probes in the same run (peaks_probed_tflops)
  cpu_baseline  the FP64 oracle on the host cores (bounded sample)
  fp64_gpu    the FP64 GPU path's molecules/s on the same molecules

--impl reference times the FP64 oracle as the reference arm.
Multi-GPU: molecules are independent, so N ranks run N independent shards
(weak scaling, no collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import molgen  # noqa: E402

# dram__bytes_read.sum + dram__bytes_write.sum of grid_xc_tc_kernel<float, 0, NQ>
# per grid point from one ncu capture of the current kernel (38 molecules:
# 16.73 B at NQ = 16, 16.90 B at NQ = 20; the points' coordinates and weights
# are 16 B); scaled by the points of a launch.  Set to None when the kernel
# changes until it has been captured again.
GRID_TC_DRAM_BYTES_PER_POINT = 16.8

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}
METRIC = "molecules/s (9-11 heavy atoms, |dE|<=1e-5 Ha) mixed vs FP64 on 1 GB300; p50/p99"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["_source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["_source"] = "fallback"
    return d


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self):
        self.samples = []
        self.proc = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", os.environ.get("LOCAL_RANK", "0")],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if not self.samples:
            return out
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, n in enumerate(names):
                if s[3 + k].lower() == "active":
                    reasons.add(n)
        out["sm_mhz"] = statistics.median(sm) if sm else None
        out["sm_max_mhz"] = max(mx) if mx else None
        out["reasons"] = sorted(reasons)
        out["samples"] = len(self.samples)
        return out


def workload(nmol, seed=2):
    return molgen.batch(seed, nmol, 9, 11)


def workload_config(nmol, world):
    """The `config` of the JSON line (both arms)."""
    return {"workload": f"{nmol} molecules/GPU, 9-11 heavy atoms (C/N/O/F+H), B3LYP(VWN5)/STO-3G, "
                        "mixed precision, 20 SCF iterations + final correction step",
            "nmol_per_gpu": nmol, "seed": 2, "l2": "inputs larger than L2 (packed ERIs ~10 MB x nmol)",
            "parallelism": f"replicas x{world}"}


def shard_indices(nmol_per_rank, rank, world):
    """Molecules of rank `rank`: r, r + N, ... of an N * nmol_per_rank set.
    Molecules are independent, so the shards need no exchange (weak scaling)."""
    return list(range(rank, nmol_per_rank * world, world))


def max_over_ranks(x):
    """Max of a host float over the ranks of the default process group
    (the only collective of the benchmark: timing, not data)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()):
        return float(x)
    dev = "cuda" if tdist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------ oracle leg
def oracle_sample(mol, n_iter_timed=2):
    """Time the FP64 oracle on one molecule: iteration-0 work (integrals,
    packed store, grid, AOs) once, then n_iter_timed Fock builds + DIIS/eigh.
    Returns per-molecule seconds for the 20 + 1 Fock-build protocol."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import scf
    Z, xyz = mol
    t0 = time.perf_counter()
    s = scf.System(Z, xyz)
    t_setup = time.perf_counter() - t0
    D = s.core_guess()
    t0 = time.perf_counter()
    for _ in range(n_iter_timed):
        F, E, _ = s.fock(D)
        _, _, D = scf.solve_fock(F, s.X, s.nocc)
    t_it = (time.perf_counter() - t0) / n_iter_timed
    return t_setup, t_it, t_setup + 21 * t_it


def _oracle_worker(mol):
    return oracle_sample(mol)


def cpu_baseline_all_cores(mols):
    """The oracle on every host core at once: one molecule per process (spawned,
    one BLAS thread each), each timed as in oracle_sample; the throughput is the
    sum of the per-process rates."""
    import multiprocessing as mp
    _threadpool_limit()
    ncores = os.cpu_count() or 1
    sample = [mols[k % len(mols)] for k in range(ncores)]
    with mp.get_context("spawn").Pool(ncores) as pool:
        res = pool.map(_oracle_worker, sample, chunksize=1)
    rate = sum(1.0 / r[2] for r in res)
    t_setup = float(np.mean([r[0] for r in res]))
    t_it = float(np.mean([r[1] for r in res]))
    return {"value": rate, "unit": "molecules/s", "cores": ncores, "kind": "oracle",
            "sample": f"{ncores} molecules of the workload, one per core in parallel: iteration-0 work once "
                      f"(mean {t_setup:.1f} s) + 2 timed Fock builds (mean {t_it:.2f} s each), each scaled "
                      f"to 21 Fock builds per molecule; value = sum of the per-core rates"}


def _threadpool_limit():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores (one molecule of the
    workload per step, bounded to one Fock build per timed step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    _threadpool_limit()
    from oracle import scf
    mol = workload(1)[0]
    t0 = time.perf_counter()
    s = scf.System(*mol)
    t_setup = time.perf_counter() - t0
    D = s.core_guess()

    def step():
        nonlocal D
        F, E, _ = s.fock(D)
        _, _, D = scf.solve_fock(F, s.X, s.nocc)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    t_it = (time.perf_counter() - t0) / args.steps
    per_mol = t_setup + 21 * t_it
    value = 1.0 / per_mol
    sample = (f"1 molecule of the 9-11 heavy-atom workload (nbf={s.nbf}, {len(s.w)} grid points): "
              f"iteration-0 work timed once ({t_setup:.1f} s), then {args.steps} timed Fock builds "
              f"({t_it:.2f} s each); per molecule = setup + 21 Fock builds")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "molecules/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_it * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.nmol, args.gpus),
            "cpu_baseline": {"value": value, "unit": "molecules/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "molecules/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- serving leg
SERVE_TOL = {"fp64": (1e-7, 1e-5), "mixed": (1e-5, 1e-5)}


def serve_run(g, precision, rate, n, seed=3):
    """Poisson serving trace (1-11 heavy atoms) through rks_submit / rks_wait /
    rks_result with the serving protocol: converge (|dE| < e_tol, max|e| <
    err_tol, at most 40 iterations), then the final step.  The mixed path's
    iteration energies carry ~1e-6 Ha of FP32 product rounding, so its dE test
    sits at 1e-5 (the reported energy comes from the exactly summed final
    step).  Latency is submit -> result published, from the library;
    sustained throughput is molecules / (last completion - first submission)."""
    t_arr, mols = molgen.serving_trace(seed, n, rate)
    pname = "mixed" if precision == g.RKS_MIXED else "fp64"
    e_tol, err_tol = SERVE_TOL[pname]
    opts = dict(precision=precision, fixed_iters=0, e_tol=e_tol, err_tol=err_tol, max_iters=40, admit_wait_us=2000)
    with g.Context(**opts) as ctx:
        warm = ctx.submit_many(mols[:8])  # module load and first launches, not measured
        for tk in warm:
            ctx.wait(tk, 600)
            ctx.result(tk)
        tickets, t_sub = [None] * n, [0.0] * n
        t0 = time.perf_counter()

        def submitter():
            for i in range(n):
                dt = t_arr[i] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                t_sub[i] = time.perf_counter() - t0
                tickets[i] = ctx.submit(*mols[i])

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        lat, done, bad, energies = [], [], 0, []
        for i, tk in enumerate(tickets):
            ctx.wait(tk, 3600)
            r = ctx.result(tk)
            lat.append(r["latency_s"])
            done.append(t_sub[i] + r["latency_s"])
            bad += r["status"] != "ok"
            energies.append((r["E"], r["gap"]))
    span = max(done) - t_sub[0]
    return {"mode": "serve", "precision": pname, "rate_per_s": rate,
            "n": n, "sustained_mol_per_s": n / span, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "not_converged": bad, "e_tol": e_tol, "err_tol": err_tol,
            "workload": "Poisson arrivals, 1-11 heavy atoms (seed 3), converge then final step, cap 40"}, energies


def serve_main(args):
    """Rate sweep, mixed then FP64 (fewer molecules: ~20x slower); the
    molecules of the FP64 runs are the first ones of the mixed runs, so the
    mixed-vs-FP64 energy and gap differences are reported on them."""
    import paper_2311_01135_gb300 as g
    g.build()
    plan = [(g.RKS_MIXED, r, args.serve_n) for r in (100, 300, 1000, 5000)]
    plan += [(g.RKS_FP64, r, max(40, args.serve_n // 10)) for r in (5, 20)]
    first_mixed = None
    for prec, rate, n in plan:
        line, en = serve_run(g, prec, rate, n)
        if prec == g.RKS_MIXED and first_mixed is None:
            first_mixed = en
        if prec == g.RKS_FP64 and first_mixed is not None:
            k = min(len(en), len(first_mixed))
            line["mixed_vs_fp64_max_abs_dE"] = max(abs(a[0] - b[0]) for a, b in zip(first_mixed[:k], en[:k]))
            line["mixed_vs_fp64_max_abs_dgap"] = max(abs(a[1] - b[1]) for a, b in zip(first_mixed[:k], en[:k]))
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------ validation
def _oracle_fixed20(mol):
    """The oracle's fixed protocol (20 iterations + the final Fock build)."""
    from oracle import scf
    r = scf.run_scf(scf.System(*mol), protocol="fixed", n_iter=20)
    return r["E"], r["gap"], r["D"]


def converge_main(args):
    """The batch workload under the converge protocol: each molecule iterates
    until |E_k - E_(k-1)| and the DIIS error fall below the thresholds (at
    most max_iters), drops out of the iterations when it does, then takes the
    final step.  Mixed on every molecule, timed with CUDA events on the
    batch's stream (setup included); the FP64 path, converged tighter, on the
    first --converge-ref-n molecules as the reference of the gate."""
    import torch
    import paper_2311_01135_gb300 as g
    g.build()
    mols = workload(args.nmol)
    copt = dict(fixed_iters=0, max_iters=100)
    with g.Context(precision=g.RKS_MIXED, e_tol=1e-6, err_tol=1e-5, **copt) as ctx:
        stream = torch.cuda.ExternalStream(ctx.stream())
        with g.Batch(ctx, mols[:8]) as Bw:  # module load, first launches
            Bw.run()
            Bw.sync()
        with g.Batch(ctx, mols) as B:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.setup()
            B.run()
            e1.record(stream)
            B.sync()
            ms = e0.elapsed_time(e1)
            rmx = [B.result(m) for m in range(len(mols))]
    nref = min(args.converge_ref_n, len(mols))
    with g.Context(precision=g.RKS_FP64, e_tol=1e-8, err_tol=1e-6, **copt) as c64, \
            g.Batch(c64, mols[:nref]) as B64:
        t0 = time.perf_counter()
        B64.run()
        B64.sync()
        t64 = time.perf_counter() - t0
        r64 = [B64.result(m) for m in range(nref)]
    it = np.array([r["iters"] for r in rmx])
    conv = np.array([r["status"] == "ok" for r in rmx])
    ok = [(a, b) for a, b in zip(rmx[:nref], r64) if a["status"] == "ok" and b["status"] == "ok"]
    dE = np.array([abs(a["E"] - b["E"]) for a, b in ok])
    dg = np.array([abs(a["gap"] - b["gap"]) for a, b in ok])
    line = {"metric": "molecules/s under the converge protocol (mixed, |dE_k| < 1e-6 Ha, DIIS error < 1e-5)",
            "value": len(mols) / (ms / 1e3), "unit": "molecules/s", "n_gpus": 1, "nmol": len(mols),
            "ms": ms, "converged": int(conv.sum()), "not_converged": int((~conv).sum()),
            "iterations": {"min": int(it.min()), "p50": float(np.median(it)), "p90": float(np.percentile(it, 90)),
                           "max": int(it.max()), "mean": float(it.mean())},
            "gate_vs_fp64_converged": {"n_checked": len(ok), "n_dE_over_1e-5": int((dE > GATE_DE).sum()),
                                       "n_dgap_over_1e-4": int((dg > GATE_DGAP).sum()),
                                       "max_abs_dE": float(dE.max()) if len(dE) else None,
                                       "max_abs_dgap": float(dg.max()) if len(dg) else None,
                                       "p99_abs_dE": float(np.percentile(dE, 99)) if len(dE) else None,
                                       "fp64": "converged to |dE_k| < 1e-8 Ha, DIIS error < 1e-6",
                                       "fp64_not_converged": sum(1 for b in r64 if b["status"] != "ok")},
            "fp64_reference_mol_per_s": nref / t64,
            "data": "synthetic",
            "config": dict(workload_config(len(mols), 1),
                           workload=f"{len(mols)} molecules/GPU, 9-11 heavy atoms (C/N/O/F+H), B3LYP(VWN5)/STO-3G, "
                                    "mixed precision, converge protocol (at most 100 iterations) + final step")}
    print(json.dumps(line), flush=True)


def large_workload(nmol, seed=4):
    """The larger-molecule workload: 20-30 heavy atoms (seed 4), basis ~120-200."""
    return molgen.batch(seed, nmol, 20, 30)


def large_main(args):
    """The 20-30-heavy-atom workload: every stage on the global-memory kernels
    (J/K, two-pass grid quadrature, SCF steps with global Jacobi scratch).
    Mixed precision on --large-n molecules (CUDA events around setup + run on
    the batch's stream), under the converge protocol (default: each molecule
    iterates until |dE_k| < 1e-6 Ha and its DIIS error < 1e-5, then takes the
    final step) or the fixed one (20 iterations + recheck + final step); stage
    times of a profiled run on the first --large-prof-n; the FP64 path on the
    first --large-fp64-n (the gate's reference, converged to 1e-8 Ha / 1e-6
    under the converge protocol; pinned to the oracle by
    tests/test_gpu_large.py); direct SCF (every quartet recomputed inside J/K,
    no packed store) on the first --large-direct-n."""
    import torch
    import paper_2311_01135_gb300 as g
    g.build()
    mols = large_workload(args.large_n)
    nbf = np.array([g.rks_nbf(Z) for Z, _ in mols])
    if args.large_protocol == "converge":
        opt = dict(fixed_iters=0, max_iters=100, e_tol=1e-6, err_tol=1e-5)
        opt64 = dict(fixed_iters=0, max_iters=100, e_tol=1e-8, err_tol=1e-6)
    else:
        opt = dict(fixed_iters=20, recheck_err=RECHECK_ERR, recheck_fp64_err=RECHECK_FP64_ERR)
        opt64 = dict(fixed_iters=20)

    def timed(ctx, sub):
        stream = torch.cuda.ExternalStream(ctx.stream())
        with g.Batch(ctx, sub) as B:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.setup()
            B.run()
            e1.record(stream)
            B.sync()
            ms = e0.elapsed_time(e1)
            return ms, [B.result(k) for k in range(len(sub))]

    with g.Context(precision=g.RKS_MIXED, **opt) as ctx:
        timed(ctx, mols[:1])  # module load, first launches
        clocks = Clocks()
        clocks.start()
        ms, rmx = timed(ctx, mols)
        ck = clocks.stop()
        probes = measured_peaks(g, ctx)
        sub = mols[:args.large_prof_n]
        sc, prof = [], {}
        if sub:
            ctx.profile(True)
            with g.Batch(ctx, sub) as Bp:
                Bp.setup()
                Bp.run()
                Bp.sync()
                sc = [Bp.dump(m, g.RKS_DUMP_SCALARS) for m in range(len(sub))]
            prof = ctx.profile_read()
            ctx.profile(False)
    n64 = min(args.large_fp64_n, len(mols))
    ms64, r64 = None, []
    if n64 > 0:
        with g.Context(precision=g.RKS_FP64, **opt64) as c64:
            ms64, r64 = timed(c64, mols[:n64])
    nd = min(args.large_direct_n, len(mols))
    msd, rd = None, []
    if nd > 0:
        with g.Context(precision=g.RKS_MIXED, direct_scf=g.RKS_DIRECT_ALWAYS, **opt) as cd:
            msd, rd = timed(cd, mols[:nd])
    gate = gate_report(rmx[:n64], r64) if n64 > 0 else None
    it = np.array([r["iters"] for r in rmx])
    ddir = [abs(a["E"] - b["E"]) for a, b in zip(rd, rmx[:nd])]
    # rooflines of the two iteration kernels, from the profiled sample
    pk = peaks()
    roof = {}
    pts = [s_[6] for s_ in sc]
    if "grid_large" in prof:
        st = prof["grid_large"]
        flops = sum(4.0 * p_ * k * k for p_, k in zip(pts, nbf[:len(sub)]))  # rho and V' passes, dense
        ach = flops / (st["ms"] / max(st["launches"], 1) / 1e3) / 1e12
        peak = probes.get("fp32_fma")
        roof["grid_large"] = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                              "frac": ach / peak if peak else None,
                              "units": "4 * points * nbf^2 per molecule per launch (T = Phi D and Phi^T X)",
                              "peak_source": "FP32 FMA measured by rks_probe_peak in this run"}
    if "jk_large" in prof:
        st = prof["jk_large"]
        nbytes = sum(4.0 * s_[5] for s_ in sc)
        ach = nbytes / (st["ms"] / max(st["launches"], 1) / 1e3) / 1e9
        roof["jk_large"] = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                            "frac": ach / pk["hbm_gbs"], "units": "4 B x packed store elements per launch",
                            "peak_source": pk["_source"]}
    line = {"metric": "molecules/s (20-30 heavy atoms) mixed vs FP64 on 1 GB300", "value": len(mols) / (ms / 1e3),
            "unit": "molecules/s", "n_gpus": 1, "ms": ms, "higher_is_better": True, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": f"{len(mols)} molecules, 20-30 heavy atoms (C/N/O/F+H), B3LYP(VWN5)/STO-3G, "
                                   "mixed precision, " + ("converge protocol (|dE_k| < 1e-6 Ha, DIIS error < 1e-5, "
                                                          "at most 100 iterations) + final step"
                                                          if args.large_protocol == "converge" else
                                                          "20 SCF iterations + recheck + final step"),
                       "seed": 4, "protocol": args.large_protocol,
                       "nbf": {"min": int(nbf.min()), "mean": float(nbf.mean()), "max": int(nbf.max())}},
            "status_not_ok": sum(1 for r in rmx if r["status"] != "ok"),
            "iterations": {"min": int(it.min()), "p50": float(np.median(it)), "max": int(it.max()),
                           "mean": float(it.mean())},
            "clocks": ck, "gate_vs_fp64_sample": gate,
            "fp64_gpu": {"value": n64 / (ms64 / 1e3), "unit": "molecules/s", "nmol": n64} if ms64 else None,
            "direct_scf": {"value": nd / (msd / 1e3), "unit": "molecules/s", "nmol": nd,
                           "max_abs_dE_vs_stored": float(max(ddir)) if ddir else None} if msd else None,
            "roofline_large": roof, "peaks_probed_tflops": probes,
            "stages_ms_sample": {k: round(v["ms"], 3) for k, v in prof.items()}, "sample_n": len(sub)}
    print(json.dumps(line), flush=True)


def validate_main(args):
    """Accuracy of the whole workload: the mixed path against the FP64 GPU path
    on every molecule, and both against the FP64 oracle on a subset stratified
    by heavy-atom count (the oracle runs on the host cores meanwhile)."""
    import multiprocessing as mp
    _threadpool_limit()
    mols = workload(args.nmol)
    nheavy = [sum(1 for z in Z if z > 1) for Z, _ in mols]
    subset = []
    for h in (9, 10, 11):
        subset += [i for i, k in enumerate(nheavy) if k == h][: args.oracle_n // 3]
    pool = mp.get_context("spawn").Pool(os.cpu_count() or 1)
    pending = pool.map_async(_oracle_fixed20, [mols[i] for i in subset], chunksize=1)
    import paper_2311_01135_gb300 as g
    g.build()
    res = {}
    for name, prec in (("mixed", g.RKS_MIXED), ("fp64", g.RKS_FP64)):
        t0 = time.perf_counter()
        with g.Context(precision=prec, fixed_iters=20) as c, g.Batch(c, mols) as B:
            B.run()
            B.sync()
            res[name] = [B.result(m) for m in range(len(mols))]
        res[name + "_s"] = time.perf_counter() - t0
    ora = pending.get()
    pool.close()
    mx, f64 = res["mixed"], res["fp64"]

    def stats(a, b):
        return float(np.max(a)), float(np.mean(a)), float(np.percentile(a, 99))

    dE = np.array([abs(a["E"] - b["E"]) for a, b in zip(mx, f64)])
    dg = np.array([abs(a["gap"] - b["gap"]) for a, b in zip(mx, f64)])
    dD = np.array([np.max(np.abs(a["D"] - b["D"])) for a, b in zip(mx, f64)])
    # molecules whose FP64 SCF is still moving after 20 iterations (DIIS error
    # above 1e-4): E[D_20] is not stationary there, so both paths' energies
    # depend on the trajectory, and FP32 rounding can steer the mixed one away
    moving = np.array([r["err_max"] > 1e-4 for r in f64])
    oE = np.array([abs(f64[i]["E"] - o[0]) for i, o in zip(subset, ora)])
    oEm = np.array([abs(mx[i]["E"] - o[0]) for i, o in zip(subset, ora)])
    ogm = np.array([abs(mx[i]["gap"] - o[1]) for i, o in zip(subset, ora)])
    line = {"mode": "validate", "nmol": len(mols), "workload": "9-11 heavy atoms, seed 2, fixed 20 iterations + final",
            "mixed_vs_fp64": {"max_abs_dE": stats(dE, None)[0], "mean_abs_dE": stats(dE, None)[1],
                              "p99_abs_dE": stats(dE, None)[2], "max_abs_dgap": float(dg.max()),
                              "max_abs_dD": float(dD.max()), "n_over_1e-5": int((dE > 1e-5).sum()),
                              "n_gap_over_1e-4": int((dg > 1e-4).sum())},
            "fp64_err_max_over_1e-4": int(moving.sum()),
            "mixed_vs_fp64_settled": {"n": int((~moving).sum()), "max_abs_dE": float(dE[~moving].max()),
                                      "max_abs_dgap": float(dg[~moving].max()),
                                      "n_over_1e-5": int((dE[~moving] > 1e-5).sum())},
            "mixed_vs_fp64_moving": {"n": int(moving.sum()),
                                     "max_abs_dE": float(dE[moving].max()) if moving.any() else None},
            "oracle_subset": len(subset),
            "fp64_vs_oracle_max_abs_dE": float(oE.max()), "mixed_vs_oracle_max_abs_dE": float(oEm.max()),
            "mixed_vs_oracle_max_abs_dgap": float(ogm.max()),
            "status_not_ok": {k: sum(r["status"] != "ok" for r in res[k]) for k in ("mixed", "fp64")},
            "wall_s": {"mixed": res["mixed_s"], "fp64": res["fp64_s"]}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU leg
# Mixed-precision options of the benchmark (and of every GPU leg below): the
# fixed protocol, with molecules still moving after the 20 iterations run
# again at the final step's precision (rks_options.recheck_err).
RECHECK_ERR, RECHECK_FP64_ERR = 1e-4, 3e-4
GATE_DE, GATE_DGAP = 1e-5, 1e-4


def fp64_leg(g, mols, device, budget_s, chunk=512):
    """The plain FP64 GPU path on the same molecules, in chunks, until every
    molecule is done or the next chunk would overrun budget_s.  Returns the
    per-molecule results (None where not run) and molecules/s."""
    import torch
    res = [None] * len(mols)
    done, t_run = 0, 0.0
    with g.Context(precision=g.RKS_FP64, fixed_iters=20, device=device) as c64:
        s64 = torch.cuda.ExternalStream(c64.stream())
        with g.Batch(c64, mols[:4]) as Bw:  # warm-up (module load, first launches)
            Bw.run()
            Bw.sync()
        t_chunk = None
        while done < len(mols):
            if t_chunk is not None and t_run + t_chunk > budget_s:
                break
            sub = mols[done:done + chunk]
            with g.Batch(c64, sub) as B64:
                f0 = torch.cuda.Event(enable_timing=True)
                f1 = torch.cuda.Event(enable_timing=True)
                f0.record(s64)
                B64.setup()
                B64.run()
                f1.record(s64)
                B64.sync()
                ms = f0.elapsed_time(f1)
                for k in range(len(sub)):
                    res[done + k] = B64.result(k)
            t_run += ms / 1e3
            t_chunk = ms / 1e3 * (chunk / len(sub))
            done += len(sub)
    return res, done / t_run if t_run > 0 else None, t_run


def gate_report(rmx, r64):
    """Mixed vs FP64 GPU (the FP64 path is itself pinned to the oracle at
    ~1e-10 Ha by the parity tests) on every molecule both ran."""
    pairs = [(a, b) for a, b in zip(rmx, r64) if b is not None]
    dE = np.array([abs(a["E"] - b["E"]) for a, b in pairs])
    dg = np.array([abs(a["gap"] - b["gap"]) for a, b in pairs])
    bad_status = sum(1 for a, b in pairs if a["status"] != "ok" or b["status"] != "ok")
    fail = (dE > GATE_DE) | (dg > GATE_DGAP)
    return {"n_checked": len(pairs), "n_dE_over_1e-5": int((dE > GATE_DE).sum()),
            "n_dgap_over_1e-4": int((dg > GATE_DGAP).sum()), "n_fail": int(fail.sum()),
            "max_abs_dE": float(dE.max()) if len(dE) else None,
            "max_abs_dgap": float(dg.max()) if len(dg) else None,
            "p99_abs_dE": float(np.percentile(dE, 99)) if len(dE) else None,
            "status_not_ok": bad_status, "n_rerun_precise": int(sum(1 for a in rmx if a["rechecked"] == 1)),
            "n_redone_fp64": int(sum(1 for a in rmx if a["rechecked"] == 2)),
            "passed": bool(len(pairs) and not fail.any() and bad_status == 0)}


def serve_leg(g, mols, rate, device):
    """A short Poisson trace of the workload's molecules through the serving
    API (rks_submit / rks_wait / rks_result), the benchmark's protocol:
    latency = submit -> result published, p50 / p99."""
    rng = np.random.default_rng(2 + int(rate))
    t_arr = np.cumsum(rng.exponential(1.0 / rate, size=len(mols)))
    with g.Context(precision=g.RKS_MIXED, fixed_iters=20, recheck_err=RECHECK_ERR,
                   recheck_fp64_err=RECHECK_FP64_ERR, device=device, admit_wait_us=2000) as ctx:
        for tk in ctx.submit_many(mols[:8]):  # module load, not measured
            ctx.wait(tk, 600)
            ctx.result(tk)
        tickets, t_sub = [None] * len(mols), [0.0] * len(mols)
        t0 = time.perf_counter()
        for i, m in enumerate(mols):
            dt = t_arr[i] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            t_sub[i] = time.perf_counter() - t0
            tickets[i] = ctx.submit(*m)
        lat, done = [], []
        for i, tk in enumerate(tickets):
            ctx.wait(tk, 3600)
            r = ctx.result(tk)
            lat.append(r["latency_s"])
            done.append(t_sub[i] + r["latency_s"])
    return {"rate_per_s": rate, "n": len(mols), "sustained_mol_per_s": len(mols) / (max(done) - t_sub[0]),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "protocol": "fixed 20 iterations + recheck + final step, Poisson arrivals"}


def measured_peaks(g, ctx):
    """TF32 tensor, FP32 and FP64 FMA peaks measured now by the library's
    probes (rks_probe_peak), TFLOP/s."""
    out = {}
    for name, kind in (("tf32_mma", g.RKS_PROBE_TF32_MMA), ("fp32_fma", g.RKS_PROBE_FP32_FMA),
                       ("fp64_fma", g.RKS_PROBE_FP64_FMA)):
        try:
            out[name] = ctx.probe_peak(kind) / 1e12
        except Exception as e:  # noqa: BLE001 - report, do not fail the bench
            out[name] = None
            out[name + "_error"] = str(e)[:200]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours")
    ap.add_argument("--nmol", type=int, default=4096)
    ap.add_argument("--fp64-budget-s", type=float, default=1800.0,
                    help="time allowed for the FP64 GPU comparison (every molecule when it fits; 0: none)")
    ap.add_argument("--serve-leg-n", type=int, default=1000)
    ap.add_argument("--serve-leg-rate", type=float, default=50.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-only", action="store_true", help="one step with per-stage times")
    ap.add_argument("--profile-precision", choices=("mixed", "fp64"), default="mixed",
                    help="--profile-only: the mixed path (default) or the plain FP64 path")
    ap.add_argument("--profile-iters", type=int, default=20, help="--profile-only: SCF iterations")
    ap.add_argument("--serve", action="store_true", help="Poisson serving sweep instead of the batch step")
    ap.add_argument("--serve-n", type=int, default=1500)
    ap.add_argument("--converge", action="store_true",
                    help="the batch workload under the converge protocol (retire on convergence)")
    ap.add_argument("--converge-ref-n", type=int, default=512)
    ap.add_argument("--validate", action="store_true",
                    help="mixed vs FP64 GPU on every molecule, and vs the oracle on a stratified subset")
    ap.add_argument("--oracle-n", type=int, default=96)
    ap.add_argument("--large", action="store_true",
                    help="the 20-30-heavy-atom workload (global-memory kernels, direct SCF sample)")
    ap.add_argument("--large-n", type=int, default=256)
    ap.add_argument("--large-fp64-n", type=int, default=4)
    ap.add_argument("--large-direct-n", type=int, default=8)
    ap.add_argument("--large-prof-n", type=int, default=16)
    ap.add_argument("--large-protocol", choices=("converge", "fixed"), default="converge")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 1)
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return serve_main(args)
    if args.validate:
        return validate_main(args)
    if args.converge:
        return converge_main(args)
    if args.large:
        return large_main(args)

    import torch
    import paper_2311_01135_gb300 as g

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    g.build()

    allm = workload(args.nmol * world)
    mols = [allm[i] for i in shard_indices(args.nmol, rank, world)]
    nmol = len(mols)
    ctx = g.Context(precision=g.RKS_MIXED, fixed_iters=20, recheck_err=RECHECK_ERR,
                    recheck_fp64_err=RECHECK_FP64_ERR, device=local)
    stream = torch.cuda.ExternalStream(ctx.stream())
    B = g.Batch(ctx, mols)  # H2D of the inputs happens here (outside the timed region)

    def step():
        B.setup()
        B.run()

    if args.profile_only:
        if args.profile_precision == "fp64" or args.profile_iters != 20:
            B.close()
            ctx.close()
            prec = g.RKS_FP64 if args.profile_precision == "fp64" else g.RKS_MIXED
            ctx = g.Context(precision=prec, fixed_iters=args.profile_iters, recheck_err=RECHECK_ERR,
                            recheck_fp64_err=RECHECK_FP64_ERR, device=local)
            B = g.Batch(ctx, mols)
        ctx.profile(True)
        B.setup()
        B.run()
        B.sync()
        prof = ctx.profile_read()
        print(json.dumps({"stages": prof, "nmol": nmol, "precision": args.profile_precision,
                          "iterations": args.profile_iters}, indent=1))
        return

    # W untimed warm-up steps; the last one records per-stage CUDA events
    # (stage profiling turns the iteration graph off, so it is never timed)
    for w in range(args.warmup):
        if w == args.warmup - 1:
            ctx.profile(True)
        step()
        B.sync()
    prof = ctx.profile_read()
    ctx.profile(False)

    clocks = Clocks()
    clocks.start()
    if dist:
        tdist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    B.sync()
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    ms = e0.elapsed_time(e1)
    ck = clocks.stop()
    ms_max = max_over_ranks(ms)
    ms_per_step = ms_max / args.steps
    rmx = [B.result(m) for m in range(nmol)]

    # ---- e2e through the serving API (host buffers)
    e2e = None
    if not args.no_e2e:
        h2d = sum(len(Z) * (4 + 24) for Z, _ in mols)
        d2h = 0
        t0 = time.perf_counter()
        tickets = ctx.submit_many(mols)
        for tk in tickets:
            ctx.wait(tk, 3600)
        out = [ctx.result(tk) for tk in tickets]
        t1 = time.perf_counter()
        for r in out:
            d2h += 8 * (r["nbf"] + r["nbf"] ** 2) + 96
        e2e = {"value": nmol * world / (t1 - t0), "unit": "molecules/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # ---- the accuracy gate: every molecule against the FP64 GPU path
    gate, fp64, n_fail, fp64_rate = None, None, 0, None
    if args.fp64_budget_s > 0:
        r64, fp64_rate, fp64_s = fp64_leg(g, mols, local, args.fp64_budget_s)
        gate = gate_report(rmx, r64)
        fp64 = {"value": fp64_rate, "unit": "molecules/s", "nmol": gate["n_checked"], "wall_s": fp64_s}
        n_fail = gate["n_fail"] + gate["status_not_ok"]
    value = (nmol - n_fail) * world / (ms_per_step / 1e3)  # molecules within the gate per second

    # ---- latency under Poisson arrivals (serving API)
    serve = None
    if args.serve_leg_n > 0:
        serve = serve_leg(g, mols[:args.serve_leg_n], args.serve_leg_rate, local)

    # ---- roofline of the dominant kernel
    pk = peaks()
    probes = measured_peaks(g, ctx)
    stages = {k: v for k, v in prof.items()}
    # the dominant kernel of the batch itself: the FP64 redo's stages run on a
    # stream of their own, overlap the rest and cover only its few molecules
    own = [k for k in ("grid_xc_tc", "grid_xc", "jk", "eri", "scf_step") if k in stages]
    dom = max(own or stages, key=lambda k: stages[k]["ms"])
    roof = roofline(dom, stages[dom], B, mols, pk, probes)
    others = {k: roofline(k, stages[k], B, mols, pk, probes)
              # the parent batch's kernels (the FP64 redo's stages share names with
              # the CUDA-core grid stages and cover only its few molecules)
              for k in ("jk", "grid_xc_tc", "grid_xc_tc_final", "jk_final")
              if k in stages and k != dom}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline_all_cores(mols)
    launches = sum(v["launches"] for v in stages.values()) * args.steps
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "molecules/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": workload_config(nmol, world),
                "e2e": e2e, "gpu_launches": launches, "clocks": ck, "roofline": roof, "roofline_other": others,
                "cpu_baseline": cpu, "gate": gate, "fp64_gpu": fp64,
                "mixed_vs_fp64_speedup": (nmol / (ms_per_step / 1e3)) / fp64_rate if fp64_rate else None,
                "latency_s": serve, "peaks_probed_tflops": probes,
                "stages_ms": {k: round(v["ms"], 3) for k, v in stages.items()}}
        print(json.dumps(line), flush=True)
    B.close()
    ctx.close()
    if dist:
        tdist.destroy_process_group()


def roofline(name, st, B, mols, pk, probes):
    """Algorithmic work of a stage per launch / its mean launch time, against
    the peak of the unit that bounds it."""
    import paper_2311_01135_gb300 as g
    ms = st["ms"] / max(st["launches"], 1)
    if name.startswith("grid_xc_tc"):
        # both contractions (rho: T = Phi D, V_xc: Phi^T X) over the AOs
        # significant in each 128-point block: 2 * 128 * n_sig^2 flops each,
        # summed over blocks (counted once; the 3xTF32 split issues 3 MMAs each)
        k = 9 if name.endswith("final") else 8
        flops = sum(4.0 * B.dump(m, g.RKS_DUMP_SCALARS)[k] for m in range(len(mols)))
        ach = flops / (ms / 1e3) / 1e12
        peak = probes.get("tf32_mma")
        src = "tcgen05 kind::tf32 dense, measured by rks_probe_peak in this run"
        if not peak:
            peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"]) * 1.1 / 2.25
            src = f"{pk['_source']} sustained bf16 x 1.1/2.25 (TF32 dense)"
        traffic = GRID_TC_DRAM_BYTES_PER_POINT * sum(len(Z) * 50 * 12 * 24 for Z, _ in mols) / 1e9 \
            if (name == "grid_xc_tc" and GRID_TC_DRAM_BYTES_PER_POINT) else None
        return {"kernel": name, "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": traffic, "traffic_unit": "GB per launch", "peak_source": src,
                "units": "4 * sum over 128-point blocks of 128 n_sig^2 per molecule per launch "
                         "(two contractions over the significant AOs)"}
    if name.startswith("grid_xc"):
        n = [g.rks_nbf(Z) for Z, _ in mols]
        P = [len(Z) * 50 * 12 * 24 for Z, _ in mols]
        flops = sum(4.0 * p * k * k for p, k in zip(P, n))
        peak = probes.get("fp32_fma") or 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        return {"kernel": name, "bound": "alu", "achieved": flops / (ms / 1e3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "frac": flops / (ms / 1e3) / 1e12 / peak, "traffic": None,
                "peak_source": "FP32 FMA measured by rks_probe_peak" if probes.get("fp32_fma") else "derived"}
    if name.startswith("jk"):
        nbytes = 0.0
        for m in range(len(mols)):
            sc = B.dump(m, g.RKS_DUMP_SCALARS)
            nbytes += sc[5] * 4
        return {"kernel": name, "bound": "hbm", "achieved": nbytes / (ms / 1e3) / 1e9, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": nbytes / (ms / 1e3) / 1e9 / pk["hbm_gbs"], "traffic": None,
                "peak_source": pk["_source"]}
    return {"kernel": name, "bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None,
            "traffic": None}


if __name__ == "__main__":
    main()
