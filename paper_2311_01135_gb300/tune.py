"""Autotuner for the launch shapes of the two per-iteration kernels.

    python -m paper_2311_01135_gb300.tune --nmol 512 [--precision mixed] [--workload large] [--out tuned.json]

For each candidate count of thread blocks per molecule it runs the batch
(setup + 2 SCF iterations + final step) once to warm up, once with stage
profiling, and keeps the fastest per kernel.  The two choices are independent:
J/K results are bit-identical for any block count, so only its time matters.
The grid count changes the grouping of the V_xc sums (results move at
~1e-7), so it is a per-deployment setting (rks_options.grid_chunks), not
a per-batch one: a molecule must not change with its company.  The library's
defaults (grid 16, J/K 8) are this tuner's choice on 512 molecules of the
9-11-heavy-atom workload on a GB300.

--workload large tunes the kernels of molecules above 96 basis functions
(20-30 heavy atoms: `grid_large`, `jk_large`) instead.  --out appends the
choice to a JSON file keyed by device, precision and workload, which
`load_choice` reads back as Context options.
"""
from __future__ import annotations

import argparse
import json
import os

from . import RKS_FP64, RKS_MIXED, Batch, Context

GRID_CANDIDATES = (4, 8, 16, 32)
JK_CANDIDATES = (1, 2, 4, 8, 16)
# stage names of the two kernels per workload and precision
STAGES = {("small", RKS_MIXED): ("grid_xc_tc", "jk"), ("small", RKS_FP64): ("grid_xc", "jk"),
          ("large", RKS_MIXED): ("grid_large", "jk_large"), ("large", RKS_FP64): ("grid_large", "jk_large")}


def _stage_ms(mols, precision, grid_chunks, jk_chunks):
    with Context(precision=precision, fixed_iters=2, grid_chunks=grid_chunks, jk_chunks=jk_chunks) as c:
        with Batch(c, mols) as B:
            B.run()
            B.sync()
            c.profile(True)
            B.setup()
            B.run()
            B.sync()
            prof = c.profile_read()
    return {k: v["ms"] for k, v in prof.items()}


def tune(mols, precision=RKS_MIXED, grid_candidates=GRID_CANDIDATES, jk_candidates=JK_CANDIDATES,
         workload="small", measure=_stage_ms):
    """Return {"grid_chunks": g, "jk_chunks": j, "grid_ms": {...}, "jk_ms": {...}}.
    measure(mols, precision, grid_chunks, jk_chunks) -> {stage: ms}."""
    grid_key, jk_key = STAGES[(workload, precision)]
    grid_ms, jk_ms = {}, {}
    for gc in grid_candidates:
        st = measure(mols, precision, gc, jk_candidates[0])
        grid_ms[gc] = st.get(grid_key, st.get("grid_xc", float("inf")))
    for jc in jk_candidates:
        st = measure(mols, precision, grid_candidates[0], jc)
        jk_ms[jc] = st.get(jk_key, float("inf"))
    return {"grid_chunks": min(grid_ms, key=grid_ms.get), "jk_chunks": min(jk_ms, key=jk_ms.get),
            "grid_ms": grid_ms, "jk_ms": jk_ms}


def _key(device, precision, workload):
    return f"{device}|{'mixed' if precision == RKS_MIXED else 'fp64'}|{workload}"


def save_choice(path, device, precision, workload, res):
    """Merge one tuning result into the JSON file at path."""
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[_key(device, precision, workload)] = {"grid_chunks": res["grid_chunks"], "jk_chunks": res["jk_chunks"]}
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def load_choice(path, device, precision, workload="small"):
    """Context options ({"grid_chunks", "jk_chunks"}) tuned for this device,
    precision and workload, or {} when the file has none."""
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return dict(json.load(f).get(_key(device, precision, workload), {}))


def _device_name(index=0):
    import subprocess
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=name", "--format=csv,noheader", "-i", str(index)],
                             capture_output=True, text=True, timeout=30).stdout.strip()
    except (OSError, subprocess.SubprocessError):
        out = ""
    return out or "unknown"


def main():
    import molgen
    ap = argparse.ArgumentParser()
    ap.add_argument("--nmol", type=int, default=512)
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--precision", choices=("mixed", "fp64"), default="mixed")
    ap.add_argument("--workload", choices=("small", "large"), default="small",
                    help="small: 9-11 heavy atoms (seed 2); large: 20-30 heavy atoms (seed 4)")
    ap.add_argument("--out", default=None, help="JSON file to record the choice in")
    args = ap.parse_args()
    if args.workload == "large":
        mols = molgen.batch(4 if args.seed is None else args.seed, args.nmol, 20, 30)
    else:
        mols = molgen.batch(2 if args.seed is None else args.seed, args.nmol, 9, 11)
    prec = RKS_MIXED if args.precision == "mixed" else RKS_FP64
    res = tune(mols, prec, workload=args.workload)
    if args.out:
        save_choice(args.out, _device_name(), prec, args.workload, res)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
