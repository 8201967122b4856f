"""Autotuner for the launch shapes of the two per-iteration kernels.

    python -m paper_2311_01135_gb300.tune --nmol 512 [--precision mixed]

For each candidate count of thread blocks per molecule it runs the batch
(setup + 2 SCF iterations + final step) once to warm up, once with stage
profiling, and keeps the fastest per kernel.  The two choices are independent:
J/K results are bit-identical for any block count, so only its time matters.
The grid count changes the grouping of the V_xc sums (results move at
~1e-7), so it is a per-deployment setting (rks_options.grid_chunks), not
a per-batch one: a molecule must not change with its company.  The library's
defaults (grid 16, J/K 8) are this tuner's choice on 512 molecules of the
9-11-heavy-atom workload on a GB300.
"""
from __future__ import annotations

import argparse
import json

from . import RKS_FP64, RKS_MIXED, Batch, Context

GRID_CANDIDATES = (4, 8, 16, 32)
JK_CANDIDATES = (1, 2, 4, 8, 16)


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


def tune(mols, precision=RKS_MIXED, grid_candidates=GRID_CANDIDATES, jk_candidates=JK_CANDIDATES):
    """Return {"grid_chunks": g, "jk_chunks": j, "grid_ms": {...}, "jk_ms": {...}}."""
    grid_key = "grid_xc_tc" if precision == RKS_MIXED else "grid_xc"
    grid_ms, jk_ms = {}, {}
    for gc in grid_candidates:
        st = _stage_ms(mols, precision, gc, jk_candidates[0])
        grid_ms[gc] = st.get(grid_key, st.get("grid_xc", float("inf")))
    for jc in jk_candidates:
        st = _stage_ms(mols, precision, grid_candidates[0], jc)
        jk_ms[jc] = st.get("jk", float("inf"))
    return {"grid_chunks": min(grid_ms, key=grid_ms.get), "jk_chunks": min(jk_ms, key=jk_ms.get),
            "grid_ms": grid_ms, "jk_ms": jk_ms}


def main():
    import molgen
    ap = argparse.ArgumentParser()
    ap.add_argument("--nmol", type=int, default=512)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--precision", choices=("mixed", "fp64"), default="mixed")
    args = ap.parse_args()
    mols = molgen.batch(args.seed, args.nmol, 9, 11)
    res = tune(mols, RKS_MIXED if args.precision == "mixed" else RKS_FP64)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
