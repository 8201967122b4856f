"""Writes large_20heavy_oracle.json: FP64 oracle values for one seeded
20-heavy-atom molecule (the larger-molecule workload: 20-30 heavy atoms,
basis above the shared-memory kernels' 96 functions).

    python tests/golden/make_large_golden.py

Calls only oracle/ (and the seeded generator molgen/, which holds none of the
method's arithmetic).  The oracle at this size takes a few minutes on a
handful of cores (the full N^4 tensor is ~2 GB), too long for a test, so
the values are stored: the GPU parity test compares against them.

Stored per matrix M (J, K_std and V_xc at the initial density D0, the output
density D of the whole run): its Frobenius norm, tr(D0 M), the bilinear
probe u^T M v with u, v = rng(12345).standard_normal(nbf) (first u, then v),
and the entries at 256 sampled (i, j) positions (rng(777) integers).
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import molgen  # noqa: E402
from oracle import scf  # noqa: E402

SEED, HEAVY = 4, 20
OUT = os.path.join(HERE, "large_20heavy_oracle.json")


def probes(n):
    rng = np.random.default_rng(12345)
    u = rng.standard_normal(n)
    v = rng.standard_normal(n)
    idx = np.random.default_rng(777).integers(0, n, size=(256, 2))
    return u, v, idx


def summary(M, D0, u, v, idx):
    return dict(fro=float(np.linalg.norm(M)), trD0=float(np.sum(D0 * M)), uMv=float(u @ M @ v),
                samples=[float(M[i, j]) for i, j in idx])


def main():
    Z, xyz = molgen.batch(SEED, 1, HEAVY, HEAVY)[0]
    t0 = time.time()
    s = scf.System(Z, xyz)
    t1 = time.time()
    n = s.nbf
    u, v, idx = probes(n)
    D0 = s.sad_guess()
    F0, E0, p0 = s.fock(D0)
    t2 = time.time()
    r = scf.run_scf(s, protocol="fixed", n_iter=20)
    t3 = time.time()
    out = dict(
        source="oracle/ (FP64), written by tests/golden/make_large_golden.py",
        molecule=dict(generator="molgen.batch", seed=SEED, n_mol=1, heavy_min=HEAVY, heavy_max=HEAVY, index=0,
                      Z=[int(z) for z in Z], xyz_sum=float(np.sum(xyz)), nbf=n),
        probe_seed=12345, sample_seed=777, sample_idx=[[int(i), int(j)] for i, j in idx],
        d0=dict(E=float(E0), Exc=float(p0["Exc"]), J=summary(p0["J"], D0, u, v, idx),
                K=summary(p0["K"], D0, u, v, idx), Vxc=summary(p0["Vxc"], D0, u, v, idx)),
        fixed20=dict(E=float(r["E"]), homo=r["homo"], lumo=r["lumo"], gap=r["gap"], max_err=r["max_err"],
                     eps=[float(e) for e in r["eps"]], D=summary(r["D"], D0, u, v, idx)),
        oracle_seconds=dict(setup=t1 - t0, fock_d0=t2 - t1, scf=t3 - t2),
    )
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(f"nbf {n}: E0 {E0:.10f}  E(20) {r['E']:.10f}  gap {r['gap']:.8f}  "
          f"max_err {r['max_err']:.2e}  times {t1 - t0:.0f}/{t2 - t1:.0f}/{t3 - t2:.0f} s")


if __name__ == "__main__":
    main()
