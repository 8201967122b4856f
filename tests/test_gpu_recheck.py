"""The mixed path's recheck on the molecules of the benchmark workload (seed 2,
9-11 heavy atoms) that are hardest for it after the fixed 20 iterations:

* tier 1 (DIIS error 1e-4 .. 3e-4): run again from the initial guess with
  every Fock build at the final step's precision -- molecules 2018 and 1724;
* tier 2 (DIIS error above 3e-4: the SCF has not converged; paper Section 3.2,
  "Numerical Error", takes float32 results for converged molecules only and
  recomputes the rest in float64): redone on the FP64 path -- molecules 2927
  (DIIS error 0.4, energies still jumping by Ha), 2955, 2998 (DIIS error
  3.8e-4, whose precise rerun missed the FP64 gap by 1.2e-4 Ha) and 901.

Gate on each against the plain FP64 GPU path (the parity tests pin that one
to the oracle at 1e-8 Ha), and for 2955 against the FP64 oracle itself:
|dE| <= 1e-5 Ha, |d gap| <= 1e-4 Ha.  A tier-1 molecule gives the same bits
alone and in the batch (every pass sums in exact fixed point); a tier-2
molecule's FP64 redo sums in FP64 atomics, alone vs in the batch <= 1e-8 Ha.
"""
import numpy as np
import pytest

import molgen

pytestmark = pytest.mark.gpu
g = pytest.importorskip("paper_2311_01135_gb300")

TIER1 = (2018, 1724)
TIER2 = (2927, 2955, 2998, 901)


@pytest.fixture(scope="module")
def mols():
    ms = molgen.batch(2, max(TIER1 + TIER2) + 1, 9, 11)
    return [ms[i] for i in TIER1 + TIER2]


@pytest.fixture(scope="module")
def runs(mols):
    out = {}
    with g.Context(precision=g.RKS_FP64, fixed_iters=20) as c, g.Batch(c, mols) as B:
        B.run()
        B.sync()
        out["fp64"] = [B.result(m) for m in range(len(mols))]
    with g.Context(precision=g.RKS_MIXED, fixed_iters=20) as c:
        with g.Batch(c, mols) as B:
            B.run()
            B.sync()
            out["mixed"] = [B.result(m) for m in range(len(mols))]
        alone = {}
        for k in (0, len(TIER1)):  # one molecule of each tier, alone
            with g.Batch(c, [mols[k]]) as B:
                B.run()
                B.sync()
                alone[k] = B.result(0)
        out["alone"] = alone
    return out


def test_tiers_and_gate(runs):
    for k, (a, b) in enumerate(zip(runs["mixed"], runs["fp64"])):
        want = 1 if k < len(TIER1) else 2
        print((TIER1 + TIER2)[k], a["rechecked"], a["E"] - b["E"], a["gap"] - b["gap"], b["err_max"])
        assert a["rechecked"] == want
        assert a["status"] == "ok" and b["status"] == "ok"
        assert abs(a["E"] - b["E"]) <= 1e-5
        assert abs(a["gap"] - b["gap"]) <= 1e-4


def test_alone_and_in_the_batch(runs):
    t1, t2 = runs["alone"][0], runs["alone"][len(TIER1)]
    assert t1["rechecked"] == 1 and t2["rechecked"] == 2
    assert t1["E"] == runs["mixed"][0]["E"] and np.array_equal(t1["D"], runs["mixed"][0]["D"])
    assert abs(t2["E"] - runs["mixed"][len(TIER1)]["E"]) <= 1e-8


def test_fp64_redo_against_the_oracle(runs):
    from oracle import scf
    k = len(TIER1) + TIER2.index(2955)
    Z, xyz = molgen.batch(2, 2956, 9, 11)[2955]
    o = scf.run_scf(scf.System(Z, xyz), protocol="fixed", n_iter=20)
    r = runs["mixed"][k]
    assert r["rechecked"] == 2
    assert abs(r["E"] - o["E"]) <= 1e-5
    assert abs(r["gap"] - o["gap"]) <= 1e-4


def test_back_to_back_runs(mols):
    """Runs enqueued one after the other without waiting (as a benchmark's
    timed loop does): each run releases the previous run's FP64 redo batch,
    whose results the previous run's last kernel may still be reading on the
    batch's stream; the release waits for that stream.  The results of the
    last run equal those of a single run."""
    sub = [mols[0], mols[len(TIER1)]]  # one molecule of each tier
    with g.Context(precision=g.RKS_MIXED, fixed_iters=20) as c, g.Batch(c, sub) as B:
        for _ in range(3):
            B.setup()
            B.run()
        B.sync()
        rep = [B.result(m) for m in range(len(sub))]
    with g.Context(precision=g.RKS_MIXED, fixed_iters=20) as c, g.Batch(c, sub) as B:
        B.run()
        B.sync()
        one = [B.result(m) for m in range(len(sub))]
    assert [r["rechecked"] for r in rep] == [1, 2]
    assert rep[0]["E"] == one[0]["E"]
    assert abs(rep[1]["E"] - one[1]["E"]) <= 1e-8
