"""Serving path (continuous batching) on the GPU, through the C ABI.

* A molecule's result does not depend on its company: alone, in a batch, in a
  serving cohort of any size.  The mixed path accumulates J/K/V_xc/E_xc in
  64-bit fixed point in every pass (integer atomics: the sum is independent
  of arrival order) and the grid kernel is chosen per molecule, so its
  results are bit-identical in any company: gate 0.  The FP64 path's FP64
  atomics reorder at ~1e-16 relative: |dE| <= 1e-10 Ha, |d gap| <= 1e-9 Ha,
  max|dD| <= 1e-8.
* Every served molecule agrees with the FP64 oracle (Section 3.1, Eq. 1) at the
  method's tolerances (|dE| <= 1e-5 Ha mixed, 1e-8 FP64).
* Host-side failure paths: a molecule larger than the HBM budget fails with
  RKS_ENOMEM, the converge protocol reports not-converged at max_iters, and
  destroying a context with work in flight returns.
"""
import threading
import time

import numpy as np
import pytest

import molgen

pytestmark = pytest.mark.gpu

g = pytest.importorskip("paper_2311_01135_gb300")


@pytest.fixture(scope="module")
def mols():
    return molgen.batch(11, 6, 1, 3)


@pytest.fixture(scope="module")
def oracle_refs(mols):
    from oracle import scf
    return [scf.run_scf(scf.System(Z, x)) for Z, x in mols]


def _batch(ctx, ms):
    with g.Batch(ctx, ms) as B:
        B.run()
        B.sync()
        return [B.result(m) for m in range(len(ms))]


def _serve(ctx, ms, stagger_s=0.0):
    tickets = []
    for Z, x in ms:
        tickets.append(ctx.submit(Z, x))
        if stagger_s:
            time.sleep(stagger_s)
    for t in tickets:
        ctx.wait(t, 600)
    return [ctx.result(t) for t in tickets]


def _same(a, b, tol_e, tol_gap, tol_d=None):
    assert a["status"] == b["status"]
    assert abs(a["E"] - b["E"]) <= tol_e, (a["E"], b["E"])
    assert abs(a["gap"] - b["gap"]) <= tol_gap
    if tol_d is not None:
        assert np.max(np.abs(a["D"] - b["D"])) <= tol_d


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_alone_and_in_the_mix(mols, prec):
    """Molecule 0 alone, in a batch with five others, and served in cohorts."""
    opts = dict(precision=g.RKS_FP64) if prec == "fp64" else dict(precision=g.RKS_MIXED, fixed_iters=20)
    tol = (1e-10, 1e-9, 1e-8) if prec == "fp64" else (0.0, 0.0, 0.0)
    with g.Context(**opts) as c:
        alone = _batch(c, mols[:1])[0]
        mix = _batch(c, list(reversed(mols)))
        _same(alone, mix[-1], *tol)
    with g.Context(max_slots=2, admit_wait_us=0, **opts) as c:
        served = _serve(c, mols)
    _same(alone, served[0], *tol)
    for a, b in zip(served, reversed(mix)):
        _same(a, b, *tol)


def test_served_results_match_oracle(mols, oracle_refs):
    with g.Context(precision=g.RKS_MIXED, fixed_iters=20, max_cohorts=3, admit_wait_us=0, max_slots=4) as c:
        got = _serve(c, mols, stagger_s=0.01)
    for r, o in zip(got, oracle_refs):
        assert r["status"] == "ok"
        assert abs(r["E"] - o["E"]) < 1e-5
        assert abs(r["gap"] - o["gap"]) < 1e-4
        assert r["latency_s"] > 0
    with g.Context(precision=g.RKS_FP64) as c:
        got = _serve(c, mols)
    for r, o in zip(got, oracle_refs):
        assert r["status"] == "ok"
        assert abs(r["E"] - o["E"]) < 1e-8
        assert np.max(np.abs(r["eps"] - o["eps"])) < 1e-8


def test_back_fill_under_a_small_budget(mols):
    """A 12 MB budget holds one or two of these molecules (about 6 MB each in FP64): the
    queue drains by retire + back-fill, and every result is still right."""
    with g.Context(precision=g.RKS_FP64) as c:
        ref = _batch(c, mols)
    with g.Context(precision=g.RKS_FP64, hbm_budget_bytes=12 << 20) as c:
        got = _serve(c, mols)
    for a, b in zip(got, ref):
        _same(a, b, 1e-10, 1e-9, 1e-8)


def test_submit_from_threads(mols):
    with g.Context(precision=g.RKS_MIXED, fixed_iters=20, admit_wait_us=1000) as c:
        out = {}

        def client(k):
            Z, x = mols[k]
            t = c.submit(Z, x)
            c.wait(t, 600)
            out[k] = c.result(t)

        th = [threading.Thread(target=client, args=(k,)) for k in range(len(mols))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        ref = _batch(c, mols)
    for k in range(len(mols)):
        _same(out[k], ref[k], 0.0, 0.0, 0.0)  # mixed: bit-identical


def test_molecule_over_budget_fails_with_enomem():
    Z, x = molgen.h2o()
    with g.Context(precision=g.RKS_FP64, hbm_budget_bytes=1 << 16) as c:
        t = c.submit(Z, x)
        c.wait(t, 60)
        assert c.poll(t) == g.RKS_FAILED
        with pytest.raises(g.RKSError) as e:
            c.result(t)
        assert e.value.code == g.RKS_ENOMEM


def test_not_converged_status():
    Z, x = molgen.h2o()
    with g.Context(precision=g.RKS_FP64, max_iters=2) as c:
        r = _serve(c, [(Z, x)])[0]
        assert r["status"] == "not_converged" and r["iters"] == 2
        b = _batch(c, [(Z, x)])[0]
        assert b["status"] == "not_converged"


def test_submit_validation_and_destroy_with_work_in_flight(mols):
    c = g.Context(precision=g.RKS_MIXED, fixed_iters=20)
    with pytest.raises(g.RKSError) as e:
        c.submit([1, 1, 1], np.zeros((3, 3)))  # odd electron count
    assert e.value.code == g.RKS_EINVAL
    tickets = c.submit_many(mols * 4)
    assert len(set(tickets)) == len(mols) * 4
    t0 = time.time()
    c.close()  # in-flight and queued tickets are failed, not waited for
    assert time.time() - t0 < 120


def test_bounded_wait_gives_up_and_context_survives():
    """The device-side failure path, without a fault: a bounded wait on an
    mbarrier nothing arrives at returns RKS_EDEVICE, and the same context
    then runs a molecule normally."""
    Z, x = molgen.h2o()
    with g.Context(precision=g.RKS_MIXED, fixed_iters=20) as c:
        assert c.selftest_bounded_wait(100000) == g.RKS_EDEVICE
        assert c.selftest_bounded_wait(0) == g.RKS_EINVAL
        r = _serve(c, [(Z, x)])[0]
        assert r["status"] == "ok"
