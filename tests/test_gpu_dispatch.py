"""The replica dispatcher with the real engine: one worker process on cuda:0
(an rks context fed through the serving calls) pulls the molecules from a
dispatcher in this process over TCP.  Its results equal a batch run of the
same molecules bit for bit on the mixed path (fixed-point sums: a molecule's
result does not depend on its company or on the path that ran it)."""
import multiprocessing as mp

import numpy as np
import pytest

import molgen

pytestmark = pytest.mark.gpu
g = pytest.importorskip("paper_2311_01135_gb300")
from paper_2311_01135_gb300 import dispatch  # noqa: E402

KEY = b"gpu-dispatch-test"
OPTS = dict(fixed_iters=20)


def _gpu_worker(address):
    eng = dispatch.EngineRunner(device=0, precision=g.RKS_MIXED, **OPTS)
    try:
        dispatch.worker_loop(address, KEY, eng, chunk=3)
    finally:
        eng.close()


def test_dispatched_results_equal_the_batch_run():
    mols = molgen.batch(11, 7, 1, 4)
    d = dispatch.Dispatcher(("127.0.0.1", 0), KEY, n_workers=1, chunk=3, timeout_s=600.0)
    p = mp.get_context("spawn").Process(target=_gpu_worker, args=(d.address,))
    p.start()
    try:
        res = d.run(mols)
    finally:
        d.close()
        p.join(timeout=120)
        if p.is_alive():
            p.kill()
            p.join()
    assert p.exitcode == 0
    with g.Context(precision=g.RKS_MIXED, **OPTS) as c, g.Batch(c, mols) as B:
        B.run()
        B.sync()
        ref = [B.result(k) for k in range(len(mols))]
    for a, b in zip(res, ref):
        assert a["status"] == b["status"] == "ok"
        assert a["E"] == b["E"] and a["gap"] == b["gap"]
        assert np.array_equal(a["D"], b["D"])
