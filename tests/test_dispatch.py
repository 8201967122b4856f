"""The replica dispatcher (paper_2311_01135_gb300/dispatch.py) on the CPU:
worker processes on this host stand in for GPUs on other boxes, with a
stand-in engine that answers each molecule with a value computed from its
atoms (the real engine is the library's serving API, covered by the GPU
tests).  Checked: every molecule is answered once, in input order, by the
replica that ran it; molecules go out largest estimated cost first; a worker
that dies with work in hand, or stops answering, loses that work to the
others and the run still completes."""
import multiprocessing as mp
import os
import time

import numpy as np
import pytest

import molgen
from paper_2311_01135_gb300 import dispatch

KEY = b"test-dispatch-key"


class FakeEngine:
    """Answers molecule i with a value of its atoms; `die_after` chunks
    submitted it exits the process, `hang_after` it stops answering."""

    def __init__(self, die_after=None, hang_after=None):
        self.n = 0
        self.die_after = die_after
        self.hang_after = hang_after

    def submit(self, jobs):
        self.n += 1
        if self.die_after is not None and self.n > self.die_after:
            os._exit(3)
        return [(i, {"E": -float(np.sum(Z)) - 1e-3 * float(np.sum(xyz)), "pid": os.getpid()}) for i, Z, xyz in jobs]

    def collect(self, handle):
        if self.hang_after is not None and self.n > self.hang_after:
            time.sleep(120)
        time.sleep(0.01)
        return handle


def _worker(address, die_after=None, hang_after=None, chunk=4):
    dispatch.worker_loop(address, KEY, FakeEngine(die_after, hang_after), chunk=chunk)


def _expected(mol):
    Z, xyz = mol
    return -float(np.sum(Z)) - 1e-3 * float(np.sum(xyz))


@pytest.fixture()
def mols():
    return molgen.batch(5, 40, 1, 6)


def _run(mols, workers, timeout_s=60.0, checkpoint=None):
    d = dispatch.Dispatcher(("127.0.0.1", 0), KEY, n_workers=len(workers), chunk=4, timeout_s=timeout_s)
    ctx = mp.get_context("spawn")
    ps = [ctx.Process(target=_worker, args=(d.address,) + w) for w in workers]
    for p in ps:
        p.start()
    try:
        res = d.run(mols, checkpoint=checkpoint)
    finally:
        d.close()
        for p in ps:
            p.join(timeout=20)
            if p.is_alive():
                p.kill()
                p.join()
    return d, res, ps


def test_two_workers_answer_every_molecule_once(mols):
    d, res, ps = _run(mols, [(), ()])
    assert all(r is not None for r in res)
    for m, r in zip(mols, res):
        assert r["E"] == _expected(m)
    assert d.stats["done"] == len(mols) and d.stats["dropped_workers"] == 0
    assert len({r["pid"] for r in res}) == 2  # both replicas took work
    # every molecule went out once, largest estimated cost first
    assert sorted(d.sent) == list(range(len(mols)))
    costs = [dispatch.cost_estimate(mols[i][0]) for i in d.sent]
    assert all(a >= b for a, b in zip(costs, costs[1:]))
    assert all(p.exitcode == 0 for p in ps)


def test_cost_estimate():
    # water: 3 atoms x 7^2; benzene-sized C6H6: 12 atoms x 36^2
    assert dispatch.cost_estimate([8, 1, 1]) == 3 * 49
    assert dispatch.cost_estimate([6] * 6 + [1] * 6) == 12 * 36 * 36


def test_worker_that_dies_loses_its_work_to_the_other(mols):
    d, res, ps = _run(mols, [(1, None), ()])
    assert all(r is not None for r in res)
    for m, r in zip(mols, res):
        assert r["E"] == _expected(m)
    assert d.stats["dropped_workers"] == 1 and d.stats["requeued"] >= 1
    assert sorted(p.exitcode for p in ps) == [0, 3]


def test_silent_worker_is_dropped_after_the_timeout(mols):
    t0 = time.monotonic()
    d, res, ps = _run(mols, [(None, 1), ()], timeout_s=2.0)
    assert all(r is not None for r in res)
    for m, r in zip(mols, res):
        assert r["E"] == _expected(m)
    assert d.stats["dropped_workers"] == 1
    assert time.monotonic() - t0 < 60


def test_checkpoint_resumes_without_redoing_work(mols, tmp_path):
    ck = str(tmp_path / "results.ckpt")
    d1, res1, _ = _run(mols, [(), ()], checkpoint=ck)
    assert d1.stats["done"] == len(mols)
    # a second run over the same molecules finds every result recorded
    d2, res2, _ = _run(mols, [], checkpoint=ck)
    assert d2.sent == [] and d2.stats["resumed"] == len(mols)
    assert [r["E"] for r in res2] == [r["E"] for r in res1]


def test_checkpoint_cut_short_redoes_only_the_missing(mols, tmp_path):
    ck = str(tmp_path / "results.ckpt")
    _run(mols, [(), ()], checkpoint=ck)
    # keep the first 10 records and half of the 11th, as a crash would
    import pickle
    with open(ck, "rb") as f:
        ends = []
        while True:
            try:
                pickle.load(f)
            except EOFError:
                break
            ends.append(f.tell())
    with open(ck, "rb") as f:
        blob = f.read()
    with open(ck, "wb") as f:
        f.write(blob[:ends[9] + (ends[10] - ends[9]) // 2])
    kept = dispatch.load_checkpoint(ck)
    assert len(kept) == 10
    d, res, ps = _run(mols, [()], checkpoint=ck)
    assert d.stats["resumed"] == 10 and len(d.sent) == len(mols) - 10
    for m, r in zip(mols, res):
        assert r["E"] == _expected(m)
    assert len(dispatch.load_checkpoint(ck)) == len(mols)


class FullFakeEngine:
    """Stand-in answering with every field the command line writes."""

    def submit(self, jobs):
        out = []
        for i, Z, xyz in jobs:
            n = int(np.sum(np.where(np.asarray(Z) > 1, 5, 1)))
            e = _expected((Z, xyz))
            out.append((i, {"E": e, "homo": -0.3, "lumo": 0.1, "gap": 0.4, "iters": 20, "nbf": n,
                            "status": "ok", "eps": np.arange(n, dtype=float) + e,
                            "D": np.full((n, n), float(i))}))
        return out

    def collect(self, handle):
        return handle


def _full_worker(address):
    dispatch.worker_loop(address, KEY, FullFakeEngine(), chunk=4)


def test_command_line_serve_round_trip(mols, tmp_path):
    import socket
    import subprocess
    import sys
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    na = np.array([len(Z) for Z, _ in mols], np.int32)
    np.savez(tmp_path / "in.npz", natom=na, Z=np.concatenate([Z for Z, _ in mols]).astype(np.int32),
             xyz=np.concatenate([x for _, x in mols]))
    env = dict(os.environ, RKS_DISPATCH_KEY=KEY.decode())
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    srv = subprocess.Popen([sys.executable, "-m", "paper_2311_01135_gb300.dispatch", "serve",
                            "--listen", f"127.0.0.1:{port}", "--workers", "2", "--input", str(tmp_path / "in.npz"),
                            "--output", str(tmp_path / "out.npz"), "--chunk", "4"], env=env, cwd=root)
    ctx = mp.get_context("spawn")
    ps = []
    try:
        time.sleep(1.0)
        deadline = time.monotonic() + 60
        while True:  # the listener may take a moment to come up (a bare TCP
            # connect fails the auth handshake and is not counted as a worker)
            try:
                socket.create_connection(("127.0.0.1", port), timeout=1).close()
                break
            except OSError:
                assert time.monotonic() < deadline
                time.sleep(0.2)
        ps = [ctx.Process(target=_full_worker, args=(("127.0.0.1", port),)) for _ in range(2)]
        for p in ps:
            p.start()
        assert srv.wait(timeout=120) == 0
    finally:
        if srv.poll() is None:
            srv.kill()
        for p in ps:
            p.join(timeout=20)
            if p.is_alive():
                p.kill()
    out = np.load(tmp_path / "out.npz")
    assert len(out["E"]) == len(mols)
    for k, m in enumerate(mols):
        assert out["E"][k] == _expected(m)
        n = int(out["nbf"][k])
        e = out["eps"][out["eps_off"][k]:out["eps_off"][k + 1]]
        D = out["D"][out["D_off"][k]:out["D_off"][k + 1]].reshape(n, n)
        assert np.array_equal(e, np.arange(n) + _expected(m)) and np.all(D == k)
    assert set(out["status"]) == {"ok"}
