"""Replica dispatcher: one batched RKS engine per GPU, on any number of hosts.

Molecules are independent (the SCF of Section 3.1 has no exchange step
between molecules), so several GPUs, on one box or on many, run as
independent replicas with no collective.  A dispatcher process holds the
molecule list; each worker process owns one GPU (one rks context) and pulls
work from the dispatcher over TCP:

* order: molecules go out largest estimated cost first (cost ~ atoms x nbf^2,
  the grid quadrature's scaling), so the last chunks are the cheapest and the
  replicas finish close together (longest-processing-time-first);
* flow: a worker keeps two chunks of `chunk` molecules in flight on its GPU
  (the next one queued while the current one runs) and asks for another as
  each finishes, so faster GPUs simply pull more;
* failure: a worker whose connection drops, or that sends nothing for
  `timeout_s` while it holds work, is dropped and its molecules go back to
  the front of the queue for the others (a result is kept once, the first
  time it arrives);
* resume: with a checkpoint file, every result is appended to it as it
  arrives (pickled, keyed by a hash of the molecule's atoms and
  coordinates), and a later run over the same molecules dispatches only
  those without a record (a record cut short by a crash is ignored).

Transport is multiprocessing.connection (TCP, HMAC challenge with a shared
auth key), meant for a trusted cluster network; messages are pickled tuples:
  worker -> dispatcher  ("want", k)                   ask for up to k molecules
                        ("done", [(i, result), ...])  results of molecules i
  dispatcher -> worker  ("work", [(i, Z, xyz), ...])
                        ("stop",)

    # dispatcher host (RKS_DISPATCH_KEY holds the shared key everywhere)
    python -m paper_2311_01135_gb300.dispatch serve --listen 0.0.0.0:7788 --workers 8 \
        --input mols.npz --output results.npz --checkpoint results.ckpt
    # each GPU (any host)
    python -m paper_2311_01135_gb300.dispatch worker --connect HOST:7788 --device 0

or from Python: Dispatcher(("0.0.0.0", 7788), authkey, n_workers=8).run(mols).

This module is host code only: every molecule a worker runs goes through the
library's serving calls (rks_submit_batch / rks_wait / rks_result).
"""
from __future__ import annotations

import argparse
import collections
import hashlib
import os
import pickle
import threading
import time
from multiprocessing.connection import Client, Listener, wait

import numpy as np


def cost_estimate(Z):
    """Relative cost of one molecule: atoms x nbf^2 (grid points scale with
    atoms, the density and V_xc contractions with nbf^2 per point)."""
    Z = np.asarray(Z)
    nbf = int(np.sum(np.where(Z > 1, 5, 1)))
    return len(Z) * nbf * nbf


def mol_key(Z, xyz):
    """Checkpoint key of a molecule: SHA-1 of its atomic numbers (int32) and
    coordinates (float64)."""
    h = hashlib.sha1()
    h.update(np.ascontiguousarray(Z, np.int32).tobytes())
    h.update(np.ascontiguousarray(xyz, np.float64).tobytes())
    return h.hexdigest()


def load_checkpoint(path, with_length=False):
    """{key: result} from an append-only checkpoint file (a trusted file:
    records are pickles); reading stops at the first incomplete record.
    with_length: also return the byte length of the complete records."""
    out, good = {}, 0
    if os.path.exists(path):
        with open(path, "rb") as f:
            while True:
                try:
                    k, r = pickle.load(f)
                except Exception:  # noqa: BLE001 - end of file, or a record cut short
                    break
                out[k] = r
                good = f.tell()
    return (out, good) if with_length else out


class Dispatcher:
    """Serves molecules to `n_workers` replicas; see the module docstring."""

    def __init__(self, address, authkey, n_workers, chunk=64, timeout_s=600.0, connect_timeout_s=60.0):
        self.listener = Listener(address, authkey=authkey)
        self.address = self.listener.address
        self.n_workers = n_workers
        self.chunk = chunk
        self.timeout_s = timeout_s
        self.connect_timeout_s = connect_timeout_s
        self._new = collections.deque()
        self._lock = threading.Lock()
        self._accepting = True
        self._acceptor = threading.Thread(target=self._accept, daemon=True)
        self._acceptor.start()
        self.stats = collections.Counter()
        self.sent = []  # molecule ids in the order they went out

    def _accept(self):
        while self._accepting:
            try:
                c = self.listener.accept()
            except Exception:  # noqa: BLE001 - listener closed, or a failed handshake
                if not self._accepting:
                    return
                continue
            with self._lock:
                self._new.append(c)

    def run(self, mols, checkpoint=None):
        """Every molecule of mols [(Z, xyz), ...] through the replicas; returns
        the results in input order.  checkpoint: path of the resume file
        (results already recorded there are not dispatched again)."""
        self._cost = [cost_estimate(Z) for Z, _ in mols]
        order = sorted(range(len(mols)), key=lambda i: -self._cost[i])
        results = [None] * len(mols)
        keys, ck = None, None
        if checkpoint:
            keys = [mol_key(Z, x) for Z, x in mols]
            done, good = load_checkpoint(checkpoint, with_length=True)
            for i, k in enumerate(keys):
                if k in done:
                    results[i] = done[k]
                    self.stats["resumed"] += 1
            # append after the last complete record (drop a record cut short)
            ck = open(checkpoint, "r+b" if os.path.exists(checkpoint) else "wb")
            ck.truncate(good)
            ck.seek(good)
        left = sum(r is None for r in results)
        queue = collections.deque(i for i in order if results[i] is None)
        # start once the expected replicas have connected (or the wait runs
        # out), so that the largest molecules spread over all of them; later
        # workers join whenever they connect
        t0 = time.monotonic()
        while left > 0 and time.monotonic() - t0 < self.connect_timeout_s:
            with self._lock:
                if len(self._new) >= self.n_workers:
                    break
            time.sleep(0.01)
        held = {}      # conn -> set of molecule ids it holds
        seen = {}      # conn -> time of its last message
        while left > 0:
            with self._lock:
                while self._new:
                    c = self._new.popleft()
                    held[c] = set()
                    seen[c] = time.monotonic()
            if not held:
                time.sleep(0.01)
                continue
            for c in wait(list(held), timeout=0.2):
                try:
                    msg = c.recv()
                except (EOFError, OSError):
                    self._drop(c, held, seen, queue, results)
                    continue
                seen[c] = time.monotonic()
                if msg[0] == "done":
                    for i, r in msg[1]:
                        held[c].discard(i)
                        if results[i] is None:
                            results[i] = r
                            left -= 1
                            self.stats["done"] += 1
                            if ck:
                                pickle.dump((keys[i], r), ck)
                                ck.flush()
                elif msg[0] == "want":
                    k = min(int(msg[1]), self.chunk)
                    out = []
                    while queue and len(out) < k:
                        i = queue.popleft()
                        if results[i] is None:
                            out.append(i)
                    held[c].update(out)
                    self.sent.extend(out)
                    try:
                        c.send(("work", [(i, np.asarray(mols[i][0], np.int32), np.asarray(mols[i][1], float))
                                         for i in out]))
                    except (EOFError, OSError):
                        self._drop(c, held, seen, queue, results)
            now = time.monotonic()
            for c in [c for c in held if held[c] and now - seen[c] > self.timeout_s]:
                self._drop(c, held, seen, queue, results)
        if ck:
            ck.close()
        with self._lock:
            idle = list(self._new)
            self._new.clear()
        for c in list(held) + idle:
            try:
                c.send(("stop",))
            except (EOFError, OSError):
                pass
        return results

    def _drop(self, c, held, seen, queue, results):
        """A worker is gone: its unfinished molecules go back to the front."""
        back = sorted((i for i in held.pop(c, ()) if results[i] is None), key=lambda i: -self._cost[i])
        queue.extendleft(reversed(back))
        seen.pop(c, None)
        self.stats["dropped_workers"] += 1
        self.stats["requeued"] += len(back)
        try:
            c.close()
        except OSError:
            pass

    def close(self):
        self._accepting = False
        try:
            self.listener.close()
        except OSError:
            pass


class EngineRunner:
    """A worker's engine: one rks context on one GPU, molecules through the
    serving calls (rks_submit_batch / rks_wait / rks_result).  submit()
    queues a chunk and returns at once; collect() waits for its results."""

    def __init__(self, device=0, **options):
        import paper_2311_01135_gb300 as g
        self.ctx = g.Context(device=device, **options)

    def submit(self, jobs):
        return [i for i, _, _ in jobs], self.ctx.submit_many([(Z, xyz) for _, Z, xyz in jobs])

    def collect(self, handle):
        ids, tickets = handle
        out = []
        for i, t in zip(ids, tickets):
            self.ctx.wait(t, 3600)
            out.append((i, self.ctx.result(t)))
        return out

    def close(self):
        self.ctx.close()


def worker_loop(address, authkey, engine, chunk=64, depth=2):
    """Pull molecules from the dispatcher at `address` until it says stop,
    with up to `depth` chunks in flight on the engine (engine.submit(jobs)
    -> handle, engine.collect(handle) -> [(i, result), ...])."""
    conn = Client(address, authkey=authkey)
    pending = collections.deque()
    try:
        while True:
            if len(pending) < depth:
                conn.send(("want", chunk))
                msg = conn.recv()
                if msg[0] == "stop":
                    return
                if msg[1]:
                    pending.append(engine.submit(msg[1]))
                    continue
                if not pending:
                    # nothing queued now (others hold the rest): ask again shortly
                    time.sleep(0.05)
                    continue
            conn.send(("done", engine.collect(pending.popleft())))
    except (EOFError, OSError):
        return
    finally:
        conn.close()


def read_molecules(path):
    """Molecules from an .npz in the batch calls' layout: natom (int32 [n]),
    Z (int32, all atoms in order), xyz (float64 [atoms, 3], bohr)."""
    f = np.load(path)
    na = np.asarray(f["natom"], np.int64)
    Z = np.asarray(f["Z"], np.int32)
    xyz = np.asarray(f["xyz"], np.float64).reshape(-1, 3)
    off = np.concatenate([[0], np.cumsum(na)])
    return [(Z[off[k]:off[k + 1]], xyz[off[k]:off[k + 1]]) for k in range(len(na))]


def write_results(path, results):
    """Results to an .npz: per molecule the scalars of rks_result_t (E, homo,
    lumo, gap, iters, nbf, status as a string), and eps and D concatenated
    with their offsets (eps_off, D_off)."""
    n = len(results)
    nbf = np.array([r["nbf"] for r in results], np.int64)
    eps_off = np.concatenate([[0], np.cumsum(nbf)])
    D_off = np.concatenate([[0], np.cumsum(nbf * nbf)])
    np.savez(path, E=np.array([r["E"] for r in results]), homo=np.array([r["homo"] for r in results]),
             lumo=np.array([r["lumo"] for r in results]), gap=np.array([r["gap"] for r in results]),
             iters=np.array([r["iters"] for r in results], np.int64), nbf=nbf,
             status=np.array([str(r["status"]) for r in results]),
             eps=np.concatenate([np.ravel(r["eps"]) for r in results]) if n else np.zeros(0),
             D=np.concatenate([np.ravel(r["D"]) for r in results]) if n else np.zeros(0),
             eps_off=eps_off, D_off=D_off)


def _key(env):
    key = os.environ.get(env, "").encode()
    if not key:
        raise SystemExit(f"set {env} to the shared auth key")
    return key


def main(argv=None):
    ap = argparse.ArgumentParser(description="RKS replicas across hosts: a dispatcher and one worker per GPU")
    sub = ap.add_subparsers(dest="cmd", required=True)
    w = sub.add_parser("worker", help="one GPU: pull molecules from a dispatcher")
    w.add_argument("--connect", required=True, help="dispatcher HOST:PORT")
    w.add_argument("--device", type=int, default=int(os.environ.get("LOCAL_RANK", "0")))
    w.add_argument("--precision", choices=("mixed", "fp64"), default="mixed")
    w.add_argument("--fixed-iters", type=int, default=20)
    w.add_argument("--chunk", type=int, default=64)
    d = sub.add_parser("serve", help="hand the molecules of --input to the workers, write --output")
    d.add_argument("--listen", required=True, help="HOST:PORT to accept workers on")
    d.add_argument("--workers", type=int, required=True, help="replicas to wait for before starting")
    d.add_argument("--input", required=True, help=".npz with natom, Z, xyz (bohr)")
    d.add_argument("--output", required=True, help=".npz of the results, input order")
    d.add_argument("--checkpoint", default=None, help="resume file (results recorded there are not redone)")
    d.add_argument("--chunk", type=int, default=64)
    d.add_argument("--timeout-s", type=float, default=600.0)
    for p in (w, d):
        p.add_argument("--authkey-env", default="RKS_DISPATCH_KEY")
    a = ap.parse_args(argv)
    key = _key(a.authkey_env)
    if a.cmd == "serve":
        host, port = a.listen.rsplit(":", 1)
        mols = read_molecules(a.input)
        disp = Dispatcher((host, int(port)), key, n_workers=a.workers, chunk=a.chunk, timeout_s=a.timeout_s)
        try:
            res = disp.run(mols, checkpoint=a.checkpoint)
        finally:
            disp.close()
        write_results(a.output, res)
        return
    host, port = a.connect.rsplit(":", 1)
    import paper_2311_01135_gb300 as g
    eng = EngineRunner(device=a.device, precision=g.RKS_MIXED if a.precision == "mixed" else g.RKS_FP64,
                       fixed_iters=a.fixed_iters)
    try:
        worker_loop((host, int(port)), key, eng, chunk=a.chunk)
    finally:
        eng.close()


if __name__ == "__main__":
    main()
