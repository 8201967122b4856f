"""Batched closed-shell Kohn-Sham (B3LYP/STO-3G) SCF on one GB300.

Thin ctypes binding over the C ABI in include/rks.h (same names).  Argument
marshalling only: every step of the method runs in the CUDA library
(paper_2311_01135_gb300/_lib/librks.so, built by `_build.build()`).  There is
no CPU fallback: importing the binding without the compiled library, or
calling it without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import LIB, build  # noqa: F401

RKS_OK, RKS_EINVAL, RKS_ENOMEM, RKS_EAGAIN, RKS_ENOTREADY = 0, -1, -2, -3, -4
RKS_ECUDA, RKS_ETIMEOUT, RKS_ENOTFOUND, RKS_EDEVICE = -5, -6, -7, -8
RKS_PENDING, RKS_RUNNING, RKS_DONE, RKS_FAILED = 0, 1, 2, 3
RKS_FP64, RKS_MIXED = 0, 1
RKS_GUESS_SAD, RKS_GUESS_CORE = 0, 1
RKS_ITER_JK_FINAL, RKS_ITER_GRID_FINAL = 1, 2
RKS_PROBE_FP32_FMA, RKS_PROBE_FP64_FMA, RKS_PROBE_TF32_MMA = 0, 1, 2
RKS_XC_NOALLOC_MAX = 65536
RKS_MAX_NBF = 224
RKS_DIRECT_NEVER, RKS_DIRECT_ALWAYS, RKS_DIRECT_AUTO = 0, 1, 2
RKS_STATUS = {0: "ok", 1: "not_converged", 2: "nonfinite", 3: "s_ill", 4: "eigh"}
(RKS_DUMP_PAIRS, RKS_DUMP_PAIR_Q, RKS_DUMP_ROW_OFF, RKS_DUMP_STORE, RKS_DUMP_S, RKS_DUMP_T, RKS_DUMP_V,
 RKS_DUMP_GRID, RKS_DUMP_J, RKS_DUMP_K, RKS_DUMP_VXC, RKS_DUMP_D, RKS_DUMP_F, RKS_DUMP_EPS, RKS_DUMP_X,
 RKS_DUMP_SCALARS, RKS_DUMP_QUARTETS) = range(17)


class rks_options(ctypes.Structure):
    _fields_ = [("basis", ctypes.c_int32), ("n_rad", ctypes.c_int32), ("n_theta", ctypes.c_int32),
                ("n_phi", ctypes.c_int32), ("becke_iters", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("fixed_iters", ctypes.c_int32), ("max_iters", ctypes.c_int32), ("e_tol", ctypes.c_double),
                ("err_tol", ctypes.c_double), ("diis_space", ctypes.c_int32),
                ("coords_in_angstrom", ctypes.c_int32), ("xc", ctypes.c_int32), ("max_slots", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_uint64), ("device", ctypes.c_int32),
                ("use_graphs", ctypes.c_int32), ("pad0", ctypes.c_int32), ("fix_theta", ctypes.c_double),
                ("grid_tc", ctypes.c_int32), ("guess", ctypes.c_int32),
                ("max_cohorts", ctypes.c_int32), ("admit_wait_us", ctypes.c_int32),
                ("grid_chunks", ctypes.c_int32), ("jk_chunks", ctypes.c_int32),
                ("iter_precision", ctypes.c_int32), ("direct_scf", ctypes.c_int32), ("recheck_err", ctypes.c_double),
                ("recheck_fp64_err", ctypes.c_double)]


class rks_result_t(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("nbf", ctypes.c_int32), ("n_occ", ctypes.c_int32),
                ("iters", ctypes.c_int32), ("e_total", ctypes.c_double), ("e_homo", ctypes.c_double),
                ("e_lumo", ctypes.c_double), ("gap", ctypes.c_double), ("e_xc", ctypes.c_double),
                ("e_nuc", ctypes.c_double), ("latency_s", ctypes.c_double),
                ("paper_converged", ctypes.c_int32), ("rechecked", ctypes.c_int32),
                ("err_max", ctypes.c_double), ("de_last", ctypes.c_double)]


class rks_stage_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int32), ("ms", ctypes.c_double),
                ("units", ctypes.c_double)]


# symbol -> (restype, argtypes); the exported set of include/rks.h
_P = ctypes.c_void_p
_SIGS = {
    "rks_options_default": (ctypes.c_int, [ctypes.POINTER(rks_options)]),
    "rks_nbf": (ctypes.c_int, [ctypes.c_int32, _P]),
    "rks_mol_bytes": (ctypes.c_int64, [ctypes.POINTER(rks_options), ctypes.c_int32, _P]),
    "rks_tc_plan": (ctypes.c_int, [ctypes.c_int32, _P, _P]),
    "rks_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "rks_last_error": (ctypes.c_char_p, [_P]),
    "rks_create": (ctypes.c_int, [ctypes.POINTER(rks_options), ctypes.POINTER(_P)]),
    "rks_destroy": (ctypes.c_int, [_P]),
    "rks_stream": (_P, [_P]),
    "rks_submit": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "rks_submit_batch": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, _P]),
    "rks_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32)]),
    "rks_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double]),
    "rks_result": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(rks_result_t), _P, _P, ctypes.c_int32]),
    "rks_batch_create": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, ctypes.POINTER(_P)]),
    "rks_batch_run": (ctypes.c_int, [_P]),
    "rks_batch_sync": (ctypes.c_int, [_P]),
    "rks_batch_result": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(rks_result_t), _P, _P,
                                        ctypes.c_int32]),
    "rks_batch_destroy": (ctypes.c_int, [_P]),
    "rks_batch_setup": (ctypes.c_int, [_P]),
    "rks_batch_fock": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "rks_batch_dump": (ctypes.c_int64, [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int64]),
    "rks_profile_enable": (ctypes.c_int, [_P, ctypes.c_int32]),
    "rks_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(rks_stage_time), ctypes.c_int32]),
    "rks_eval_boys": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_int32]),
    "rks_eval_xc": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, _P, _P, ctypes.c_int32]),
    "rks_eval_xc_noalloc": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, _P, _P, ctypes.c_int32]),
    "rks_selftest_bounded_wait": (ctypes.c_int, [_P, ctypes.c_int32]),
    "rks_probe_peak": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
}

_lib = None


def lib():
    """Load librks.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"CUDA library not built: {LIB} missing (run paper_2311_01135_gb300._build)")
        L = ctypes.CDLL(LIB)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class RKSError(RuntimeError):
    def __init__(self, code, where=""):
        L = lib()
        msg = L.rks_strerror(code).decode()
        detail = L.rks_last_error(None).decode()
        super().__init__(f"{where}: {msg} ({code}) {detail}")
        self.code = code


def _chk(rc, where):
    if rc < 0:
        raise RKSError(rc, where)
    return rc


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def options(**kw):
    o = rks_options()
    lib().rks_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def rks_nbf(Z):
    Z = np.ascontiguousarray(Z, np.int32)
    return _chk(lib().rks_nbf(len(Z), _ptr(Z)), "rks_nbf")


def rks_mol_bytes(Z, **opts):
    """Device bytes the molecule adds to a batch under these options."""
    Z = np.ascontiguousarray(Z, np.int32)
    o = options(**opts)
    return _chk(lib().rks_mol_bytes(ctypes.byref(o), len(Z), _ptr(Z)), "rks_mol_bytes")


RKS_TC_PLAN_INTS = 100


def rks_tc_plan(Z):
    """(NQ, plan[RKS_TC_PLAN_INTS]) of the tensor-core grid kernel's column
    plan; NQ = 0 when the CUDA-core grid kernel takes the molecule."""
    Z = np.ascontiguousarray(Z, np.int32)
    plan = np.zeros(RKS_TC_PLAN_INTS, np.int32)
    nq = _chk(lib().rks_tc_plan(len(Z), _ptr(Z), _ptr(plan)), "rks_tc_plan")
    return nq, plan


class Context:
    """rks_create / rks_destroy, plus the serving calls."""

    def __init__(self, **opts):
        self.opts = options(**opts)
        h = ctypes.c_void_p()
        _chk(lib().rks_create(ctypes.byref(self.opts), ctypes.byref(h)), "rks_create")
        self.h = h

    def close(self):
        if self.h:
            lib().rks_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def stream(self):
        return lib().rks_stream(self.h)

    # serving API
    def submit(self, Z, xyz):
        Z = np.ascontiguousarray(Z, np.int32)
        xyz = np.ascontiguousarray(xyz, np.float64).reshape(-1, 3)
        t = ctypes.c_uint64()
        _chk(lib().rks_submit(self.h, len(Z), _ptr(Z), _ptr(xyz), ctypes.byref(t)), "rks_submit")
        return t.value

    def submit_many(self, mols):
        """Queue [(Z, xyz), ...] in one call (rks_submit_batch); returns the tickets."""
        na = np.array([len(Z) for Z, _ in mols], np.int32)
        Z = np.ascontiguousarray(np.concatenate([np.asarray(z, np.int32) for z, _ in mols]), np.int32)
        xyz = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).reshape(-1, 3)
                                                   for _, x in mols]), np.float64)
        t = np.zeros(len(mols), np.uint64)
        _chk(lib().rks_submit_batch(self.h, len(mols), _ptr(na), _ptr(Z), _ptr(xyz), _ptr(t)),
             "rks_submit_batch")
        return [int(x) for x in t]

    def poll(self, ticket):
        s = ctypes.c_int32()
        _chk(lib().rks_poll(self.h, ticket, ctypes.byref(s)), "rks_poll")
        return s.value

    def wait(self, ticket, timeout_s=600.0):
        return _chk(lib().rks_wait(self.h, ticket, timeout_s), "rks_wait")

    def result(self, ticket, nbf_cap=RKS_MAX_NBF):
        r = rks_result_t()
        eps = np.zeros(nbf_cap)
        D = np.zeros(nbf_cap * nbf_cap)
        _chk(lib().rks_result(self.h, ticket, ctypes.byref(r), _ptr(eps), _ptr(D), nbf_cap), "rks_result")
        n = r.nbf
        return _res_dict(r, eps[:n].copy(), D[:n * n].reshape(n, n).copy())

    # profiling
    def profile(self, on=True):
        _chk(lib().rks_profile_enable(self.h, int(on)), "rks_profile_enable")

    def profile_read(self):
        buf = (rks_stage_time * 64)()
        n = _chk(lib().rks_profile_read(self.h, buf, 64), "rks_profile_read")
        return {buf[i].name.decode(): dict(launches=buf[i].launches, ms=buf[i].ms, units=buf[i].units)
                for i in range(n)}

    def eval_boys(self, mmax, T, precision=RKS_FP64):
        T = np.ascontiguousarray(T, np.float64)
        out = np.zeros((len(T), mmax + 1))
        _chk(lib().rks_eval_boys(self.h, mmax, len(T), _ptr(T), _ptr(out), precision), "rks_eval_boys")
        return out

    def eval_xc(self, rho, sigma, precision=RKS_FP64):
        rho = np.ascontiguousarray(rho, np.float64)
        sigma = np.ascontiguousarray(sigma, np.float64)
        e, vr, vs = (np.zeros(len(rho)) for _ in range(3))
        _chk(lib().rks_eval_xc(self.h, len(rho), _ptr(rho), _ptr(sigma), _ptr(e), _ptr(vr), _ptr(vs),
                               precision), "rks_eval_xc")
        return e, vr, vs

    def probe_peak(self, kind):
        """rks_probe_peak: measured operations per second of RKS_PROBE_* kind."""
        v = ctypes.c_double()
        _chk(lib().rks_probe_peak(self.h, kind, ctypes.byref(v)), "rks_probe_peak")
        return v.value

    def selftest_bounded_wait(self, spins=100000):
        """rks_selftest_bounded_wait: the return code (RKS_EDEVICE expected)."""
        return lib().rks_selftest_bounded_wait(self.h, spins)

    def eval_xc_noalloc(self, rho, sigma, precision=RKS_FP64):
        """rks_eval_xc_noalloc: as eval_xc, staged through the library's static scratch."""
        rho = np.ascontiguousarray(rho, np.float64)
        sigma = np.ascontiguousarray(sigma, np.float64)
        e, vr, vs = (np.zeros(len(rho)) for _ in range(3))
        _chk(lib().rks_eval_xc_noalloc(self.h, len(rho), _ptr(rho), _ptr(sigma), _ptr(e), _ptr(vr), _ptr(vs),
                                       precision), "rks_eval_xc_noalloc")
        return e, vr, vs


def _res_dict(r, eps, D):
    return dict(status=RKS_STATUS.get(r.status, r.status), nbf=r.nbf, nocc=r.n_occ, iters=r.iters,
                E=r.e_total, homo=r.e_homo, lumo=r.e_lumo, gap=r.gap, Exc=r.e_xc, Enuc=r.e_nuc,
                latency_s=r.latency_s, paper_converged=bool(r.paper_converged), err_max=r.err_max,
                de_last=r.de_last, rechecked=int(r.rechecked), eps=eps, D=D)


class Batch:
    """rks_batch_*: a fixed set of molecules resident on the device."""

    def __init__(self, ctx: Context, mols):
        self.ctx = ctx
        na = np.array([len(Z) for Z, _ in mols], np.int32)
        Z = np.ascontiguousarray(np.concatenate([np.asarray(Z, np.int32) for Z, _ in mols] or [np.zeros(0, np.int32)]))
        xyz = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).reshape(-1, 3) for _, x in mols]
                                                  or [np.zeros((0, 3))]))
        h = ctypes.c_void_p()
        _chk(lib().rks_batch_create(ctx.h, len(mols), _ptr(na), _ptr(Z), _ptr(xyz), ctypes.byref(h)),
             "rks_batch_create")
        self.h = h
        self.n = len(mols)
        self.nbf = [rks_nbf(Z) for Z, _ in mols]

    def close(self):
        if self.h:
            lib().rks_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def setup(self):
        _chk(lib().rks_batch_setup(self.h), "rks_batch_setup")

    def run(self):
        _chk(lib().rks_batch_run(self.h), "rks_batch_run")

    def sync(self):
        _chk(lib().rks_batch_sync(self.h), "rks_batch_sync")

    def result(self, m):
        n = self.nbf[m]
        r = rks_result_t()
        eps = np.zeros(n)
        D = np.zeros(n * n)
        _chk(lib().rks_batch_result(self.h, m, ctypes.byref(r), _ptr(eps), _ptr(D), n), "rks_batch_result")
        return _res_dict(r, eps, D.reshape(n, n))

    def fock(self, Ds, final_step=False):
        Dall = np.ascontiguousarray(np.concatenate([np.asarray(D, np.float64).ravel() for D in Ds]))
        _chk(lib().rks_batch_fock(self.h, _ptr(Dall), int(final_step)), "rks_batch_fock")

    def dump(self, m, what, dtype=np.float64, count=None):
        n = self.nbf[m]
        cap = count if count is not None else max(8 * n * n, 1 << 20)
        while True:
            buf = np.zeros(cap, np.uint8)
            got = lib().rks_batch_dump(self.h, m, what, _ptr(buf), cap)
            if got == RKS_EINVAL and cap < (1 << 34):
                cap *= 8
                continue
            _chk(got, "rks_batch_dump")
            return buf[:got].view(dtype).copy()

    def matrix(self, m, what):
        n = self.nbf[m]
        return self.dump(m, what).reshape(n, n)
