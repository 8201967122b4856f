"""The C ABI boundary without a GPU: the library loads, exports every function
include/rks.h declares, the ctypes structures match the C layout (checked by
compiling a probe against the header with gcc), and the host-only entries
(options, basis size, error names, context creation without a device) behave
as documented."""
import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "rks.h")

g = pytest.importorskip("paper_2311_01135_gb300")


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(g.LIB):
        if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("library not built and no nvcc")
        g.build()
    return g.lib()


def _declared():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(rks_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_function_is_exported(L):
    names = _declared()
    assert len(names) >= 24
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding registers a signature for each one
    assert not [n for n in names if n not in g._SIGS], [n for n in names if n not in g._SIGS]


def _c_layout(tmp_path):
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no gcc")
    fields = [f for f, _ in g.rks_options._fields_]
    rfields = [f for f, _ in g.rks_result_t._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HDR}"', 'int main(void) {',
             'printf("opt %zu\\n", sizeof(rks_options));',
             'printf("res %zu\\n", sizeof(rks_result_t));',
             'printf("stage %zu\\n", sizeof(rks_stage_time));']
    lines += [f'printf("o.{f} %zu\\n", offsetof(rks_options, {f}));' for f in fields]
    lines += [f'printf("r.{f} %zu\\n", offsetof(rks_result_t, {f}));' for f in rfields]
    lines += ['return 0; }']
    c = tmp_path / "probe.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", str(c), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return dict(line.split() for line in out.strip().splitlines())


def test_struct_layout_matches_header(tmp_path):
    lay = _c_layout(tmp_path)
    assert int(lay["opt"]) == ctypes.sizeof(g.rks_options)
    assert int(lay["res"]) == ctypes.sizeof(g.rks_result_t)
    assert int(lay["stage"]) == ctypes.sizeof(g.rks_stage_time)
    for f, _ in g.rks_options._fields_:
        assert int(lay["o." + f]) == getattr(g.rks_options, f).offset, f
    for f, _ in g.rks_result_t._fields_:
        assert int(lay["r." + f]) == getattr(g.rks_result_t, f).offset, f


def test_options_default(L):
    o = g.rks_options()
    assert L.rks_options_default(ctypes.byref(o)) == 0
    assert (o.n_rad, o.n_theta, o.n_phi, o.becke_iters) == (50, 12, 24, 3)
    assert o.precision == g.RKS_FP64 and o.xc == 1 and o.diis_space == 8
    assert o.guess == g.RKS_GUESS_SAD and o.fix_theta == 0.1 and o.grid_tc == 1
    assert o.max_cohorts == 4 and o.admit_wait_us == 20000
    assert o.iter_precision == 0 and o.recheck_err == 1e-4 and o.recheck_fp64_err == 3e-4
    assert o.direct_scf == g.RKS_DIRECT_NEVER
    assert L.rks_options_default(None) == g.RKS_EINVAL


def test_header_constants_match_binding():
    src = open(HDR).read()
    for name in ("RKS_MAX_NBF", "RKS_DIRECT_NEVER", "RKS_DIRECT_ALWAYS", "RKS_DIRECT_AUTO",
                 "RKS_ITER_JK_FINAL", "RKS_ITER_GRID_FINAL"):
        m = re.search(r"#define\s+" + name + r"\s+(\d+)", src)
        assert m and int(m.group(1)) == getattr(g, name), name


def test_larger_workload_fits_the_basis_cap(L):
    """The 20-30-heavy-atom workload (seed 4) stays within RKS_MAX_NBF, and
    spans the global-memory kernels' range (above 96 functions)."""
    import molgen
    nbf = [g.rks_nbf(Z) for Z, _ in molgen.batch(4, 256, 20, 30)]
    assert min(nbf) > 96 and max(nbf) <= g.RKS_MAX_NBF


def test_nbf_and_validation(L):
    assert g.rks_nbf([8, 1, 1]) == 7
    assert g.rks_nbf([6, 6, 1, 1, 1, 1]) == 14
    Z = np.array([2], np.int32)  # helium: not in the element set
    assert L.rks_nbf(1, Z.ctypes.data) == g.RKS_EINVAL
    assert L.rks_nbf(0, Z.ctypes.data) == g.RKS_EINVAL


def test_mol_bytes_footprint(L):
    """The admission figure: grows with the molecule, FP64 above mixed,
    direct SCF drops the packed store (the bulk for 20-30 heavy atoms),
    invalid molecules are rejected."""
    import molgen
    w = g.rks_mol_bytes([8, 1, 1])
    small = g.rks_mol_bytes(molgen.batch(2, 1, 9, 9)[0][0], precision=g.RKS_MIXED)
    Zb = molgen.batch(4, 1, 20, 20)[0][0]
    big = g.rks_mol_bytes(Zb, precision=g.RKS_MIXED)
    big_direct = g.rks_mol_bytes(Zb, precision=g.RKS_MIXED, direct_scf=g.RKS_DIRECT_ALWAYS)
    assert 0 < w < small < big
    assert g.rks_mol_bytes(Zb, precision=g.RKS_FP64) > big
    n = g.rks_nbf(Zb)
    npair = n * (n + 1) // 2
    # the store's unscreened capacity is about npair^2 / 2 elements of 4 bytes
    assert big - big_direct > 0.4 * 4 * npair * npair / 2
    Z = np.array([2], np.int32)
    assert L.rks_mol_bytes(None, 1, Z.ctypes.data) == g.RKS_EINVAL
    assert L.rks_mol_bytes(None, 0, Z.ctypes.data) == g.RKS_EINVAL


def test_error_names(L):
    for code in range(0, -9, -1):
        assert L.rks_strerror(code)
    assert L.rks_strerror(-8) != L.rks_strerror(-7)


def test_null_handles_are_rejected(L):
    assert L.rks_destroy(None) == g.RKS_EINVAL
    assert L.rks_batch_run(None) == g.RKS_EINVAL
    assert L.rks_batch_sync(None) == g.RKS_EINVAL
    assert L.rks_batch_destroy(None) == g.RKS_EINVAL
    assert L.rks_poll(None, 1, None) == g.RKS_EINVAL
    assert L.rks_submit_batch(None, 0, None, None, None, None) == g.RKS_EINVAL


def test_bad_options_rejected_before_any_device_call(L):
    o = g.rks_options()
    L.rks_options_default(ctypes.byref(o))
    o.precision = 7
    h = ctypes.c_void_p()
    assert L.rks_create(ctypes.byref(o), ctypes.byref(h)) == g.RKS_EINVAL
    L.rks_options_default(ctypes.byref(o))
    o.max_cohorts = 0
    assert L.rks_create(ctypes.byref(o), ctypes.byref(h)) == g.RKS_EINVAL
    L.rks_options_default(ctypes.byref(o))
    o.direct_scf = 3
    assert L.rks_create(ctypes.byref(o), ctypes.byref(h)) == g.RKS_EINVAL


def test_create_without_a_device_fails_loudly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(g.RKSError) as e:
        g.Context()
    assert e.value.code == g.RKS_ECUDA
