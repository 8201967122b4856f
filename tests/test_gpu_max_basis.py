"""The largest basis the kernels take (nbf close to 96): a seeded 15-heavy-atom
molecule (seed 101, nbf 95).  Exercises the paths the 9-11-heavy-atom
workload does not reach: the J/K kernel's reduced shared-memory plan (pair
table left in global memory when D/J/K fill shared memory) and the CUDA-core
grid kernel in the mixed iterations (the tensor-core kernel takes nbf <= 80).

Stage parity at the oracle's SAD density (FP64 path <= 1e-10 abs, as for the
9-heavy-atom molecule) and the mixed final-step Fock build (<= 2e-5 abs on
J/K/V_xc, as there)."""
import numpy as np
import pytest

import molgen

pytestmark = pytest.mark.gpu
g = pytest.importorskip("paper_2311_01135_gb300")


@pytest.fixture(scope="module")
def big():
    from oracle import scf
    Z, xyz = molgen.batch(101, 1, 14, 16)[0]
    assert 90 <= g.rks_nbf(Z) <= g.RKS_MAX_NBF
    s = scf.System(Z, xyz)
    D0 = s.sad_guess()
    F0, E0, parts0 = s.fock(D0)
    return Z, xyz, D0, E0, parts0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_max_basis_fock(big, prec):
    Z, xyz, D0, E0, parts0 = big
    p = g.RKS_FP64 if prec == "fp64" else g.RKS_MIXED
    tol = 1e-10 if prec == "fp64" else 2e-5
    with g.Context(precision=p) as c, g.Batch(c, [(Z, xyz)]) as B:
        B.fock([D0], final_step=True)
        for what, key in ((g.RKS_DUMP_J, "J"), (g.RKS_DUMP_K, "K"), (g.RKS_DUMP_VXC, "Vxc")):
            assert np.max(np.abs(B.matrix(0, what) - parts0[key])) < tol, key
        sc = B.dump(0, g.RKS_DUMP_SCALARS)
        assert abs(sc[1] - parts0["Exc"]) < (1e-10 if prec == "fp64" else 1e-5)
        assert abs(sc[0] - E0) < (1e-9 if prec == "fp64" else 2e-4)


def test_max_basis_iterations_mixed(big):
    """A few mixed iterations (CUDA-core grid kernel, FP32 J/K with the
    reduced plan) run and stay finite; the energy is checked against the
    FP64 path after the same iterations."""
    Z, xyz, *_ = big
    out = {}
    for name, p in (("fp64", g.RKS_FP64), ("mixed", g.RKS_MIXED)):
        with g.Context(precision=p, fixed_iters=3) as c, g.Batch(c, [(Z, xyz)]) as B:
            B.run()
            B.sync()
            out[name] = B.result(0)
    assert out["mixed"]["status"] == "ok" and np.isfinite(out["mixed"]["E"])
    assert abs(out["mixed"]["E"] - out["fp64"]["E"]) < 5e-4
