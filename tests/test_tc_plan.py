"""Host logic of the tensor-core grid kernel's column plan (rks_tc_plan), on
the CPU: the plan must put every AO of the molecule in exactly one kernel
column, in the places its unit words say, in the smallest class that holds it.
A wrong plan would scatter V_xc into the wrong matrix elements."""
import numpy as np
import pytest

import molgen

g = pytest.importorskip("paper_2311_01135_gb300")
EMPTY = 63


def ao_first(Z):
    out, a = [], 0
    for z in Z:
        out.append(a)
        a += 1 if z == 1 else 5
    return out


def check_plan(Z):
    Z = np.asarray(Z, np.int32)
    nbf = g.rks_nbf(Z)
    nq, plan = g.rks_tc_plan(Z)
    nheavy = int((Z > 1).sum())
    # the smallest class whose padded size holds the basis and whose units hold the heavy atoms
    want = next((q for q in (4, 8, 12, 16, 20) if 4 * q >= nbf and nheavy <= 4 * (q // 5)), 0)
    if len(Z) > 63:
        want = 0
    assert nq == want, (list(Z), nq, want)
    if nq == 0:
        return nq
    U, R = nq // 5, nq % 5
    first = ao_first(Z)
    perm = plan[20:20 + 4 * nq]
    assert (plan[20 + 4 * nq:] == -1).all()
    assert sorted(int(x) for x in perm if x >= 0) == list(range(nbf))
    seen = set()
    for q in range(4):
        for k in range(U):
            w = int(plan[q * 5 + k]) & 0xFFFFFFFF
            cols = perm[q * nq + 5 * k: q * nq + 5 * k + 5]
            if w >> 31:
                A = w & 63
                assert Z[A] > 1 and A not in seen
                seen.add(A)
                assert list(cols) == [first[A] + r for r in range(5)]
            else:
                for r in range(5):
                    A = (w >> (6 * r)) & 63
                    if A == EMPTY:
                        assert cols[r] == -1
                    else:
                        assert Z[A] == 1 and A not in seen
                        seen.add(A)
                        assert cols[r] == first[A]
        w = int(plan[q * 5 + 4]) & 0xFFFFFFFF
        for r in range(R):
            A = (w >> (6 * r)) & 63
            c = perm[q * nq + 5 * U + r]
            if A == EMPTY:
                assert c == -1
            else:
                assert Z[A] == 1 and A not in seen
                seen.add(A)
                assert c == first[A]
    assert seen == set(range(len(Z)))
    return nq


def test_workload_molecules():
    """Every molecule of a 9-11-heavy-atom sample gets a plan, almost always in
    the class of its basis rounded up to 16."""
    mols = molgen.batch(2, 512, 9, 11)
    bigger = 0
    for Z, _ in mols:
        nq = check_plan(Z)
        assert nq > 0
        bigger += 4 * nq > (g.rks_nbf(Z) + 15) // 16 * 16
    assert bigger <= 2


def test_small_and_edge_molecules():
    for Z in ([1, 1], [8, 1, 1], [7, 7], [6, 1, 1, 1, 1], [9] * 16, [6] * 9 + [1] * 3, [1] * 62, [1] * 4,
              [6, 6, 8, 8] + [1] * 20, [1] * 5 + [6] * 15):
        check_plan(Z)
    assert g.rks_tc_plan(np.array([1] * 64))[0] == 0     # more atoms than the 6-bit ids hold
    assert g.rks_tc_plan(np.array([6] * 17))[0] == 0     # basis above 80
    assert g.rks_tc_plan(np.array([6] * 9 + [1] * 3))[0] == 16  # 9 heavy atoms need three units a quarter
    with pytest.raises(Exception):
        g.rks_tc_plan(np.array([2, 2]))


def test_larger_molecules_take_no_plan():
    """Molecules of the 20-30-heavy-atom workload (above 80 functions) get no
    tensor-core plan: the global-memory kernels take them."""
    for Z, _ in molgen.batch(4, 32, 20, 30):
        assert g.rks_nbf(Z) > 96
        assert check_plan(Z) == 0
