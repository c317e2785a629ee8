"""Configuration selection and configuration MPS through the C ABI (host code, no device)
against oracle/configs.py: the selected configurations are the nmax lowest of the oracle's
candidates (energies to 1e-10; exactly degenerate pairs, such as spin-flipped
determinants, may trade places), each with the oracle's energy; the import arrays are
consistent (sizes, selectors with one 1 per column, coefficients in the wavefunction); and
the argument checks."""
import ctypes

import numpy as np
import pytest

import qcinputs as q
from tests._lib import ensure_built


def _check_selection(steps, en, nmax, cands):
    byst = {c[2]: c[0] for c in cands}
    cands = sorted(cands)
    m = min(nmax, len(cands))
    assert len(steps) == m
    assert len({tuple(s) for s in steps}) == m
    assert np.abs(en - np.array([c[0] for c in cands[:m]])).max() <= 1e-10
    for s, e in zip(steps, en):
        assert abs(byst[tuple(int(x) for x in s)] - e) <= 1e-10
    # everything clearly below the last selected energy is selected
    chosen = {tuple(int(x) for x in s) for s in steps}
    for e, _, st in cands:
        if e < en[-1] - 1e-9:
            assert st in chosen


@pytest.mark.parametrize("L,N,two_s,nmax", [(5, 4, 0, 1), (5, 4, 0, 20), (6, 5, 1, 40), (6, 6, 2, 500),
                                            (7, 8, 0, 150)])
def test_u1_selection_matches_the_oracle(L, N, two_s, nmax):
    import paper_2603_28648_b300 as qd
    from oracle import configs as oc
    lib = qd.load(ensure_built())
    h, V = q.make_integrals(L, 5)
    steps, en = qd.select_configs(qd.U1, h, V, N, two_s, nmax, lib=lib)
    _check_selection(steps, en, nmax, oc.candidates_u1(h, V, N, two_s))


@pytest.mark.parametrize("L,N,two_s,nmax", [(5, 4, 0, 12), (6, 5, 1, 30), (6, 6, 2, 30), (6, 6, 0, 400),
                                            (7, 7, 3, 60)])
def test_su2_selection_matches_the_oracle(L, N, two_s, nmax):
    import paper_2603_28648_b300 as qd
    from oracle import configs as oc
    lib = qd.load(ensure_built())
    h, V = q.make_integrals(L, 5)
    steps, en = qd.select_configs(qd.SU2, h, V, N, two_s, nmax, lib=lib)
    _check_selection(steps, en, nmax, oc.candidates_su2(h, V, N, two_s))


@pytest.mark.parametrize("sym", [0, 1])
def test_config_mps_arrays(sym):
    """Sizes and selector structure of the import arrays: bond b has one state per
    distinct prefix of length b, bond L-1 none, bond L the vacuum, and the data ends with
    a wavefunction whose entries are the coefficients (one per configuration)."""
    import paper_2603_28648_b300 as qd
    lib = qd.load(ensure_built())
    L, N, two_s = 7, 6, 0
    h, V = q.make_integrals(L, 8)
    steps, _ = qd.select_configs(sym, h, V, N, two_s, 25, lib=lib)
    coef = np.arange(1, len(steps) + 1, dtype=float)
    center, nsec, sec, data = qd.config_mps(sym, L, N, two_s, steps, coef, lib=lib)
    assert center == L - 2 and len(nsec) == L + 1 and nsec[L - 1] == 0
    trip = sec.reshape(-1, 3)
    dims = np.split(trip[:, 2], np.cumsum(nsec)[:-1])
    for b in range(L - 1):
        assert dims[b].sum() == len({tuple(s[:b]) for s in steps})
    assert list(trip[-1]) == [0, 0, 1]
    # one 1 per selector column (the states of bonds 1 .. L-2), plus the coefficient 1.0
    assert np.count_nonzero(data == 1.0) == sum(int(dims[b].sum()) for b in range(1, L - 1)) + 1
    assert sorted(x for x in data if x not in (0.0, 1.0)) == list(coef[1:])


def test_invalid_configurations_are_rejected():
    import paper_2603_28648_b300 as qd
    lib = qd.load(ensure_built())
    L = 4
    good = np.array([[3, 3, 0, 0]], dtype=np.uint8)
    qd.config_mps(qd.U1, L, 4, 0, good, [1.0], lib=lib)
    for sym, N, s, st, c in [(qd.U1, 4, 0, [[3, 3, 0, 4]], [1.0]),      # step outside 0..3
                             (qd.U1, 4, 2, [[3, 3, 0, 0]], [1.0]),      # outside the target
                             (qd.SU2, 2, 0, [[2, 1, 0, 0]], [1.0]),     # spin below zero
                             (qd.U1, 4, 0, [[3, 3, 0, 0]], [0.0])]:     # zero wavefunction
        with pytest.raises(qd.QcdmrgError):
            qd.config_mps(sym, L, N, s, np.array(st, dtype=np.uint8), c, lib=lib)
    h, V = q.make_integrals(L, 1)
    with pytest.raises(qd.QcdmrgError):
        qd.select_configs(qd.U1, h, V, 9, 1, 5, lib=lib)                # N > 2L
    with pytest.raises(qd.QcdmrgError):
        qd.select_configs(qd.SU2, h, V, 4, 6, 5, lib=lib)               # 2S > N
    u8 = ctypes.POINTER(ctypes.c_uint8)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    assert lib.qcdmrg_select_configs(0, L, 4, 0, ctypes.cast(None, dp), ctypes.cast(None, dp), 5,
                                     ctypes.cast(None, u8), ctypes.cast(None, dp), ctypes.cast(None, ip)) == -1
    # a data buffer that is too small
    nsec = np.zeros(L + 1, dtype=np.int32)
    sec = np.zeros(64, dtype=np.int32)
    data = np.zeros(1)
    one = np.ones(1)
    rc = lib.qcdmrg_config_mps(0, L, 4, 0, 1, good.ctypes.data_as(u8), one.ctypes.data_as(dp), None,
                               nsec.ctypes.data_as(ip), sec.ctypes.data_as(ip), sec.size, data.ctypes.data_as(dp),
                               0, None, None)
    assert rc == -1


def test_selection_at_the_cas54_36_shape():
    """L = 36, N = 54, S = 0: asking for every candidate returns the 1 + 2 * 27 * 9 +
    2 * C(27,2) * C(9,2) + (27 * 9)^2 = 84,808 determinants within two electrons of the aufbau
    reference, sorted by energy, all distinct; the lowest is the reference (at these integrals)
    with the closed-shell energy 2 sum_i h_ii + sum_ij (2 (ii|jj) - (ij|ji)) over its orbitals."""
    import math
    import paper_2603_28648_b300 as qd
    lib = qd.load(ensure_built())
    L, N = 36, 54
    h, V = q.make_integrals(L, q.integrals.BASE_SEED + 2)
    steps, en = qd.select_configs(qd.U1, h, V, N, 0, 100000, lib=lib)
    nocc, nvir = 27, 9
    total = 1 + 2 * nocc * nvir + 2 * math.comb(nocc, 2) * math.comb(nvir, 2) + (nocc * nvir) ** 2
    assert len(steps) == total == 84808
    assert np.all(np.diff(en) >= 0)
    assert len({s.tobytes() for s in steps}) == total
    occ = [p for p in range(L) if steps[0][p] == 3]
    assert len(occ) == nocc and not np.any((steps[0] == 1) | (steps[0] == 2))
    e = 2 * sum(h[i, i] for i in occ) + sum(2 * V[i, i, j, j] - V[i, j, j, i] for i in occ for j in occ)
    assert abs(en[0] - e) <= 1e-9 * abs(e)
