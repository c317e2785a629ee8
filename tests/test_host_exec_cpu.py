"""Host logic without a GPU, numerically: the library's own FP64 H_eff task lists
(complementary-operator rules, renormalization, centre plan) executed with plain loops,
and the tiled work items of the tensor-core path evaluated in FP64 (views, panels, term
scalars, T tiles, split stage-2 items), both against the oracle's sigma, on imported
MPS of several shapes, edge centres included, and on the M-expansion of an SU(2) MPS; with
the normal/complementary switch at several cuts as well. Every launch is bounds-checked.
tests/host_exec.cpp holds the test-only host executor; the product path still needs CUDA."""
import os
import struct
import subprocess

import numpy as np
import pytest

import qcinputs as q


@pytest.fixture(scope="module")
def host_exec(tmp_path_factory):
    from tests._lib import build_host_executable
    out = build_host_executable("host_exec.cpp", str(tmp_path_factory.mktemp("hostexec") / "host_exec"))
    if out is None:
        pytest.skip("g++ not available")
    return out


def _write(path, mps, h, V):
    from oracle.mpsu1 import export_abi
    nsec, sec, data = export_abi(mps)
    with open(path, "wb") as f:
        f.write(struct.pack("<7q", mps.L, mps.N, mps.two_sz, mps.center, len(nsec), len(sec), len(data)))
        f.write(np.ascontiguousarray(h, "<f8").tobytes())
        f.write(np.ascontiguousarray(V, "<f8").tobytes())
        f.write(np.asarray(nsec, "<i4").tobytes())
        f.write(np.asarray(sec, "<i4").tobytes())
        f.write(np.asarray(data, "<f8").tobytes())


def _env(switch, sum_gemm=0):
    return dict(os.environ, HOST_EXEC_PAIR_SWITCH=str(switch), HOST_EXEC_SUM_GEMM=str(sum_gemm))


def _run(exe, tmp, mps, h, V, switch=0, sum_gemm=0):
    fin, fout = str(tmp / "in.bin"), str(tmp / "out.bin")
    _write(fin, mps, h, V)
    r = subprocess.run([exe, fin, fout], capture_output=True, text=True, timeout=600,
                       env=_env(switch, sum_gemm))
    assert r.returncode == 0, r.stderr
    out = np.fromfile(fout, "<f8")
    n = len(out) // 2
    return out[:n], out[n:]


@pytest.mark.parametrize("L,N,two_sz,D,c,seed", [(6, 6, 0, 16, 2, 3), (7, 5, 1, 16, 2, 4), (5, 4, 0, 8, 0, 5),
                                                  (6, 6, 2, 16, 4, 6), (8, 8, 0, 32, 3, 7)])
def test_library_task_lists_match_the_oracle(host_exec, tmp_path, L, N, two_sz, D, c, seed):
    from oracle.dmrgu1 import DMRGU1
    from oracle.mpsu1 import MPSU1
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, two_sz, D, q.SYM_U1, seed, c))
    h, V = q.make_integrals(L, seed + 1)
    s64, st = _run(host_exec, tmp_path, m, h, V)
    ref = m.psi_to_flat(DMRGU1(h, V, N, two_sz).sigma(m))
    assert np.linalg.norm(s64 - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.linalg.norm(st - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("switch", [0, 3])
def test_library_task_lists_on_an_su2_state(host_exec, tmp_path, switch):
    from oracle.fci import FCI
    from oracle.mpssu2 import TangentSU2, to_u1
    t = TangentSU2(7, 7, 1, 2, cap=2, seed=9)
    mps, C = to_u1(t)
    psi = np.random.default_rng(4).normal(size=C.shape[1])
    mps.psi = mps.psi_from_flat(C @ psi)
    h, V = q.make_integrals(7, 13)
    s64, st = _run(host_exec, tmp_path, mps, h, V, switch)
    ref = t.heff(FCI(h, V, 7, 1), psi)
    for s in (s64, st):
        assert np.linalg.norm(C.T @ s - ref) <= 1e-12 * np.linalg.norm(ref)


def _sweeps(exe, tmp, mps, h, V, D, nsweeps, switch=0, sum_gemm=0):
    fin, fout = str(tmp / "sw_in.bin"), str(tmp / "sw_out.bin")
    _write(fin, mps, h, V)
    r = subprocess.run([exe, fin, fout, "sweep", str(D), str(nsweeps), "1e-10"], capture_output=True,
                       text=True, timeout=600, env=_env(switch, sum_gemm))
    assert r.returncode == 0, r.stderr
    return np.fromfile(fout, "<f8")


@pytest.mark.parametrize("L,N,D,c,mps_seed,int_seed", [(6, 6, 8, 2, 3, 4), (7, 5, 12, 3, 5, 6)])
def test_engine_sweeps_match_the_oracle(host_exec, tmp_path, L, N, D, c, mps_seed, int_seed):
    from oracle.dmrgu1 import DMRGU1
    from oracle.mpsu1 import MPSU1
    two = N % 2
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, two, D, q.SYM_U1, mps_seed, c))
    h, V = q.make_integrals(L, int_seed)
    E = _sweeps(host_exec, tmp_path, m, h, V, D, 2)
    Eo, _, _ = DMRGU1(h, V, N, two).sweeps(m, D, 2, tol=1e-12)
    assert np.abs(E - np.array(Eo)).max() <= 1e-9


def test_engine_sweeps_at_exact_bond_dimension_give_fci(host_exec, tmp_path):
    from oracle.fci import FCI
    from oracle.mpsu1 import MPSU1
    L, N, D = 6, 6, 64
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, D, q.SYM_U1, 3, 2))
    h, V = q.make_integrals(L, 11)
    E = _sweeps(host_exec, tmp_path, m, h, V, D, 2)
    e0, _ = FCI(h, V, N, 0).ground_state()
    assert abs(E[-1] - e0) <= 1e-9


# Normal/complementary switch: left blocks at cuts <= switch and right blocks beyond it hold
# the normal pairs. The cases put the switch left of, at, and right of the centre cut, so the
# switching enlargement runs in the left chain, the right chain and at the centre, and the
# centre uses either decomposition; edge centres included.
@pytest.mark.parametrize("L,N,two_sz,D,c,seed,switch", [(6, 6, 0, 16, 2, 3, 1), (6, 6, 0, 16, 2, 3, 2),
                                                         (6, 6, 0, 16, 2, 3, 3), (6, 6, 0, 16, 2, 3, 5),
                                                         (7, 5, 1, 16, 2, 4, 2), (8, 8, 0, 32, 3, 7, 4),
                                                         (8, 8, 0, 32, 3, 7, 6), (6, 6, 0, 16, 0, 3, 3),
                                                         (7, 7, 1, 16, 5, 8, 3)])
def test_switched_task_lists_match_the_oracle(host_exec, tmp_path, L, N, two_sz, D, c, seed, switch):
    from oracle.dmrgu1 import DMRGU1
    from oracle.mpsu1 import MPSU1
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, two_sz, D, q.SYM_U1, seed, c))
    h, V = q.make_integrals(L, seed + 1)
    s64, st = _run(host_exec, tmp_path, m, h, V, switch)
    ref = m.psi_to_flat(DMRGU1(h, V, N, two_sz).sigma(m))
    assert np.linalg.norm(s64 - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.linalg.norm(st - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("L,N,D,c,mps_seed,int_seed,switch", [(6, 6, 8, 2, 3, 4, 2), (6, 6, 8, 2, 3, 4, 3),
                                                               (7, 5, 12, 3, 5, 6, 3)])
def test_switched_sweeps_match_the_oracle(host_exec, tmp_path, L, N, D, c, mps_seed, int_seed, switch):
    """Sweeps move the centre across the switch in both directions: blocks are renormalized
    as normal on one side and complementary on the other, and the switching enlargement is
    rebuilt at every crossing."""
    from oracle.dmrgu1 import DMRGU1
    from oracle.mpsu1 import MPSU1
    two = N % 2
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, two, D, q.SYM_U1, mps_seed, c))
    h, V = q.make_integrals(L, int_seed)
    E = _sweeps(host_exec, tmp_path, m, h, V, D, 2, switch)
    Eo, _, _ = DMRGU1(h, V, N, two).sweeps(m, D, 2, tol=1e-12)
    assert np.abs(E - np.array(Eo)).max() <= 1e-9


def test_switched_rdm1_equals_unswitched(host_exec, tmp_path):
    """With the switch on, the 1-RDM at the last centre is taken on an environment rebuilt with
    normal pairs on the left (then the switched one is restored): same matrix, and its trace
    is N."""
    from oracle.mpsu1 import MPSU1
    L, N = 6, 6
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, 16, q.SYM_U1, 9, L - 2))
    h, V = q.make_integrals(L, 10)
    fin, fout = str(tmp_path / "r_in.bin"), str(tmp_path / "r_out.bin")
    _write(fin, m, h, V)
    g = []
    for switch in (0, 3):
        r = subprocess.run([host_exec, fin, fout, "rdm1"], capture_output=True, text=True, timeout=600,
                           env=_env(switch))
        assert r.returncode == 0, r.stderr
        g.append(np.fromfile(fout, "<f8").reshape(L, L))
    assert np.abs(g[1] - g[0]).max() <= 1e-12
    assert abs(np.trace(g[0]) - N) <= 1e-10


@pytest.mark.parametrize("switch,sum_gemm", [(0, 1), (3, -1)])
def test_operator_sum_forms_match_the_oracle(host_exec, tmp_path, switch, sum_gemm):
    """The GEMM form of the operator sums without the switch, and the block-by-block form
    with it: the same sigma and sweep energies as the oracle."""
    from oracle.dmrgu1 import DMRGU1
    from oracle.mpsu1 import MPSU1
    L, N, D, c = 8, 8, 32, 3
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, D, q.SYM_U1, 7, c))
    h, V = q.make_integrals(L, 8)
    s64, st = _run(host_exec, tmp_path, m, h, V, switch, sum_gemm)
    ref = m.psi_to_flat(DMRGU1(h, V, N, 0).sigma(m))
    assert np.linalg.norm(s64 - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.linalg.norm(st - ref) <= 1e-12 * np.linalg.norm(ref)
    m2 = MPSU1.from_raw(q.random_mps_blocks(6, 6, 0, 8, q.SYM_U1, 3, 2))
    h2, V2 = q.make_integrals(6, 4)
    E = _sweeps(host_exec, tmp_path, m2, h2, V2, 8, 2, switch, sum_gemm)
    Eo, _, _ = DMRGU1(h2, V2, 6, 0).sweeps(m2, 8, 2, tol=1e-12)
    assert np.abs(E - np.array(Eo)).max() <= 1e-9


def test_switch_leaves_sigma_unchanged_at_the_cas54_36_shape(host_exec, tmp_path):
    """At L=36, N=54 (D=64, centre 17) the switch changes which block stores the pair
    operators, not H_eff: sigma with the switch at the centre cut and two cuts left of it
    equals the unswitched sigma, and the tiled work items agree with the FP64 task lists."""
    from oracle.mpsu1 import MPSU1
    L, N, D, c = 36, 54, 64, 17
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, D, q.SYM_U1, 3, c))
    h, V = q.make_integrals(L, 4)
    s0, t0 = _run(host_exec, tmp_path, m, h, V, 0)
    assert np.linalg.norm(t0 - s0) <= 1e-13 * np.linalg.norm(s0)
    for switch in (18, 16):
        s1, t1 = _run(host_exec, tmp_path, m, h, V, switch)
        assert np.linalg.norm(s1 - s0) <= 1e-13 * np.linalg.norm(s0)
        assert np.linalg.norm(t1 - s0) <= 1e-13 * np.linalg.norm(s0)


@pytest.mark.parametrize("L,N,two_sz,D,c,seed,switch", [(4, 4, 0, 8, 1, 3, 0), (5, 5, 1, 8, 1, 3, 0),
                                                         (6, 5, 1, 16, 0, 6, 0), (8, 8, 0, 32, 3, 7, 0),
                                                         (7, 7, 1, 16, 5, 8, 3)])
def test_rdm2_by_centre_walk_matches_brute_force(host_exec, tmp_path, L, N, two_sz, D, c, seed, switch):
    """The library's centre-walk 2-RDM (every element measured once at its centre, exact
    moves) against the 2-RDM of the expanded MPS vector, element by element; afterwards the
    MPS is the one imported (same psi at the same centre) and its energy equals
    sum h gamma + 1/2 sum V Gamma."""
    from oracle.fci import FCI
    from oracle.mpsu1 import MPSU1, Projector
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, two_sz, D, q.SYM_U1, seed, c))
    h, V = q.make_integrals(L, seed + 1)
    fin, fout = str(tmp_path / "w_in.bin"), str(tmp_path / "w_out.bin")
    _write(fin, m, h, V)
    r = subprocess.run([host_exec, fin, fout, "rdm2sweep"], capture_output=True, text=True, timeout=600,
                       env=_env(switch))
    assert r.returncode == 0, r.stderr
    out = np.fromfile(fout, "<f8")
    G = out[:L ** 4].reshape(L, L, L, L)
    f = FCI(h, V, N, two_sz)
    v = Projector(m, f.space).apply(m.psi)
    g1, Gf = f.rdm12(v / np.linalg.norm(v))
    assert np.abs(G - Gf).max() <= 1e-12 * max(1.0, np.abs(Gf).max())
    rest = out[L ** 4:]
    n = rest.size // 2
    psi, sig = rest[:n], rest[n:]
    assert np.array_equal(psi, m.psi_to_flat())        # the MPS is restored after the walk
    E = psi @ sig / (psi @ psi)
    assert abs(np.sum(h * g1) + 0.5 * np.sum(V * G) - E) <= 1e-10 * abs(E)


def test_rdm2_by_centre_walk_identities_at_L12(host_exec, tmp_path):
    """Beyond brute-force sizes (L=12, N=12, D=32): properties of any 2-RDM of the state —
    sum_pr Gamma_pprr = N(N-1), the symmetries Gamma_pqrs = Gamma_rspq = Gamma_qpsr, and the
    energy of the MPS (from H_eff psi after the walk) equal to sum h gamma + 1/2 sum V Gamma
    with gamma_pq = sum_r Gamma_pqrr / (N-1); the last weighs every element by V."""
    from oracle.mpsu1 import MPSU1
    L, N, D, c = 12, 12, 32, 5
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, D, q.SYM_U1, 5, c))
    h, V = q.make_integrals(L, 6)
    fin, fout = str(tmp_path / "w_in.bin"), str(tmp_path / "w_out.bin")
    _write(fin, m, h, V)
    r = subprocess.run([host_exec, fin, fout, "rdm2sweep"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    out = np.fromfile(fout, "<f8")
    G = out[:L ** 4].reshape(L, L, L, L)
    assert abs(np.einsum("pprr->", G) - N * (N - 1)) <= 1e-10
    assert np.abs(G - G.transpose(2, 3, 0, 1)).max() <= 1e-13
    assert np.abs(G - G.transpose(1, 0, 3, 2)).max() <= 1e-13
    g = np.einsum("pqrr->pq", G) / (N - 1)
    rest = out[L ** 4:]
    n = rest.size // 2
    psi, sig = rest[:n], rest[n:]
    E = psi @ sig / (psi @ psi)
    assert abs(np.sum(h * g) + 0.5 * np.sum(V * G) - E) <= 1e-11 * abs(E)


# SU(2) spin adaptation: the library's reduced-operator task lists (rules_su2.cpp) and its
# SU(2) truncation and centre moves against the operator-based SU(2) oracle.
def _write_su2(path, mps, h, V):
    from oracle.dmrgsu2 import export_abi_su2
    nsec, sec, data = export_abi_su2(mps)
    with open(path, "wb") as f:
        f.write(struct.pack("<7q", mps.L, mps.N, mps.two_s, mps.center, len(nsec), len(sec), len(data)))
        f.write(np.ascontiguousarray(h, "<f8").tobytes())
        f.write(np.ascontiguousarray(V, "<f8").tobytes())
        f.write(np.asarray(nsec, "<i4").tobytes())
        f.write(np.asarray(sec, "<i4").tobytes())
        f.write(np.asarray(data, "<f8").tobytes())


def _run_su2(exe, tmp, mps, h, V, extra=()):
    fin, fout = str(tmp / "su2_in.bin"), str(tmp / "su2_out.bin")
    _write_su2(fin, mps, h, V)
    r = subprocess.run([exe, fin, fout] + list(extra), capture_output=True, text=True, timeout=900,
                       env=dict(os.environ, HOST_EXEC_SU2="1"))
    assert r.returncode == 0, r.stderr
    return np.fromfile(fout, "<f8")


@pytest.mark.parametrize("L,N,two_s,D,c", [(4, 4, 0, 16, 1), (5, 5, 1, 8, 1), (5, 4, 2, 8, 2), (6, 6, 0, 6, 0),
                                           (6, 5, 1, 6, 4), (6, 6, 2, 5, 2), (8, 8, 0, 20, 3)])
def test_su2_task_lists_match_the_oracle(host_exec, tmp_path, L, N, two_s, D, c):
    from oracle.dmrgsu2 import DMRGSU2, MPSSU2
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 5, c))
    h, V = q.make_integrals(L, 11)
    out = _run_su2(host_exec, tmp_path, mps, h, V)
    n = len(out) // 2
    ref = mps.psi_to_flat(DMRGSU2(h, V, N, two_s).sigma(mps))
    assert n == len(ref)
    for s in (out[:n], out[n:]):
        assert np.linalg.norm(s - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("L,N,two_s,D,c", [(6, 6, 0, 400, 2), (6, 5, 1, 8, 2), (6, 6, 2, 10, 1)])
def test_su2_engine_sweeps_match_the_oracle(host_exec, tmp_path, L, N, two_s, D, c):
    """Davidson, SU(2) truncation (multiplet weights of sectors coupled to several
    partner spins) and the 6j recoupling of the two-site guess at every centre move,
    two sweeps; at the exact bond dimension (first case) the spin-filtered FCI energy."""
    from oracle.dmrgsu2 import DMRGSU2, MPSSU2
    from oracle.fci import FCI
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 2, c))
    h, V = q.make_integrals(L, 13)
    E = _run_su2(host_exec, tmp_path, mps, h, V, ["sweep", str(D), "2", "1e-10"])
    Eo, _, _ = DMRGSU2(h, V, N, two_s).sweeps(mps, D, nsweeps=2, tol=1e-12)
    assert np.abs(E - np.array(Eo)).max() <= 1e-9
    if D == 400:
        e_fci, _ = FCI(h, V, N, two_s).ground_state(two_s=two_s)
        assert abs(E[-1] - e_fci) <= 1e-9


@pytest.mark.parametrize("L,N,two_s,D,c", [(8, 8, 0, 20, 3), (12, 5, 1, 100, 5)])
def test_mixed_davidson_policy_reaches_the_fp64_energy_with_few_fp64_products(host_exec, tmp_path, L, N, two_s,
                                                                               D, c):
    """The mixed policy (BF16 -> BF16x3 -> FP64 residual correction) against the FP64
    Davidson from the same start, with the BF16 forms emulated on the host as the FP64
    product plus a deterministic relative perturbation of each sigma element of their
    rounding size (2^-9, 2^-18). Both converge to the residual 1e-8; the energies agree to
    1e-10 and the mixed solve spends at most 8 FP64 products (one per outer check of the
    refinement) where the FP64 solve spends all of its."""
    from oracle.dmrgsu2 import MPSSU2
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 5, c))
    h, V = q.make_integrals(L, 11)
    o = _run_su2(host_exec, tmp_path, mps, h, V, ["davidson"])
    e64, emix, r64, rmix, c64, cmix, n64, nmix64, nbf16, nx3 = o[:10]
    assert c64 == 1.0 and cmix == 1.0
    assert r64 < 1e-8 and rmix < 1e-8
    assert abs(emix - e64) < 1e-10
    assert nmix64 <= 8 and n64 > 4 * nmix64
    assert nbf16 + nx3 > 0


@pytest.mark.parametrize("L,N,two_s,D", [(6, 6, 0, 8), (7, 7, 1, 10)])
def test_su2_rdm1_is_the_energy_gradient_in_h(host_exec, tmp_path, L, N, two_s, D):
    """The SU(2) one-particle density matrix at the centre (L-2, L-1) against central
    differences of E = psi^T H_eff psi / psi^T psi in symmetric perturbations of h (E is
    linear in h at fixed MPS), with H_eff from the library's SU(2) task lists (which match
    the oracle); trace N, symmetric."""
    from oracle.dmrgsu2 import MPSSU2
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 5, L - 2))
    h, V = q.make_integrals(L, 11)
    g = _run_su2(host_exec, tmp_path, mps, h, V, ["rdm1"]).reshape(L, L)
    assert abs(np.trace(g) - N) < 1e-12
    assert np.abs(g - g.T).max() < 1e-14
    psi = mps.psi_to_flat()

    def energy(hh):
        out = _run_su2(host_exec, tmp_path, mps, hh, V)
        s = out[:len(out) // 2]
        return psi @ s / (psi @ psi)
    eps = 1e-5
    for p, r in [(0, 0), (1, 3), (2, L - 1), (L - 1, L - 1)]:
        dh = np.zeros((L, L))
        dh[p, r] += 1.0
        if p != r:
            dh[r, p] += 1.0
        fd = (energy(h + eps * dh) - energy(h - eps * dh)) / (2 * eps)
        an = g[p, r] + (g[r, p] if p != r else 0.0)
        assert abs(fd - an) <= 1e-8 * max(1.0, abs(an))


@pytest.mark.parametrize("L,N,two_s,D", [(5, 5, 1, 8), (5, 4, 2, 8)])
def test_su2_rdm2_equals_the_fci_rdm_of_the_expanded_state(host_exec, tmp_path, L, N, two_s, D):
    """The SU(2) two-particle density matrix (environment probes with unit integrals on
    each permutation orbit of (pq|rs)) against the plain definition: the two-site state
    expanded to determinants (Clebsch-Gordan map of its reduced elements, the projector of
    the oracle tests), its 2-RDM by the FCI oracle's E_pq action, averaged over the 8
    permutations; gamma the same way; and E = sum h gamma + 1/2 sum V Gamma."""
    from oracle.dmrgsu2 import DMRGSU2, MPSSU2
    from oracle.fci import FCI
    from tests.test_oracle_dmrgsu2 import projector
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 5, L - 2))
    h, V = q.make_integrals(L, 11)
    G = _run_su2(host_exec, tmp_path, mps, h, V, ["rdm2"]).reshape(L, L, L, L)
    g = _run_su2(host_exec, tmp_path, mps, h, V, ["rdm1"]).reshape(L, L)
    P, pairs, space = projector(mps)
    x = np.array([mps.psi[a, b] for a, b in pairs])
    v = P @ x
    g1, Gf = FCI(h, V, N, two_s).rdm12(v / np.linalg.norm(v))
    axes = [(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2),
            (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0), (3, 2, 1, 0)]
    Gs = sum(Gf.transpose(a) for a in axes) / 8.0
    assert np.abs(G - Gs).max() <= 1e-10
    assert np.abs(g - g1).max() <= 1e-10
    sig = mps.psi_to_flat(DMRGSU2(h, V, N, two_s).sigma(mps))
    psi = mps.psi_to_flat()
    E = psi @ sig / (psi @ psi)
    assert abs(np.sum(h * g) + 0.5 * np.sum(V * G) - E) <= 1e-10 * abs(E)


# SU(2) with the normal/complementary switch: left blocks past the switch cut hold P^k, Q^k
# of the orbitals to their right (formed from their A^k, B^k at the switch), right blocks
# beyond it hold A^k, B^k of their own orbitals, and the centre terms pair the sides
# accordingly. The oracle keeps normal operators on both sides, so its sigma does not
# depend on the switch.
@pytest.mark.parametrize("L,N,two_s,D,c,switch", [(8, 8, 0, 20, 3, s) for s in range(1, 8)] +
                         [(7, 6, 2, 8, 2, 1), (7, 6, 2, 8, 2, 3), (7, 6, 2, 8, 2, 5), (6, 5, 1, 6, 4, 2),
                          (6, 5, 1, 6, 4, 5), (5, 5, 1, 8, 1, 2)])
def test_su2_switched_task_lists_match_the_oracle(host_exec, tmp_path, L, N, two_s, D, c, switch):
    from oracle.dmrgsu2 import DMRGSU2, MPSSU2
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 5, c))
    h, V = q.make_integrals(L, 11)
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    _write_su2(fin, mps, h, V)
    r = subprocess.run([host_exec, fin, fout], capture_output=True, text=True, timeout=900,
                       env=dict(_env(switch), HOST_EXEC_SU2="1"))
    assert r.returncode == 0, r.stderr
    out = np.fromfile(fout, "<f8")
    n = len(out) // 2
    ref = mps.psi_to_flat(DMRGSU2(h, V, N, two_s).sigma(mps))
    assert n == len(ref)
    for s in (out[:n], out[n:]):
        assert np.linalg.norm(s - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("L,N,two_s,D,c,switch", [(6, 6, 0, 8, 2, 3), (6, 5, 1, 8, 2, 2), (7, 7, 1, 10, 2, 3)])
def test_su2_switched_sweeps_match_the_oracle(host_exec, tmp_path, L, N, two_s, D, c, switch):
    """Two sweeps across the switch cut in both directions (truncation, renormalization
    of normal and complementary pairs, the switching enlargement on either side)."""
    from oracle.dmrgsu2 import DMRGSU2, MPSSU2
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 2, c))
    h, V = q.make_integrals(L, 13)
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    _write_su2(fin, mps, h, V)
    r = subprocess.run([host_exec, fin, fout, "sweep", str(D), "2", "1e-10"], capture_output=True, text=True,
                       timeout=900, env=dict(_env(switch), HOST_EXEC_SU2="1"))
    assert r.returncode == 0, r.stderr
    E = np.fromfile(fout, "<f8")
    Eo, _, _ = DMRGSU2(h, V, N, two_s).sweeps(mps, D, nsweeps=2, tol=1e-12)
    assert np.abs(E - np.array(Eo)).max() <= 1e-9


def test_su2_switch_leaves_sigma_unchanged_after_moves(host_exec, tmp_path):
    """Exact centre moves in both directions renormalize blocks on either side of the
    switch; at every centre reached the wavefunction and sigma equal those without it."""
    from oracle.dmrgsu2 import MPSSU2
    L, N, two_s, D, c = 6, 6, 0, 8, 2
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 2, c))
    h, V = q.make_integrals(L, 13)
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    _write_su2(fin, mps, h, V)

    def run(switch, targets):
        r = subprocess.run([host_exec, fin, fout, "moveto", targets], capture_output=True, text=True, timeout=900,
                           env=dict(_env(switch), HOST_EXEC_SU2="1"))
        assert r.returncode == 0, r.stderr
        o = np.fromfile(fout, "<f8")
        return o[:len(o) // 2], o[len(o) // 2:]

    for targets in ("0,4", "4,1", "0,4,0"):
        p0, s0 = run(0, targets)
        for switch in (1, 2, 3, 4):
            p1, s1 = run(switch, targets)
            assert np.abs(p1 - p0).max() <= 1e-13
            assert np.linalg.norm(s1 - s0) <= 1e-13 * np.linalg.norm(s0)


def test_su2_switched_rdm1_and_rdm2_equal_unswitched(host_exec, tmp_path):
    """With the switch the blocks at the centre (L-2, L-1) hold complementary pairs on the
    left: the one-particle density matrix is taken after a rebuild with normal pairs on the
    left (the switched environment is restored), and the probes of the two-particle density
    matrix read <H_eff> of whichever partition is built; both equal the unswitched ones."""
    from oracle.dmrgsu2 import MPSSU2
    L, N, two_s, D = 6, 6, 0, 8
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 5, L - 2))
    h, V = q.make_integrals(L, 11)
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    _write_su2(fin, mps, h, V)
    out = {}
    for switch in (0, 3):
        for mode in ("rdm1", "rdm2"):
            r = subprocess.run([host_exec, fin, fout, mode], capture_output=True, text=True, timeout=900,
                               env=dict(_env(switch), HOST_EXEC_SU2="1"))
            assert r.returncode == 0, r.stderr
            out[switch, mode] = np.fromfile(fout, "<f8")
    assert np.abs(out[3, "rdm1"] - out[0, "rdm1"]).max() <= 1e-12
    assert np.abs(out[3, "rdm2"] - out[0, "rdm2"]).max() <= 1e-11


@pytest.mark.parametrize("L,N,two_s,D,c,budget", [(8, 8, 0, 20, 3, 4096), (8, 8, 0, 20, 3, 1), (6, 5, 1, 6, 4, 2048)])
def test_tiled_passes_match_the_oracle(host_exec, tmp_path, L, N, two_s, D, c, budget):
    """The tiled work items with the T arena split into passes (budget: bytes of one plane
    per pass; 1 gives one T_t per pass): evaluated pass by pass, each pass's T_t forgotten
    before the next, sigma equals the oracle's; the unbounded plan has one pass."""
    from oracle.dmrgsu2 import DMRGSU2, MPSSU2
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 5, c))
    h, V = q.make_integrals(L, 11)
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    _write_su2(fin, mps, h, V)
    ref = mps.psi_to_flat(DMRGSU2(h, V, N, two_s).sigma(mps))
    passes = {}
    for b in (0, budget):
        r = subprocess.run([host_exec, fin, fout], capture_output=True, text=True, timeout=900,
                           env=dict(os.environ, HOST_EXEC_SU2="1", HOST_EXEC_T_BUDGET=str(b)))
        assert r.returncode == 0, r.stderr
        passes[b] = int(r.stderr.split("tiled_passes=")[1].split()[0])
        out = np.fromfile(fout, "<f8")
        n = len(out) // 2
        assert np.linalg.norm(out[n:] - ref) <= 1e-12 * np.linalg.norm(ref)
    assert passes[0] == 1 and passes[budget] > 1


@pytest.mark.parametrize("sym,L,N,s,D,c,eps,dmin", [("u1", 6, 6, 0, 16, 2, 1e-4, 2), ("su2", 6, 6, 0, 12, 2, 1e-2, 2),
                                                    ("su2", 6, 5, 1, 12, 2, 1e-3, 3)])
def test_dynamic_selection_sweeps_match_the_oracle(host_exec, tmp_path, sym, L, N, s, D, c, eps, dmin):
    """Sweeps whose truncations keep the smallest bond dimension in [D_min, D] with a
    discarded weight of at most eps, against the oracle's sweeps with the same rule:
    energies (1e-9) and the largest number of states kept."""
    if sym == "u1":
        from oracle.dmrgu1 import DMRGU1
        from oracle.mpsu1 import MPSU1
        mps = MPSU1.from_raw(q.random_mps_blocks(L, N, s, D, q.SYM_U1, 2, c))
        h, V = q.make_integrals(L, 13)
        fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
        _write(fin, mps, h, V)
        env = _env(0)
        orc = DMRGU1(h, V, N, s)
    else:
        from oracle.dmrgsu2 import DMRGSU2, MPSSU2
        mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, s, D, q.SYM_SU2, 2, c))
        h, V = q.make_integrals(L, 13)
        fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
        _write_su2(fin, mps, h, V)
        env = dict(_env(0), HOST_EXEC_SU2="1")
        orc = DMRGSU2(h, V, N, s)
    r = subprocess.run([host_exec, fin, fout, "sweep", str(D), "2", "1e-10", repr(eps), str(dmin)],
                       capture_output=True, text=True, timeout=900, env=env)
    assert r.returncode == 0, r.stderr
    out = np.fromfile(fout, "<f8")
    E, maxk, sumk = out[:-2], int(out[-2]), int(out[-1])
    Eo, _, _ = orc.sweeps(mps, D, nsweeps=2, tol=1e-12, trunc_eps=eps, D_min=dmin)
    assert np.abs(E - np.array(Eo)).max() <= 1e-9
    assert (maxk, sumk) == (orc.max_kept, orc.total_kept)
    # the rule kept fewer states than the fixed bond dimension does
    orc.sweeps(mps, D, nsweeps=2, tol=1e-12)
    assert sumk < orc.total_kept


@pytest.mark.parametrize("L,N,two_s,D,c", [(5, 5, 1, 8, 1), (5, 4, 2, 8, 2), (6, 6, 0, 8, 2)])
def test_su2_rdm2_by_expanded_walk_equals_the_fci_rdm(host_exec, tmp_path, L, N, two_s, D, c):
    """The SU(2) two-particle density matrix element by element: the state's M = S
    expansion (its site tensors and two-site state written through Clebsch-Gordan
    coefficients as a U(1) MPS) walked by the U(1) centre walk, against the FCI 2-RDM of
    the determinant-expanded state (no permutation average); afterwards the SU(2) state
    and its sigma are unchanged."""
    from oracle.dmrgsu2 import DMRGSU2, MPSSU2
    from oracle.fci import FCI
    from tests.test_oracle_dmrgsu2 import projector
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 5, c))
    h, V = q.make_integrals(L, 11)
    out = _run_su2(host_exec, tmp_path, mps, h, V, ["rdm2sweep"])
    G = out[:L ** 4].reshape(L, L, L, L)
    rest = out[L ** 4:]
    ps, sg = rest[:len(rest) // 2], rest[len(rest) // 2:]
    P, pairs, space = projector(mps)
    x = np.array([mps.psi[a, b] for a, b in pairs])
    v = P @ x
    _, Gf = FCI(h, V, N, two_s).rdm12(v / np.linalg.norm(v))
    assert np.abs(G - Gf).max() <= 1e-10
    psi = mps.psi_to_flat()
    assert np.abs(ps - psi).max() <= 1e-12
    ref = mps.psi_to_flat(DMRGSU2(h, V, N, two_s).sigma(mps))
    assert np.linalg.norm(sg - ref) <= 1e-12 * np.linalg.norm(ref)


def _orbital_rdm_ref(dets, v, L):
    from oracle import orbital_qi as qi
    R = np.zeros((L, L, 16, 16))
    for i in range(L):
        for j in range(i + 1, L):
            R[i, j] = qi.two_orbital_rdm(dets, v, i, j)
    return R


@pytest.mark.parametrize("L,N,two_sz,D,c,seed,switch,sum_gemm", [(4, 4, 0, 8, 1, 3, 0, 0), (5, 5, 1, 8, 1, 3, 0, 0),
                                                                  (6, 5, 1, 16, 0, 6, 0, 0), (7, 7, 1, 16, 5, 8, 3, 0),
                                                                  (7, 7, 1, 16, 5, 8, 4, 1), (8, 8, 0, 32, 3, 7, 0, -1)])
def test_orbital_rdm_by_centre_walk_matches_the_partial_trace(host_exec, tmp_path, L, N, two_sz, D, c, seed, switch,
                                                                sum_gemm):
    """Two-orbital density matrices of every pair by one walk of the centre (right blocks
    keeping the matrix units of their orbitals) against the partial trace of the expanded
    MPS vector, element by element; afterwards the MPS is the one imported."""
    from oracle.fci import FCI
    from oracle.mpsu1 import MPSU1, Projector
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, two_sz, D, q.SYM_U1, seed, c))
    h, V = q.make_integrals(L, seed + 1)
    fin, fout = str(tmp_path / "o_in.bin"), str(tmp_path / "o_out.bin")
    _write(fin, m, h, V)
    r = subprocess.run([host_exec, fin, fout, "orbrdm"], capture_output=True, text=True, timeout=600,
                       env=_env(switch, sum_gemm))
    assert r.returncode == 0, r.stderr
    out = np.fromfile(fout, "<f8")
    R = out[:L * L * 256].reshape(L, L, 16, 16)
    f = FCI(h, V, N, two_sz)
    v = Projector(m, f.space).apply(m.psi)
    assert np.abs(R - _orbital_rdm_ref(f.space.dets, v, L)).max() <= 1e-12
    rest = out[L * L * 256:]
    assert np.array_equal(rest[:rest.size // 2], m.psi_to_flat())


@pytest.mark.parametrize("L,N,two_s,D,c", [(5, 5, 1, 8, 1), (5, 4, 2, 8, 2), (6, 6, 0, 8, 2), (5, 5, 3, 6, 2)])
def test_su2_orbital_rdm_is_the_multiplet_average(host_exec, tmp_path, L, N, two_s, D, c):
    """SU(2): the same walk on the expansion of each of the state's 2S + 1 components,
    averaged, against the oracle's multiplet average of the partial trace (components by S_-
    from the determinant-expanded M = S state); the SU(2) state and its sigma are unchanged
    afterwards."""
    from oracle.dmrgsu2 import DMRGSU2, MPSSU2
    from tests.test_oracle_dmrgsu2 import projector
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 5, c))
    h, V = q.make_integrals(L, 11)
    out = _run_su2(host_exec, tmp_path, mps, h, V, ["orbrdm"])
    R = out[:L * L * 256].reshape(L, L, 16, 16)
    from oracle import orbital_qi as qi
    P, pairs, space = projector(mps)
    v = P @ np.array([mps.psi[a, b] for a, b in pairs])
    for i in range(L):
        for j in range(i + 1, L):
            assert np.abs(R[i, j] - qi.multiplet_rdm(L, N, two_s, v, i, j)).max() <= 1e-12
    rest = out[L * L * 256:]
    ps, sg = rest[:rest.size // 2], rest[rest.size // 2:]
    assert np.abs(ps - mps.psi_to_flat()).max() <= 1e-12
    ref = mps.psi_to_flat(DMRGSU2(h, V, N, two_s).sigma(mps))
    assert np.linalg.norm(sg - ref) <= 1e-12 * np.linalg.norm(ref)


def test_orbital_rdm_identities_at_L12(host_exec, tmp_path):
    """Beyond brute-force sizes (L=12, N=12, D=32): every rho_ij has unit trace, is symmetric
    and positive semidefinite, and the one-orbital matrix of orbital i is the same from
    every pair that holds it."""
    from oracle.mpsu1 import MPSU1
    L, N, D, c = 12, 12, 32, 5
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, D, q.SYM_U1, 5, c))
    h, V = q.make_integrals(L, 6)
    fin, fout = str(tmp_path / "o_in.bin"), str(tmp_path / "o_out.bin")
    _write(fin, m, h, V)
    r = subprocess.run([host_exec, fin, fout, "orbrdm"], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr
    R = np.fromfile(fout, "<f8")[:L * L * 256].reshape(L, L, 16, 16)
    one = {}
    for i in range(L):
        for j in range(i + 1, L):
            rr = R[i, j]
            assert abs(np.trace(rr) - 1) <= 1e-12
            assert np.abs(rr - rr.T).max() <= 1e-13
            assert np.linalg.eigvalsh(rr).min() >= -1e-12
            t = rr.reshape(4, 4, 4, 4)
            one.setdefault(i, []).append(np.einsum("xyzy->xz", t))
            one.setdefault(j, []).append(np.einsum("xyxz->yz", t))
    for i, mats in one.items():
        assert max(np.abs(mm - mats[0]).max() for mm in mats) <= 1e-12


def _write_arrays(path, L, N, two_s, center, nsec, sec, data, h, V):
    with open(path, "wb") as f:
        f.write(struct.pack("<7q", L, N, two_s, center, len(nsec), len(sec), len(data)))
        f.write(np.ascontiguousarray(h, "<f8").tobytes())
        f.write(np.ascontiguousarray(V, "<f8").tobytes())
        f.write(np.asarray(nsec, "<i4").tobytes())
        f.write(np.asarray(sec, "<i4").tobytes())
        f.write(np.asarray(data, "<f8").tobytes())


@pytest.mark.parametrize("sym,L,N,two_s,nmax", [(0, 5, 4, 0, 20), (0, 6, 5, 1, 40), (1, 5, 4, 0, 12),
                                                (1, 6, 5, 1, 30), (1, 6, 6, 2, 30)])
def test_config_mps_is_the_configuration_state(host_exec, tmp_path, sym, L, N, two_s, nmax):
    """The library's MPS of sum_k c_k |config_k> (selected configurations, random c_k)
    carries exactly that state: its 2-RDM by the centre walk equals the FCI 2-RDM of the
    oracle's determinant expansion of the configurations (CSFs by Clebsch-Gordan
    coefficients for SU(2)), element by element."""
    import paper_2603_28648_b300 as qd
    from oracle import configs as oc
    from oracle.fci import FCI
    from tests._lib import ensure_built
    lib = qd.load(ensure_built())
    h, V = q.make_integrals(L, 5)
    steps, _ = qd.select_configs(sym, h, V, N, two_s, nmax, lib=lib)
    coef = np.random.default_rng(1).normal(size=len(steps))
    center, nsec, sec, data = qd.config_mps(sym, L, N, two_s, steps, coef, lib=lib)
    fin, fout = str(tmp_path / "c_in.bin"), str(tmp_path / "c_out.bin")
    _write_arrays(fin, L, N, two_s, center, nsec, sec, data, h, V)
    env = dict(os.environ, HOST_EXEC_SU2="1") if sym else dict(os.environ)
    r = subprocess.run([host_exec, fin, fout, "rdm2sweep"], capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr
    G = np.fromfile(fout, "<f8")[:L ** 4].reshape(L, L, L, L)
    _, v = oc.config_vector([tuple(int(x) for x in s) for s in steps], coef, L, N, two_s, bool(sym))
    _, Gf = FCI(h, V, N, two_s).rdm12(v / np.linalg.norm(v))
    assert np.abs(G - Gf).max() <= 1e-12


@pytest.mark.parametrize("sym,L,N,two_s,nmax,D", [(0, 6, 6, 0, 30, 64), (1, 6, 6, 0, 30, 64),
                                                  (1, 6, 5, 1, 20, 64)])
def test_warmup_half_sweep_bounds_and_limit(host_exec, tmp_path, sym, L, N, two_s, nmax, D):
    """The warm-up from the reference alone (the other selected configurations only span the
    left bases): the first solve, at the right end, is at or below the CI energy of the
    selected configurations (its space contains theirs), and at a bond dimension that
    truncates nothing the following sweeps reach the FCI energy."""
    import scipy.linalg as sl
    import paper_2603_28648_b300 as qd
    from oracle import configs as oc
    from oracle.fci import FCI
    from tests._lib import ensure_built
    lib = qd.load(ensure_built())
    h, V = q.make_integrals(L, 5)
    steps, _ = qd.select_configs(sym, h, V, N, two_s, nmax, lib=lib)
    coef = np.zeros(len(steps))
    coef[0] = 1.0
    center, nsec, sec, data = qd.config_mps(sym, L, N, two_s, steps, coef, lib=lib)
    fin, fout = str(tmp_path / "w_in.bin"), str(tmp_path / "w_out.bin")
    _write_arrays(fin, L, N, two_s, center, nsec, sec, data, h, V)
    env = dict(os.environ, HOST_EXEC_SU2="1") if sym else dict(os.environ)
    r = subprocess.run([host_exec, fin, fout, "warmup", str(D), "2", "1e-10"], capture_output=True, text=True,
                       timeout=900, env=env)
    assert r.returncode == 0, r.stderr
    E = np.fromfile(fout, "<f8")
    f = FCI(h, V, N, two_s)
    P = np.stack([oc.config_vector([tuple(int(x) for x in s)], [1.0], L, N, two_s, bool(sym))[1] for s in steps], 1)
    H = f.matrix()
    e_ci = sl.eigh(P.T @ (H @ P), P.T @ P, eigvals_only=True)[0]
    e_fci, _ = f.ground_state(two_s=two_s)
    assert E[0] <= e_ci + 1e-9
    assert abs(E[-1] - e_fci) <= 1e-8


@pytest.mark.parametrize("seed", [1, 2])
def test_qi_ordering_recovers_the_chain_energy(host_exec, tmp_path, seed):
    """The quantum-information ordering end to end: a half-filled hopping chain (t = -1,
    on-site repulsion 4, weak random couplings) with its orbitals in a hidden order; DMRG at
    D = 16 in the given order, rho_ij of its state (library walk), mutual information and
    Fiedler order (library), integrals reordered, DMRG again; after two such rounds the
    energy equals that of the chain in its true order (1e-6) and lies clearly below the
    energy in the scrambled order."""
    import paper_2603_28648_b300 as qd
    from oracle.mpsu1 import MPSU1
    from tests._lib import ensure_built
    lib = qd.load(ensure_built())
    L, N, D = 8, 8, 16
    rng = np.random.default_rng(seed)
    perm = rng.permutation(L)
    h = 0.01 * rng.normal(size=(L, L))
    h = h + h.T
    for k in range(L - 1):
        h[perm[k], perm[k + 1]] = h[perm[k + 1], perm[k]] = -1.0
    V = np.zeros((L,) * 4)
    for p in range(L):
        V[p, p, p, p] = 4.0

    def dmrg(hh, VV):
        m = MPSU1.from_raw(q.random_mps_blocks(L, N, 0, D, q.SYM_U1, 3, L // 2 - 1))
        fin, fout = str(tmp_path / "q_in.bin"), str(tmp_path / "q_out.bin")
        _write(fin, m, hh, VV)
        r = subprocess.run([host_exec, fin, fout, "sweeprdm", str(D), "4", "1e-9"], capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr
        out = np.fromfile(fout, "<f8")
        return out[3], out[4:].reshape(L, L, 16, 16)

    e_scr, R = dmrg(h, V)
    order = np.arange(L)
    for _ in range(2):
        _, I = qd.orbital_entanglement(R, lib=lib)
        o, _ = qd.fiedler_order(I, lib=lib)
        order = order[o]
        e_qi, R = dmrg(*qd.reorder_integrals(h, V, order))
    e_true, _ = dmrg(*qd.reorder_integrals(h, V, perm))
    assert e_qi <= e_true + 1e-6
    assert e_scr - e_qi > 0.05


@pytest.mark.parametrize("L,N,two_sz,D,c", [(2, 2, 0, 4, 0), (2, 1, -1, 4, 0), (3, 1, 1, 4, 0), (3, 2, 0, 16, 1),
                                            (4, 0, 0, 4, 1), (4, 8, 0, 4, 1), (4, 7, 1, 8, 1), (5, 5, 5, 4, 2)])
def test_degenerate_fillings_and_minimal_chains_u1(host_exec, tmp_path, L, N, two_sz, D, c):
    """The edge cases of the method: the shortest chain (L = 2, both sites at the centre, no
    environment), the empty and the full chain (one state; sigma = 0 and sigma = E_full psi),
    one electron, one hole, the fully polarised state (2Sz = N = L, one state): both
    host-executed forms equal the oracle's sigma."""
    from oracle.dmrgu1 import DMRGU1
    from oracle.mpsu1 import MPSU1
    m = MPSU1.from_raw(q.random_mps_blocks(L, N, two_sz, D, q.SYM_U1, 3, c))
    h, V = q.make_integrals(L, 4)
    s64, st = _run(host_exec, tmp_path, m, h, V)
    ref = m.psi_to_flat(DMRGU1(h, V, N, two_sz).sigma(m))
    scale = max(np.linalg.norm(ref), np.linalg.norm(m.psi_to_flat()))
    assert np.linalg.norm(s64 - ref) <= 1e-13 * scale
    assert np.linalg.norm(st - ref) <= 1e-13 * scale
    if N == 2 * L:
        # the full chain: sigma = (2 sum_p h_pp + sum_pq (2 (pp|qq) - (pq|qp))) psi
        e = 2 * np.trace(h) + sum(2 * V[p, p, r, r] - V[p, r, r, p] for p in range(L) for r in range(L))
        assert np.linalg.norm(s64 - e * m.psi_to_flat()) <= 1e-12 * abs(e) * np.linalg.norm(m.psi_to_flat())
    if N == 0:
        assert not np.any(s64) and not np.any(st)


@pytest.mark.parametrize("L,N,two_s,D,c", [(2, 2, 0, 4, 0), (3, 1, 1, 4, 0), (3, 6, 0, 4, 1), (4, 0, 0, 4, 1),
                                           (4, 4, 4, 4, 1), (3, 3, 3, 4, 1), (5, 9, 1, 6, 2)])
def test_degenerate_fillings_and_minimal_chains_su2(host_exec, tmp_path, L, N, two_s, D, c):
    """SU(2) edge cases: L = 2, one electron, the full and the empty chain, the maximal spin
    S = N/2 (one multiplet), one hole: the reduced-operator task lists equal the SU(2)
    oracle's sigma."""
    from oracle.dmrgsu2 import DMRGSU2, MPSSU2
    mps = MPSSU2.from_raw(q.random_mps_blocks(L, N, two_s, D, q.SYM_SU2, 5, c))
    h, V = q.make_integrals(L, 11)
    out = _run_su2(host_exec, tmp_path, mps, h, V)
    n = out.size // 2
    ref = mps.psi_to_flat(DMRGSU2(h, V, N, two_s).sigma(mps))
    scale = max(np.linalg.norm(ref), np.linalg.norm(mps.psi_to_flat()))
    assert np.linalg.norm(out[:n] - ref) <= 1e-13 * scale
    assert np.linalg.norm(out[n:] - ref) <= 1e-13 * scale


@pytest.mark.parametrize("sym", ["u1", "su2"])
def test_dmrg_scf_macro_iterations_match_the_fci_pipeline(host_exec, tmp_path, sym):
    """Two DMRG-SCF macro-iterations (7 orbitals, 1 core, CAS(4,5), S = 0) with the library's
    own DMRG as the active-space solver (host-executed sweeps at a bond dimension that
    truncates nothing, then Gamma by the walk and gamma = sum_r Gamma_pqrr / (N - 1)), and with
    the FCI oracle as the solver (the lowest 2Sz = 0 state for U(1), the lowest singlet for
    SU(2)): at each macro-iteration the energies agree to 1e-8, the
    density matrices to 1e-7 and the library's orbital gradients from either to 1e-6; the
    steepest-descent rotation between them is the library's."""
    import paper_2603_28648_b300 as qd
    from oracle.fci import FCI
    from tests._lib import ensure_built
    lib = qd.load(ensure_built())
    n, nc, na, N = 7, 1, 5, 4
    h, V = q.make_integrals(n, 21)
    for it in range(2):
        e_core, ha, Va = qd.active_space(h, V, nc, na, lib=lib)
        if sym == "u1":
            from oracle.mpsu1 import MPSU1
            m = MPSU1.from_raw(q.random_mps_blocks(na, N, 0, 16, q.SYM_U1, 3 + it, 1))
            fin = str(tmp_path / "scf_in.bin")
            _write(fin, m, ha, Va)
            env = dict(os.environ)
            D = 16
        else:
            from oracle.dmrgsu2 import MPSSU2
            m = MPSSU2.from_raw(q.random_mps_blocks(na, N, 0, 10, q.SYM_SU2, 3 + it, 1))
            fin = str(tmp_path / "scf_in.bin")
            _write_su2(fin, m, ha, Va)
            env = dict(os.environ, HOST_EXEC_SU2="1")
            D = 10
        fout = str(tmp_path / "scf_out.bin")
        r = subprocess.run([host_exec, fin, fout, "sweepgamma", str(D), "4", "1e-11"], capture_output=True,
                           text=True, timeout=600, env=env)
        assert r.returncode == 0, r.stderr
        out = np.fromfile(fout, "<f8")
        e_dmrg, G2 = out[0] + e_core, out[1:].reshape(na, na, na, na)
        g1 = np.einsum("pqrr->pq", G2) / (N - 1)
        f = FCI(ha, Va, N, 0, e_core)
        # U(1) fixes 2Sz = 0 only (its ground state may be a triplet's M = 0 component);
        # SU(2) fixes S = 0
        e_fci, c = f.ground_state(two_s=0 if sym == "su2" else None)
        f1, f2 = f.rdm12(c)
        assert abs(e_dmrg - e_fci) <= 1e-8
        assert np.abs(g1 - f1).max() <= 1e-7 and np.abs(G2 - f2).max() <= 1e-7
        G = qd.orbital_gradient(h, V, nc, na, g1, G2, lib=lib)
        Gf = qd.orbital_gradient(h, V, nc, na, f1, f2, lib=lib)
        assert np.abs(G - Gf).max() <= 1e-6 * max(1.0, np.abs(Gf).max())
        _, h, V = qd.rotate_orbitals(-0.01 * G, h, V, lib=lib)
