"""Host logic without a GPU, numerically: the library's own FP64 H_eff task lists
(complementary-operator rules, renormalization, centre plan) executed with plain loops,
and the tiled work items of the tensor-core path evaluated in FP64 (views, panels, term
scalars, T tiles, split stage-2 items), both against the oracle's sigma, on imported
MPS of several shapes, edge centres included, and on the M-expansion of an SU(2) MPS.
tests/host_exec.cpp holds the test-only host executor; the product path still needs CUDA."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

import qcinputs as q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_28648_b300", "csrc")
HOST_SOURCES = ["core.cpp", "rules.cpp", "init.cpp", "engine.cpp", "tiled.cpp"]


@pytest.fixture(scope="module")
def host_exec(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("hostexec") / "host_exec")
    inc = ["-I", CSRC]
    if os.path.isdir("/usr/local/cuda/include"):
        inc += ["-I", "/usr/local/cuda/include"]
    subprocess.run(["g++", "-O2", "-std=c++17", "-pthread"] + inc + [os.path.join(ROOT, "tests", "host_exec.cpp")] +
                   [os.path.join(CSRC, s) for s in HOST_SOURCES] + ["-o", out], check=True)
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


def _run(exe, tmp, mps, h, V):
    fin, fout = str(tmp / "in.bin"), str(tmp / "out.bin")
    _write(fin, mps, h, V)
    r = subprocess.run([exe, fin, fout], capture_output=True, text=True, timeout=600)
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


def test_library_task_lists_on_an_su2_state(host_exec, tmp_path):
    from oracle.fci import FCI
    from oracle.mpssu2 import TangentSU2, to_u1
    t = TangentSU2(7, 7, 1, 2, cap=2, seed=9)
    mps, C = to_u1(t)
    psi = np.random.default_rng(4).normal(size=C.shape[1])
    mps.psi = mps.psi_from_flat(C @ psi)
    h, V = q.make_integrals(7, 13)
    s64, st = _run(host_exec, tmp_path, mps, h, V)
    ref = t.heff(FCI(h, V, 7, 1), psi)
    for s in (s64, st):
        assert np.linalg.norm(C.T @ s - ref) <= 1e-12 * np.linalg.norm(ref)


def _sweeps(exe, tmp, mps, h, V, D, nsweeps):
    fin, fout = str(tmp / "sw_in.bin"), str(tmp / "sw_out.bin")
    _write(fin, mps, h, V)
    r = subprocess.run([exe, fin, fout, "sweep", str(D), str(nsweeps), "1e-10"], capture_output=True,
                       text=True, timeout=600)
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
