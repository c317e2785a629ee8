"""Host logic without a GPU: the task lists the library plans — every launch of the
environment build (renormalization, enlargement sums, their GEMM form), the H_eff psi
FP64 segments and the tiled tensor-core work items — stay inside the buffers they
address, no work item is empty, and both H_eff plans count the same algorithmic flops.
The library's host sources are compiled with g++ together with tests/planner_check.cpp,
which records allocations instead of computing."""
import subprocess

import pytest


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    from tests._lib import build_host_executable
    out = build_host_executable("planner_check.cpp", str(tmp_path_factory.mktemp("planner") / "planner_check"))
    if out is None:
        pytest.skip("g++ not available")
    return out


@pytest.mark.parametrize("L,N,D,switch,sum_gemm", [(6, 6, 16, 0, 0), (7, 5, 16, 0, 0), (12, 12, 32, 0, 0),
                                                    (36, 54, 64, 0, 0), (12, 12, 32, 4, 0), (12, 12, 32, 6, 0),
                                                    (36, 54, 64, 18, 0), (36, 54, 4096, 18, 0),
                                                    (36, 54, 1024, 0, 1)])
def test_plans_stay_in_bounds(checker, L, N, D, switch, sum_gemm):
    """switch: cut of the normal/complementary switch (0: normal pairs on the left everywhere;
    at the centre cut L/2 the right blocks switch; at L/2 - 2 the centre uses the mirrored
    decomposition with normal pairs on the right). The D=4096 case is the full CAS(54,36)-shaped
    size of the switched run (task lists only: about 15 s); sum_gemm 1 takes the GEMM form of the
    operator sums without the switch."""
    r = subprocess.run([checker, str(L), str(N), str(D), str(switch), str(sum_gemm)], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fails=0" in r.stdout


@pytest.mark.parametrize("L,N,D,switch", [(6, 6, 16, 0), (12, 12, 64, 0), (36, 54, 256, 0), (12, 12, 64, 6),
                                          (36, 54, 256, 18), (36, 54, 256, 19), (36, 54, 2048, 19),
                                          (36, 54, 4096, 19)])
def test_su2_plans_stay_in_bounds(checker, L, N, D, switch):
    """The SU(2) reduced-operator task lists (environment build, enlargement sums, centre
    FP64 segments and tiled work items) at the CAS(54,36) shape and smaller, with normal
    pairs on the left at every cut and with the switch at and past the centre cut; D = 2048
    and 4096 with the switch one cut past the centre are the benchmark's own launch
    configurations (task lists only: about 14 s each)."""
    r = subprocess.run([checker, str(L), str(N), str(D), str(switch), "0", "1"], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fails=0" in r.stdout
