"""Host-side checks of the C ABI: the library builds, loads and exports every
function the header declares; no compute calls (no GPU here)."""
import ctypes
import subprocess

import pytest

from tests._lib import ensure_built, header_functions, HEADER


def test_library_exports_every_declared_symbol():
    path = ensure_built()
    lib = ctypes.CDLL(path)
    names = header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_the_header():
    import paper_2603_28648_b300 as qd
    assert sorted(qd.EXPORTS) == header_functions()


def test_create_without_device_fails_cleanly():
    import paper_2603_28648_b300 as qd
    from tests._lib import cuda_available
    if cuda_available():
        pytest.skip("a device is present")
    ensure_built()
    with pytest.raises(qd.QcdmrgError):
        qd.Context()


def test_header_compiles_as_c():
    r = subprocess.run(["gcc", "-fsyntax-only", "-x", "c", HEADER], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.parametrize("field,value", [("pair_switch", -1), ("sum_gemm", 2), ("sum_gemm", -2),
                                         ("hbm_budget_gb", -1.0), ("tmp_budget_gb", -1.0), ("symmetry", 7),
                                         ("tile_chunk", -1), ("tile_chunk", 65537)])
def test_create_rejects_bad_configuration_before_cuda(field, value):
    """Configuration errors are EINVAL whether or not a device is present (no CUDA call is
    made for them)."""
    import paper_2603_28648_b300 as qd
    path = ensure_built()
    lib = ctypes.CDLL(path)
    cfg = qd.Config(qd.U1, 0, 0.0, 0.0, 0, 0, 0)
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    assert lib.qcdmrg_create(ctypes.byref(h), ctypes.byref(cfg)) == -1
    assert not h.value


def test_su2_accepts_the_normal_complementary_switch():
    """The spin-adapted rules place the pair operators on either side of a cut, so an SU(2)
    context with the normal/complementary switch is a valid configuration: it is not
    rejected as EINVAL (without a GPU the call then fails at its first CUDA call)."""
    import paper_2603_28648_b300 as qd
    path = ensure_built()
    lib = ctypes.CDLL(path)
    cfg = qd.Config(qd.SU2, 0, 0.0, 0.0, 0, 3, 0)
    h = ctypes.c_void_p()
    rc = lib.qcdmrg_create(ctypes.byref(h), ctypes.byref(cfg))
    assert rc != -1
    if rc == 0:
        lib.qcdmrg_destroy(h)
