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


def test_binding_names_every_status_code():
    import re
    import paper_2603_28648_b300 as qd
    with open(HEADER) as f:
        codes = {int(v): n for n, v in re.findall(r"#define QCDMRG_(E[A-Z]+) \((-\d+)\)", f.read())}
    assert codes and codes == qd._ERRORS


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


def test_extrapolation_recovers_exact_polynomials():
    """qcdmrg_extrapolate (no context, no device): points on a known line or parabola give
    back its coefficients, whose first is the truncation-free energy; the paper's two
    extrapolations are a parabola in 1/D and a line in the truncation error."""
    import numpy as np
    import paper_2603_28648_b300 as qd
    lib = qd.load(ensure_built())
    eps = np.array([3e-5, 2e-5, 1.2e-5, 6e-6, 2.5e-6])
    e0, a = -327.2469, 41.7
    c = qd.extrapolate(eps, e0 + a * eps, 1, lib=lib)
    assert abs(c[0] - e0) < 1e-10 and abs(c[1] - a) < 1e-6 * abs(a)
    inv_d = 1.0 / np.array([1024, 2048, 4096, 8192, 12288])
    b, q2 = 0.93, -310.0
    c = qd.extrapolate(inv_d, e0 + b * inv_d + q2 * inv_d ** 2, 2, lib=lib)
    assert abs(c[0] - e0) < 1e-9 and abs(c[1] - b) < 1e-6 and abs(c[2] - q2) < 1e-3
    # least squares: symmetric noise around a line leaves the line
    x = np.array([1.0, 2.0, 3.0, 4.0])
    y = 2.0 + 0.5 * x + np.array([0.1, -0.1, -0.1, 0.1])
    c = qd.extrapolate(x, y, 1, lib=lib)
    assert abs(c[0] - 2.0) < 1e-12 and abs(c[1] - 0.5) < 1e-12
    # too few points, equal abscissae, bad degree
    for xs, ys, deg in (([1.0], [1.0], 1), ([1.0, 1.0, 1.0], [1.0, 2.0, 3.0], 1), ([1.0, 2.0], [1.0, 2.0], 4)):
        with pytest.raises(qd.QcdmrgError):
            qd.extrapolate(xs, ys, deg, lib=lib)
