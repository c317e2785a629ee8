"""Python binding of libqcdmrg (two-site DMRG H_eff.psi on B300).

Argument marshalling only: every step of the computation runs inside the
CUDA library. Importing the package does not load the library; creating a
Context does, and fails loudly if libqcdmrg.so is missing or no CUDA device
is usable.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqcdmrg.so")

QCDMRG_OK = 0
U1, SU2 = 0, 1
FP64, TF32, BF16, BF16X3 = 0, 1, 2, 3
PRECISIONS = {"fp64": FP64, "tf32": TF32, "bf16": BF16, "bf16x3": BF16X3}

_ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ESTATE", -5: "ENOTCONV",
           -6: "ETIMEOUT", -7: "EIO", -8: "EINTERNAL"}


class QcdmrgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"qcdmrg {_ERRORS.get(code, code)}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("symmetry", ctypes.c_int), ("device", ctypes.c_int),
                ("tmp_budget_gb", ctypes.c_double), ("hbm_budget_gb", ctypes.c_double),
                ("autotune_off", ctypes.c_int), ("pair_switch", ctypes.c_int), ("sum_gemm", ctypes.c_int),
                ("tile_chunk", ctypes.c_int)]


class MpsDesc(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("center", ctypes.c_int),
                ("bond_nsec", ctypes.POINTER(ctypes.c_int)),
                ("bond_sec", ctypes.POINTER(ctypes.c_int))]


class DavOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("m_max", ctypes.c_int),
                ("policy", ctypes.c_int), ("precision", ctypes.c_int), ("tau1", ctypes.c_double),
                ("tau2", ctypes.c_double)]


class SweepOpts(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int), ("dav", DavOpts), ("trunc_eps", ctypes.c_double), ("D_min", ctypes.c_int)]


class SweepReport(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("energy_mixed", ctypes.c_double),
                ("max_trunc_err", ctypes.c_double), ("seconds", ctypes.c_double),
                ("n_hpsi", ctypes.c_int * 4), ("n_steps", ctypes.c_int), ("max_D", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("heff_flops", ctypes.c_double), ("heff_seconds", ctypes.c_double),
                ("env_flops", ctypes.c_double), ("env_seconds", ctypes.c_double),
                ("psi_size", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("live_bytes", ctypes.c_int64),
                ("nterms", ctypes.c_int), ("nlaunch", ctypes.c_int),
                ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64),
                ("evictions", ctypes.c_int), ("restores", ctypes.c_int),
                ("copy_wait_seconds", ctypes.c_double), ("heff_bytes", ctypes.c_double),
                ("tile_kmax", ctypes.c_int), ("tile_width", ctypes.c_int), ("tunes", ctypes.c_int),
                ("tune_seconds", ctypes.c_double), ("f64_tiles", ctypes.c_int64 * 4),
                ("f64_split_tiles", ctypes.c_int64), ("dav_hpsi", ctypes.c_int * 4),
                ("dav_seconds", ctypes.c_double), ("dav_energy_mixed", ctypes.c_double),
                ("tile_chunk", ctypes.c_int), ("tile_passes", ctypes.c_int), ("tile_t_bytes", ctypes.c_int64)]


EXPORTS = [
    "qcdmrg_create", "qcdmrg_destroy", "qcdmrg_last_error", "qcdmrg_load_integrals",
    "qcdmrg_set_target", "qcdmrg_import_mps", "qcdmrg_build_env", "qcdmrg_psi_size",
    "qcdmrg_apply_heff", "qcdmrg_apply_heff_dev", "qcdmrg_stats", "qcdmrg_init_mps",
    "qcdmrg_get_bond", "qcdmrg_get_psi", "qcdmrg_check_device", "qcdmrg_davidson",
    "qcdmrg_truncate", "qcdmrg_move_center", "qcdmrg_sweep", "qcdmrg_heff_diag",
    "qcdmrg_apply_heff_noalloc", "qcdmrg_graph_create", "qcdmrg_graph_launch",
    "qcdmrg_graph_info", "qcdmrg_graph_destroy", "qcdmrg_rdm1", "qcdmrg_rdm2", "qcdmrg_rdm2_sweep", "qcdmrg_set_psi",
    "qcdmrg_export_mps", "qcdmrg_checkpoint", "qcdmrg_restore", "qcdmrg_psi_layout",
    "qcdmrg_energy_grad", "qcdmrg_truncate_dbss", "qcdmrg_extrapolate", "qcdmrg_active_space",
    "qcdmrg_orbital_gradient", "qcdmrg_rotate_orbitals", "qcdmrg_orbital_rdm",
    "qcdmrg_orbital_entanglement", "qcdmrg_fiedler_order", "qcdmrg_select_configs", "qcdmrg_config_mps",
    "qcdmrg_sweep_left", "qcdmrg_ordering_cost", "qcdmrg_refine_order", "qcdmrg_orbital_hessian_diag",
]

_lib = None


def load(path=None):
    """Load the shared library (once). Raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise FileNotFoundError(f"{p} not built: run __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    P = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    lib.qcdmrg_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Config)]
    lib.qcdmrg_destroy.argtypes = [P]
    lib.qcdmrg_last_error.argtypes = [P]
    lib.qcdmrg_last_error.restype = ctypes.c_char_p
    lib.qcdmrg_load_integrals.argtypes = [P, ctypes.c_int, dp, dp, ctypes.c_double]
    lib.qcdmrg_set_target.argtypes = [P, ctypes.c_int, ctypes.c_int]
    lib.qcdmrg_import_mps.argtypes = [P, ctypes.POINTER(MpsDesc), dp, ctypes.c_size_t]
    lib.qcdmrg_build_env.argtypes = [P]
    lib.qcdmrg_psi_size.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
    lib.qcdmrg_apply_heff.argtypes = [P, ctypes.c_int, dp, dp]
    lib.qcdmrg_apply_heff_dev.argtypes = [P, ctypes.c_int, P, P, P]
    lib.qcdmrg_stats.argtypes = [P, ctypes.POINTER(Stats)]
    lib.qcdmrg_init_mps.argtypes = [P, ctypes.c_int, ctypes.c_uint64, ctypes.c_int]
    ip = ctypes.POINTER(ctypes.c_int)
    lib.qcdmrg_get_bond.argtypes = [P, ctypes.c_int, ip, ip, ctypes.c_int]
    lib.qcdmrg_get_psi.argtypes = [P, dp, ctypes.c_size_t]
    lib.qcdmrg_check_device.argtypes = [P]
    lib.qcdmrg_davidson.argtypes = [P, ctypes.POINTER(DavOpts), dp, dp, ctypes.POINTER(ctypes.c_int)]
    lib.qcdmrg_truncate.argtypes = [P, ctypes.c_int, ctypes.c_int, dp]
    lib.qcdmrg_move_center.argtypes = [P, ctypes.c_int]
    lib.qcdmrg_heff_diag.argtypes = [P, dp, ctypes.c_size_t]
    lib.qcdmrg_apply_heff_noalloc.argtypes = [P, P, P, P]
    lib.qcdmrg_graph_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P)]
    lib.qcdmrg_graph_launch.argtypes = [P, P]
    lib.qcdmrg_graph_info.argtypes = [P, dp, ctypes.POINTER(ctypes.c_int)]
    lib.qcdmrg_graph_destroy.argtypes = [P]
    lib.qcdmrg_rdm1.argtypes = [P, dp]
    lib.qcdmrg_rdm2.argtypes = [P, dp]
    lib.qcdmrg_rdm2_sweep.argtypes = [P, dp]
    lib.qcdmrg_export_mps.argtypes = [P, ip, ip, ip, ip, ctypes.c_int, dp, ctypes.c_size_t, ip,
                                      ctypes.POINTER(ctypes.c_size_t)]
    lib.qcdmrg_checkpoint.argtypes = [P, ctypes.c_char_p]
    lib.qcdmrg_psi_layout.argtypes = [P, ip, ctypes.c_int, ip, ctypes.POINTER(ctypes.c_size_t)]
    lib.qcdmrg_energy_grad.argtypes = [P, dp, dp, dp, dp]
    lib.qcdmrg_restore.argtypes = [P, ctypes.c_char_p]
    lib.qcdmrg_set_psi.argtypes = [P, dp, ctypes.c_size_t]
    lib.qcdmrg_sweep.argtypes = [P, ctypes.POINTER(SweepOpts), ctypes.POINTER(SweepReport)]
    lib.qcdmrg_truncate_dbss.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, ip]
    lib.qcdmrg_extrapolate.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp]
    ci = ctypes.c_int
    lib.qcdmrg_active_space.argtypes = [ci, ci, ci, dp, dp, dp, dp, dp]
    lib.qcdmrg_orbital_gradient.argtypes = [ci, ci, ci, dp, dp, dp, dp, dp]
    lib.qcdmrg_rotate_orbitals.argtypes = [ci, dp, dp, dp, dp, dp, dp]
    lib.qcdmrg_orbital_hessian_diag.argtypes = [ci, ci, ci, dp, dp, dp, dp, dp]
    lib.qcdmrg_orbital_rdm.argtypes = [P, dp]
    lib.qcdmrg_orbital_entanglement.argtypes = [ci, dp, dp, dp]
    lib.qcdmrg_fiedler_order.argtypes = [ci, dp, ip, dp]
    u8p = ctypes.POINTER(ctypes.c_uint8)
    lib.qcdmrg_select_configs.argtypes = [ci, ci, ci, ci, dp, dp, ci, u8p, dp, ip]
    lib.qcdmrg_config_mps.argtypes = [ci, ci, ci, ci, ci, u8p, dp, ip, ip, ip, ci, dp, ctypes.c_size_t, ip,
                                      ctypes.POINTER(ctypes.c_size_t)]
    lib.qcdmrg_sweep_left.argtypes = [P, ctypes.POINTER(SweepOpts), ctypes.POINTER(SweepReport)]
    lib.qcdmrg_ordering_cost.argtypes = [ci, dp, ip, ctypes.c_double, dp]
    lib.qcdmrg_refine_order.argtypes = [ci, dp, ctypes.c_double, ip, ci, ip]
    for f in EXPORTS:
        getattr(lib, f).restype = getattr(lib, f).restype or ctypes.c_int
    lib.qcdmrg_last_error.restype = ctypes.c_char_p
    if path is None:
        _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Context:
    """One qcdmrg context (one device, one problem)."""

    def __init__(self, device=0, symmetry=U1, tmp_budget_gb=0.0, hbm_budget_gb=0.0, autotune=True,
                 pair_switch=0, sum_gemm=0, tile_chunk=0, lib=None):
        self.lib = lib or load()
        self.symmetry = symmetry
        self.h = ctypes.c_void_p()
        cfg = Config(symmetry, device, tmp_budget_gb, hbm_budget_gb, 0 if autotune else 1, pair_switch, sum_gemm,
                     tile_chunk)
        rc = self.lib.qcdmrg_create(ctypes.byref(self.h), ctypes.byref(cfg))
        if rc != QCDMRG_OK:
            raise QcdmrgError(rc, "context creation failed (no usable CUDA device?)")

    def _check(self, rc):
        if rc != QCDMRG_OK:
            raise QcdmrgError(rc, self.lib.qcdmrg_last_error(self.h).decode())
        return rc

    def close(self):
        if self.h:
            self.lib.qcdmrg_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_integrals(self, h, V, e_core=0.0):
        h = np.ascontiguousarray(h, dtype=np.float64)
        V = np.ascontiguousarray(V, dtype=np.float64)
        self._check(self.lib.qcdmrg_load_integrals(self.h, h.shape[0], _dptr(h), _dptr(V), e_core))

    def set_target(self, N, two_s):
        self._check(self.lib.qcdmrg_set_target(self.h, N, two_s))

    def import_mps(self, L, center, bond_nsec, bond_sec, data):
        nsec = np.ascontiguousarray(bond_nsec, dtype=np.int32)
        sec = np.ascontiguousarray(bond_sec, dtype=np.int32)
        if sec.size == 0:
            sec = np.zeros(3, dtype=np.int32)
        data = np.ascontiguousarray(data, dtype=np.float64)
        d = MpsDesc(L, center, nsec.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                    sec.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        self._check(self.lib.qcdmrg_import_mps(self.h, ctypes.byref(d), _dptr(data), data.size))

    def init_mps(self, D, seed, center):
        self._check(self.lib.qcdmrg_init_mps(self.h, D, seed, center))

    def bond(self, b):
        n = ctypes.c_int()
        self._check(self.lib.qcdmrg_get_bond(self.h, b, ctypes.byref(n), None, 0))
        buf = (ctypes.c_int * max(1, 3 * n.value))()
        self._check(self.lib.qcdmrg_get_bond(self.h, b, ctypes.byref(n), buf, 3 * n.value))
        return {(buf[3 * i], buf[3 * i + 1]): buf[3 * i + 2] for i in range(n.value)}

    def psi(self):
        n = self.psi_size()
        out = np.empty(n)
        self._check(self.lib.qcdmrg_get_psi(self.h, _dptr(out), n))
        return out

    def set_psi(self, psi):
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        self._check(self.lib.qcdmrg_set_psi(self.h, _dptr(psi), psi.size))

    def build_env(self):
        self._check(self.lib.qcdmrg_build_env(self.h))

    def psi_size(self):
        n = ctypes.c_size_t()
        self._check(self.lib.qcdmrg_psi_size(self.h, ctypes.byref(n)))
        return n.value

    def apply_heff(self, psi, precision=FP64):
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        out = np.empty_like(psi)
        self._check(self.lib.qcdmrg_apply_heff(self.h, precision, _dptr(psi), _dptr(out)))
        return out

    def apply_heff_dev(self, psi_ptr, sigma_ptr, stream=0, precision=FP64):
        self._check(self.lib.qcdmrg_apply_heff_dev(self.h, precision, ctypes.c_void_p(psi_ptr),
                                                   ctypes.c_void_p(sigma_ptr),
                                                   ctypes.c_void_p(stream)))

    @staticmethod
    def dav_opts(tol=1e-6, max_iter=300, m_max=32, policy=0, precision=FP64, tau1=1e-2, tau2=1e-5):
        return DavOpts(tol, max_iter, m_max, policy, precision, tau1, tau2)

    def davidson(self, allow_notconv=False, **kw):
        """Returns (energy, residual, iterations)."""
        e, r, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        o = self.dav_opts(**kw)
        rc = self.lib.qcdmrg_davidson(self.h, ctypes.byref(o), ctypes.byref(e), ctypes.byref(r),
                                      ctypes.byref(it))
        if not (allow_notconv and rc == -5):
            self._check(rc)
        return e.value, r.value, it.value

    def apply_heff_noalloc(self, psi_ptr, sigma_ptr, stream=0):
        """FP64 H_eff psi on device arrays without any allocation in the call
        (stage-1 intermediates in the library's fixed 32 MiB device array)."""
        self._check(self.lib.qcdmrg_apply_heff_noalloc(self.h, ctypes.c_void_p(psi_ptr),
                                                       ctypes.c_void_p(sigma_ptr),
                                                       ctypes.c_void_p(stream)))

    def rdm1(self, L):
        g = np.empty((L, L))
        self._check(self.lib.qcdmrg_rdm1(self.h, _dptr(g)))
        return g

    def export_mps(self):
        """(L, center, bond_nsec, bond_sec, data) in the layout import_mps reads."""
        L, c, ns, nd = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        self._check(self.lib.qcdmrg_export_mps(self.h, ctypes.byref(L), ctypes.byref(c), None, None, 0, None, 0,
                                               ctypes.byref(ns), ctypes.byref(nd)))
        nsec = np.zeros(L.value + 1, dtype=np.int32)
        sec = np.zeros(max(1, 3 * ns.value), dtype=np.int32)
        data = np.zeros(nd.value)
        ipt = ctypes.POINTER(ctypes.c_int)
        self._check(self.lib.qcdmrg_export_mps(self.h, ctypes.byref(L), ctypes.byref(c),
                                               nsec.ctypes.data_as(ipt), sec.ctypes.data_as(ipt), sec.size,
                                               _dptr(data), data.size, ctypes.byref(ns), ctypes.byref(nd)))
        return L.value, c.value, nsec, sec[:3 * ns.value], data

    def psi_layout(self):
        """Sub-blocks of psi in flat order: rows of (x n, x 2Sz, i, j, y n, y 2Sz, rows, cols)."""
        nb, ne = ctypes.c_int(), ctypes.c_size_t()
        self._check(self.lib.qcdmrg_psi_layout(self.h, None, 0, ctypes.byref(nb), ctypes.byref(ne)))
        out = np.zeros((max(1, nb.value), 8), dtype=np.int32)
        self._check(self.lib.qcdmrg_psi_layout(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), out.size,
                                               ctypes.byref(nb), ctypes.byref(ne)))
        return out[:nb.value]

    def energy_grad(self, L, dpsi=True, gamma1=False, gamma2=False):
        """(E, dE/dpsi or None, gamma (L x L) or None, Gamma (L^4) or None) of the current state."""
        e = ctypes.c_double()
        d = np.empty(self.psi_size()) if dpsi else None
        g1 = np.empty((L, L)) if gamma1 else None
        g2 = np.empty((L, L, L, L)) if gamma2 else None
        ptr = lambda a: _dptr(a) if a is not None else None
        self._check(self.lib.qcdmrg_energy_grad(self.h, ctypes.byref(e), ptr(d), ptr(g1), ptr(g2)))
        return e.value, d, g1, g2

    def checkpoint(self, path):
        self._check(self.lib.qcdmrg_checkpoint(self.h, os.fsencode(path)))

    def restore(self, path):
        self._check(self.lib.qcdmrg_restore(self.h, os.fsencode(path)))

    def rdm2(self, L):
        """Spin-summed 2-RDM, averaged over the 8-fold permutations of (pq|rs)
        (L^4/8 environment builds: small active spaces)."""
        g = np.empty((L, L, L, L))
        self._check(self.lib.qcdmrg_rdm2(self.h, _dptr(g)))
        return g

    def rdm2_sweep(self, L):
        """Spin-summed 2-RDM element by element (no permutation average), measured while the
        centre walks the chain once (O(L^4) small products; the MPS is restored afterwards)."""
        g = np.empty((L, L, L, L))
        self._check(self.lib.qcdmrg_rdm2_sweep(self.h, _dptr(g)))
        return g

    def orbital_rdm(self, L):
        """Two-orbital reduced density matrices, shape (L, L, 16, 16): [i, j] for i < j is
        rho_ij with row 4 x + y (x, y the states of orbitals i, j), zero for i >= j; one walk
        of the centre (the MPS is restored afterwards)."""
        r = np.empty((L, L, 16, 16))
        self._check(self.lib.qcdmrg_orbital_rdm(self.h, _dptr(r)))
        return r

    def heff_diag(self):
        out = np.empty(self.psi_size())
        self._check(self.lib.qcdmrg_heff_diag(self.h, _dptr(out), out.size))
        return out

    def truncate(self, D, direction):
        err = ctypes.c_double()
        self._check(self.lib.qcdmrg_truncate(self.h, D, direction, ctypes.byref(err)))
        return err.value

    def move_center(self, target):
        self._check(self.lib.qcdmrg_move_center(self.h, target))

    def sweep(self, D, allow_notconv=False, trunc_eps=0.0, D_min=1, **kw):
        """One sweep; trunc_eps > 0 selects the bond dimension of each truncation
        dynamically in [D_min, D]."""
        o = SweepOpts(D, self.dav_opts(**kw), trunc_eps, D_min)
        r = SweepReport()
        rc = self.lib.qcdmrg_sweep(self.h, ctypes.byref(o), ctypes.byref(r))
        if not (allow_notconv and rc == -5):
            self._check(rc)
        return {"energy": r.energy, "energy_mixed": r.energy_mixed, "max_trunc_err": r.max_trunc_err,
                "seconds": r.seconds, "n_hpsi": list(r.n_hpsi), "n_steps": r.n_steps, "max_D": r.max_D}

    def sweep_left(self, D, allow_notconv=False, trunc_eps=0.0, D_min=1, **kw):
        """Optimise and truncate from the current centre leftwards to sites (0, 1): the
        warm-up half sweep after import_configs."""
        o = SweepOpts(D, self.dav_opts(**kw), trunc_eps, D_min)
        r = SweepReport()
        rc = self.lib.qcdmrg_sweep_left(self.h, ctypes.byref(o), ctypes.byref(r))
        if not (allow_notconv and rc == -5):
            self._check(rc)
        return {"energy": r.energy, "energy_mixed": r.energy_mixed, "max_trunc_err": r.max_trunc_err,
                "seconds": r.seconds, "n_hpsi": list(r.n_hpsi), "n_steps": r.n_steps, "max_D": r.max_D}

    def import_configs(self, L, N, two_s, steps, coef, symmetry=None):
        """Import the MPS of sum_k coef[k] |config_k> (qcdmrg_config_mps), centre L-2."""
        sym = self.symmetry if symmetry is None else symmetry
        center, nsec, sec, data = config_mps(sym, L, N, two_s, steps, coef, lib=self.lib)
        self.import_mps(L, center, nsec, sec, data)
        return center

    def truncate_dbss(self, D_min, D_max, eps, direction):
        """Returns (discarded weight, states kept)."""
        err, kept = ctypes.c_double(), ctypes.c_int()
        self._check(self.lib.qcdmrg_truncate_dbss(self.h, D_min, D_max, eps, direction, ctypes.byref(err),
                                                  ctypes.byref(kept)))
        return err.value, kept.value

    def check_device(self):
        self._check(self.lib.qcdmrg_check_device(self.h))

    def stats(self):
        s = Stats()
        self._check(self.lib.qcdmrg_stats(self.h, ctypes.byref(s)))
        out = {f: getattr(s, f) for f, _ in Stats._fields_}
        return {f: (list(v) if isinstance(v, ctypes.Array) else v) for f, v in out.items()}


def extrapolate(x, energy, degree=1, lib=None):
    """qcdmrg_extrapolate: least-squares polynomial of the given degree through the
    points (x[i], energy[i]); returns its coefficients, the first being the value at
    x = 0."""
    import numpy as np
    lib = lib or load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    e = np.ascontiguousarray(energy, dtype=np.float64)
    if x.shape != e.shape:
        raise ValueError("x and energy differ in length")
    c = np.zeros(degree + 1)
    rc = lib.qcdmrg_extrapolate(_dptr(x), _dptr(e), len(x), degree, _dptr(c))
    if rc != 0:
        raise QcdmrgError(rc, "qcdmrg_extrapolate: invalid points")
    return c


def _f64(a):
    import numpy as np
    return np.ascontiguousarray(a, dtype=np.float64)


def active_space(h, V, ncore, nact, lib=None):
    """qcdmrg_active_space: (e_core, h_act, V_act) of the frozen-core active space."""
    import numpy as np
    lib = lib or load()
    h, V = _f64(h), _f64(V)
    n = h.shape[0]
    e = ctypes.c_double()
    ha, Va = np.zeros((nact, nact)), np.zeros((nact,) * 4)
    rc = lib.qcdmrg_active_space(n, ncore, nact, _dptr(h), _dptr(V), ctypes.byref(e), _dptr(ha), _dptr(Va))
    if rc != 0:
        raise QcdmrgError(rc, "qcdmrg_active_space: invalid arguments")
    return e.value, ha, Va


def orbital_gradient(h, V, ncore, nact, gamma1, gamma2, lib=None):
    """qcdmrg_orbital_gradient: dE/dkappa (n x n, antisymmetric)."""
    import numpy as np
    lib = lib or load()
    h, V, g1, g2 = _f64(h), _f64(V), _f64(gamma1), _f64(gamma2)
    n = h.shape[0]
    G = np.zeros((n, n))
    rc = lib.qcdmrg_orbital_gradient(n, ncore, nact, _dptr(h), _dptr(V), _dptr(g1), _dptr(g2), _dptr(G))
    if rc != 0:
        raise QcdmrgError(rc, "qcdmrg_orbital_gradient: invalid arguments")
    return G


def orbital_hessian_diag(h, V, ncore, nact, gamma1, gamma2, lib=None):
    """qcdmrg_orbital_hessian_diag: d^2E/dkappa_pq^2 (n x n, symmetric, zero diagonal)."""
    lib = lib or load()
    h, V, g1, g2 = _f64(h), _f64(V), _f64(gamma1), _f64(gamma2)
    n = h.shape[0]
    H = np.zeros((n, n))
    rc = lib.qcdmrg_orbital_hessian_diag(n, ncore, nact, _dptr(h), _dptr(V), _dptr(g1), _dptr(g2), _dptr(H))
    if rc != 0:
        raise QcdmrgError(rc, "qcdmrg_orbital_hessian_diag: invalid arguments")
    return H


def rotate_orbitals(kappa, h, V, lib=None):
    """qcdmrg_rotate_orbitals: (U = exp(kappa), h', V') for an antisymmetric kappa."""
    import numpy as np
    lib = lib or load()
    k, h, V = _f64(kappa), _f64(h), _f64(V)
    n = h.shape[0]
    U, h2, V2 = np.zeros((n, n)), np.zeros((n, n)), np.zeros((n,) * 4)
    rc = lib.qcdmrg_rotate_orbitals(n, _dptr(k), _dptr(h), _dptr(V), _dptr(U), _dptr(h2), _dptr(V2))
    if rc != 0:
        raise QcdmrgError(rc, "qcdmrg_rotate_orbitals: kappa must be antisymmetric")
    return U, h2, V2


def orbital_entanglement(rho, lib=None):
    """qcdmrg_orbital_entanglement: (s1, mutual) from the (L, L, 16, 16) blocks of
    Context.orbital_rdm."""
    import numpy as np
    lib = lib or load()
    r = _f64(rho)
    L = r.shape[0]
    if r.shape != (L, L, 16, 16):
        raise ValueError("rho must have shape (L, L, 16, 16)")
    s1, mi = np.zeros(L), np.zeros((L, L))
    rc = lib.qcdmrg_orbital_entanglement(L, _dptr(r), _dptr(s1), _dptr(mi))
    if rc != 0:
        raise QcdmrgError(rc, "qcdmrg_orbital_entanglement: invalid arguments")
    return s1, mi


def fiedler_order(mutual, lib=None):
    """qcdmrg_fiedler_order: (order, fiedler vector) of a symmetric mutual-information
    matrix; h[np.ix_(order, order)] is the reordered chain."""
    import numpy as np
    lib = lib or load()
    m = _f64(mutual)
    L = m.shape[0]
    order, f = np.zeros(L, dtype=np.int32), np.zeros(L)
    rc = lib.qcdmrg_fiedler_order(L, _dptr(m), order.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(f))
    if rc != 0:
        raise QcdmrgError(rc, "qcdmrg_fiedler_order: invalid arguments")
    return order.astype(np.int64), f


def select_configs(symmetry, h, V, N, two_s, nmax, lib=None):
    """qcdmrg_select_configs: (steps (count x L uint8), energies) of the nmax lowest
    configurations within two electrons of the aufbau reference."""
    lib = lib or load()
    h, V = _f64(h), _f64(V)
    L = h.shape[0]
    steps = np.zeros((nmax, L), dtype=np.uint8)
    en = np.zeros(nmax)
    cnt = ctypes.c_int()
    rc = lib.qcdmrg_select_configs(symmetry, L, N, two_s, _dptr(h), _dptr(V), nmax,
                                   steps.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _dptr(en),
                                   ctypes.byref(cnt))
    if rc != 0:
        raise QcdmrgError(rc, "qcdmrg_select_configs: invalid arguments")
    return steps[:cnt.value].copy(), en[:cnt.value].copy()


def config_mps(symmetry, L, N, two_s, steps, coef, lib=None):
    """qcdmrg_config_mps: (center, bond_nsec, bond_sec, data) of sum_k coef[k] |config_k>."""
    lib = lib or load()
    st = np.ascontiguousarray(steps, dtype=np.uint8).reshape(-1, L)
    c = _f64(coef).reshape(-1)
    if c.size != st.shape[0]:
        raise ValueError("one coefficient per configuration")
    u8 = st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    ip = ctypes.POINTER(ctypes.c_int)
    center, nsec_n, ndata = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
    nsec = np.zeros(L + 1, dtype=np.int32)
    rc = lib.qcdmrg_config_mps(symmetry, L, N, two_s, st.shape[0], u8, _dptr(c), ctypes.byref(center),
                               nsec.ctypes.data_as(ip), None, 0, None, 0, ctypes.byref(nsec_n), ctypes.byref(ndata))
    if rc != 0:
        raise QcdmrgError(rc, "qcdmrg_config_mps: invalid configurations")
    sec = np.zeros(max(3, 3 * nsec_n.value), dtype=np.int32)
    data = np.zeros(max(1, ndata.value))
    rc = lib.qcdmrg_config_mps(symmetry, L, N, two_s, st.shape[0], u8, _dptr(c), ctypes.byref(center),
                               nsec.ctypes.data_as(ip), sec.ctypes.data_as(ip), sec.size, _dptr(data), data.size,
                               ctypes.byref(nsec_n), ctypes.byref(ndata))
    if rc != 0:
        raise QcdmrgError(rc, "qcdmrg_config_mps: invalid configurations")
    return center.value, nsec, sec[:3 * nsec_n.value], data[:ndata.value]


def ordering_cost(mutual, order, eta=2.0, lib=None):
    """qcdmrg_ordering_cost: sum_{i<j} I_ij |pos_i - pos_j|^eta of a chain order."""
    lib = lib or load()
    m = _f64(mutual)
    o = np.ascontiguousarray(order, dtype=np.int32)
    c = ctypes.c_double()
    rc = lib.qcdmrg_ordering_cost(m.shape[0], _dptr(m), o.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), eta,
                                  ctypes.byref(c))
    if rc != 0:
        raise QcdmrgError(rc, "qcdmrg_ordering_cost: invalid arguments")
    return c.value


def refine_order(mutual, order, eta=2.0, max_swaps=10000, lib=None):
    """qcdmrg_refine_order: (improved order, exchanges made)."""
    lib = lib or load()
    m = _f64(mutual)
    o = np.array(order, dtype=np.int32)
    n = ctypes.c_int()
    rc = lib.qcdmrg_refine_order(m.shape[0], _dptr(m), eta, o.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 max_swaps, ctypes.byref(n))
    if rc != 0:
        raise QcdmrgError(rc, "qcdmrg_refine_order: invalid arguments")
    return o.astype(np.int64), n.value


def reorder_integrals(h, V, order):
    """Integrals of the chain in the given orbital order: h[o][o], V[o][o][o][o]."""
    import numpy as np
    o = np.asarray(order)
    return _f64(h)[np.ix_(o, o)], _f64(V)[np.ix_(o, o, o, o)]


class HeffGraph:
    """H_eff psi of one or several contexts captured in one CUDA graph."""

    def __init__(self, contexts, psi_ptrs, sigma_ptrs, precision=FP64):
        self.lib = contexts[0].lib
        n = len(contexts)
        P = ctypes.c_void_p
        ctxs = (P * n)(*[c.h.value for c in contexts])
        ps = (P * n)(*psi_ptrs)
        ss = (P * n)(*sigma_ptrs)
        self.h = P()
        rc = self.lib.qcdmrg_graph_create(ctxs, n, precision, ps, ss, ctypes.byref(self.h))
        if rc != QCDMRG_OK:
            raise QcdmrgError(rc, self.lib.qcdmrg_last_error(contexts[0].h).decode())
        self._ctx = contexts

    def launch(self, stream=0):
        rc = self.lib.qcdmrg_graph_launch(self.h, ctypes.c_void_p(stream))
        if rc != QCDMRG_OK:
            raise QcdmrgError(rc, "graph launch failed")

    def info(self):
        f, n = ctypes.c_double(), ctypes.c_int()
        self.lib.qcdmrg_graph_info(self.h, ctypes.byref(f), ctypes.byref(n))
        return f.value, n.value

    def close(self):
        if self.h:
            self.lib.qcdmrg_graph_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
