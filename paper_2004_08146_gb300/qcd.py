"""Thin ctypes binding of libqcd (include/qcd.h): same names as the C ABI,
argument marshalling only.  Device buffers are passed as torch tensors (their
``data_ptr()``) or raw integers; every computation runs in libqcd.so.

Importing this module loads ``libqcd.so`` from this package directory and
raises ``ImportError`` when it is missing: there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqcd.so")

QCD_OK, QCD_EINVAL, QCD_ENOMEM, QCD_ENOTSETUP, QCD_ENOCONV, QCD_ETIMEOUT, QCD_ECUDA = range(7)
QCD_OP_D, QCD_OP_Q = 0, 1
QCD_FP64, QCD_FP32 = 0, 1
QCD_MIXED = 1
QCD_SMOOTHER_SAP, QCD_SMOOTHER_GMRES = 0, 1
QCD_EXTRACT_HARMONIC, QCD_EXTRACT_RITZ = 0, 1

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libqcd.so not built ({LIB_PATH}); run __graft_entry__.build()")
_lib = ctypes.CDLL(LIB_PATH)


class qcd_params(ctypes.Structure):
    _fields_ = [
        ("antiperiodic_t", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("correction_form", ctypes.c_int),
        ("use_mg", ctypes.c_int),
        ("setup_iters", ctypes.c_int),
        ("smoother", ctypes.c_int),
        ("nu", ctypes.c_int),
        ("sap_block", ctypes.c_int * 4),
        ("sap_block_iters", ctypes.c_int),
        ("sap_block_tol", ctypes.c_double),
        ("gmres_smooth_iters", ctypes.c_int),
        ("inner_tol", ctypes.c_double),
        ("inner_maxiter", ctypes.c_int),
        ("coarse_tol", ctypes.c_double),
        ("coarse_maxiter", ctypes.c_int),
        ("plain_maxiter", ctypes.c_int),
        ("m_min", ctypes.c_int),
        ("m_max", ctypes.c_int),
        ("block", ctypes.c_int),
        ("n_init", ctypes.c_int),
        ("shift_rho", ctypes.c_int),
        ("update_every", ctypes.c_int),
        ("extraction", ctypes.c_int),
        ("max_outer", ctypes.c_int),
        ("seed", ctypes.c_ulonglong),
        ("verbose", ctypes.c_int),
        ("levels", ctypes.c_int),
        ("nv2", ctypes.c_int),
        ("agg2", ctypes.c_int * 4),
        ("nu2", ctypes.c_int),
        ("coarse_layout", ctypes.c_int),
        ("coarse_tensor", ctypes.c_int),
        ("sap_half", ctypes.c_int),
        ("confirm", ctypes.c_int),
        ("coarse_ctas", ctypes.c_int),
        ("guard", ctypes.c_int),
    ]


class qcd_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("refinements", ctypes.c_int),
                ("residual", ctypes.c_double), ("seconds", ctypes.c_double)]


class qcd_eig_info(ctypes.Structure):
    _fields_ = [("outer", ctypes.c_int), ("inner", ctypes.c_int), ("locked", ctypes.c_int),
                ("updates", ctypes.c_int), ("converged", ctypes.c_int),
                ("max_residual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("coarse_solves", ctypes.c_longlong), ("coarse_iterations", ctypes.c_longlong)]


class qcd_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_longlong), ("timed", ctypes.c_longlong),
                ("total_ms", ctypes.c_double), ("bytes", ctypes.c_double), ("flops", ctypes.c_double),
                ("timed_bytes", ctypes.c_double), ("timed_flops", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "qcd_default_params": (None, [ctypes.POINTER(qcd_params)]),
    "qcd_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(qcd_params), _P]),
    "qcd_destroy": (_I, [_P]),
    "qcd_last_error": (ctypes.c_char_p, [_P]),
    "qcd_set_params": (_I, [_P, ctypes.POINTER(qcd_params)]),
    "qcd_set_gauge": (_I, [_P, _DP, _IP, _D, _D]),
    "qcd_apply_Q": (_I, [_P, _P, _P, _D]),
    "qcd_apply": (_I, [_P, _I, _I, _I, _P, _P, _DP]),
    "qcd_mg_setup": (_I, [_P, _I, _IP]),
    "qcd_mg_update_from_eigvecs": (_I, [_P, _P, _I]),
    "qcd_shifted_solve": (_I, [_P, _P, _P, _D, _D, ctypes.POINTER(qcd_solve_info)]),
    "qcd_shifted_solve_batched": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _DP, _D,
                                       ctypes.POINTER(qcd_solve_info)]),
    "qcd_eigs": (_I, [_P, _I, _D, _DP, _P, ctypes.POINTER(qcd_eig_info)]),
    "qcd_mg_info": (_I, [_P, _IP]),
    "qcd_mg_restrict": (_I, [_P, _I, _I, _P, _P]),
    "qcd_mg_prolong": (_I, [_P, _I, _I, _P, _P]),
    "qcd_local_coherence": (_I, [_P, _I, _P, _DP]),
    "qcd_eig_derivative": (_I, [_P, _DP, _I, _P, _DP]),
    "qcd_eig_force": (_I, [_P, _I, _P, _P]),
    "qcd_bilinear_force": (_I, [_P, _I, _P, _P, _I, _P]),
    "qcd_coarse_apply": (_I, [_P, _I, _I, _I, _P, _P, _DP]),
    "qcd_mg_get_P": (_I, [_P, _DP]),
    "qcd_mg_get_coarse": (_I, [_P, _DP]),
    "qcd_mg_info2": (_I, [_P, ctypes.POINTER(ctypes.c_int)]),
    "qcd_mg_get_P2": (_I, [_P, _DP]),
    "qcd_mg_get_coarse2": (_I, [_P, _DP]),
    "qcd_projected_eig": (_I, [_P, _I, _DP, _DP, _I, _DP, _DP]),
    "qcd_sap": (_I, [_P, _I, _I, _I, _P, _P, _DP, _I, _D]),
    "qcd_mg_cycle": (_I, [_P, _I, _I, _I, _P, _P, _DP]),
    "qcd_sap_static": (_I, [_P, _I, _I, _I, _P, _P, _DP, _I, _D]),
    "qcd_stats_reset": (_I, [_I, ctypes.c_char_p]),
    "qcd_stats_read": (_I, [ctypes.POINTER(qcd_kernel_stat), _I, _IP]),
    "qcd_stats_sap_work": (_I, [_DP, _DP]),
    "qcd_stats_wait_timeouts": (_I, [ctypes.POINTER(ctypes.c_ulonglong)]),
    "qcd_selftest_wait_limit": (_I, [_P]),
    "qcd_fma_peak": (_I, [_I, _DP]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


class QcdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libqcd error {code}: {msg}")
        self.code = code


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    return ctypes.c_void_p(x.data_ptr())


def _dbl(arr):
    a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64))
    return a, a.ctypes.data_as(_DP)


def qcd_stats_reset(mode=0, kernel=None):
    """Launch accounting: mode 0 counts, 1 times every launch, 2 times `kernel`."""
    rc = _lib.qcd_stats_reset(int(mode), kernel.encode() if kernel else None)
    if rc != QCD_OK:
        raise QcdError(rc, "qcd_stats_reset")


def qcd_stats_read():
    n = ctypes.c_int(0)
    _lib.qcd_stats_read(None, 0, ctypes.byref(n))
    arr = (qcd_kernel_stat * max(1, n.value))()
    _lib.qcd_stats_read(arr, n.value, ctypes.byref(n))
    return [dict(name=a.name.decode(), launches=a.launches, timed=a.timed, total_ms=a.total_ms, bytes=a.bytes,
                 flops=a.flops, timed_bytes=a.timed_bytes, timed_flops=a.timed_flops) for a in arr[:n.value]]


def qcd_stats_sap_work():
    """(sum block sites x steps, sum block sites x k(k+1)/2) of the SAP block solves."""
    a, b = ctypes.c_double(0), ctypes.c_double(0)
    rc = _lib.qcd_stats_sap_work(ctypes.byref(a), ctypes.byref(b))
    if rc != QCD_OK:
        raise QcdError(rc, "qcd_stats_sap_work")
    return a.value, b.value


def qcd_stats_wait_timeouts():
    """Bounded device-side waits that gave up since the library was loaded (0 in a correct run)."""
    n = ctypes.c_ulonglong(0)
    rc = _lib.qcd_stats_wait_timeouts(ctypes.byref(n))
    if rc != QCD_OK:
        raise QcdError(rc, "qcd_stats_wait_timeouts")
    return n.value


def qcd_fma_peak(prec):
    """Measured FMA throughput (TFLOP/s) of the current device for QCD_FP32 / QCD_FP64."""
    t = ctypes.c_double(0)
    rc = _lib.qcd_fma_peak(int(prec), ctypes.byref(t))
    if rc != QCD_OK:
        raise QcdError(rc, "qcd_fma_peak")
    return t.value


def default_params(**kw):
    p = qcd_params()
    _lib.qcd_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k in ("sap_block", "agg2"):
            setattr(p, k, (ctypes.c_int * 4)(*v))
        else:
            setattr(p, k, v)
    return p


class Context:
    """One libqcd context (qcd_create / qcd_destroy) on a CUDA stream."""

    def __init__(self, params=None, stream=0, **kw):
        self.params = params if params is not None else default_params(**kw)
        self.h = _P()
        rc = _lib.qcd_create(ctypes.byref(self.h), ctypes.byref(self.params), _P(stream))
        if rc != QCD_OK:
            raise QcdError(rc, "qcd_create failed")

    def _check(self, rc, allow=(QCD_OK,)):
        if rc not in allow:
            raise QcdError(rc, _lib.qcd_last_error(self.h).decode())
        return rc

    def close(self):
        if self.h:
            _lib.qcd_destroy(self.h)
            self.h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- C-ABI mirrors
    def qcd_set_params(self, params):
        self.params = params
        return self._check(_lib.qcd_set_params(self.h, ctypes.byref(params)))

    def qcd_set_gauge(self, U, dims, m0, csw):
        Uh = np.ascontiguousarray(np.asarray(U, dtype=np.complex128)).view(np.float64)
        d = (ctypes.c_int * 4)(*[int(x) for x in dims])
        self.dims = tuple(int(x) for x in dims)
        self._U_keep = Uh
        return self._check(_lib.qcd_set_gauge(self.h, Uh.ctypes.data_as(_DP), d, float(m0), float(csw)))

    def qcd_apply_Q(self, inp, out, tau=0.0):
        return self._check(_lib.qcd_apply_Q(self.h, _ptr(inp), _ptr(out), float(tau)))

    def qcd_apply(self, op, prec, nrhs, inp, out, tau):
        t, tp = _dbl(tau)
        return self._check(_lib.qcd_apply(self.h, op, prec, nrhs, _ptr(inp), _ptr(out), tp))

    def qcd_mg_setup(self, Nv, block):
        b = (ctypes.c_int * 4)(*[int(x) for x in block])
        return self._check(_lib.qcd_mg_setup(self.h, int(Nv), b))

    def qcd_mg_update_from_eigvecs(self, V, nvec):
        return self._check(_lib.qcd_mg_update_from_eigvecs(self.h, _ptr(V), int(nvec)))

    def qcd_shifted_solve(self, b, x, tau, tol):
        info = qcd_solve_info()
        rc = _lib.qcd_shifted_solve(self.h, _ptr(b), _ptr(x), float(tau), float(tol), ctypes.byref(info))
        self._check(rc, (QCD_OK, QCD_ENOCONV))
        return rc, info

    def qcd_shifted_solve_batched(self, bs, xs, taus, tol):
        n = len(bs)
        barr = (_P * n)(*[_ptr(b).value for b in bs])
        xarr = (_P * n)(*[_ptr(x).value for x in xs])
        t, tp = _dbl(taus)
        info = qcd_solve_info()
        rc = _lib.qcd_shifted_solve_batched(self.h, n, barr, xarr, tp, float(tol), ctypes.byref(info))
        self._check(rc, (QCD_OK, QCD_ENOCONV))
        return rc, info

    def qcd_eigs(self, k, tol, V=None):
        lam = np.zeros(int(k), dtype=np.float64)
        info = qcd_eig_info()
        rc = _lib.qcd_eigs(self.h, int(k), float(tol), lam.ctypes.data_as(_DP), _ptr(V), ctypes.byref(info))
        self._check(rc, (QCD_OK, QCD_ENOCONV))
        return rc, lam, info

    def qcd_mg_info(self):
        out = (ctypes.c_int * 8)()
        self._check(_lib.qcd_mg_info(self.h, out))
        return dict(coarse_sites=out[0], nv=out[1], cdims=tuple(out[2:6]), block_sites=out[6])

    def qcd_mg_restrict(self, prec, nrhs, r, xc):
        return self._check(_lib.qcd_mg_restrict(self.h, prec, nrhs, _ptr(r), _ptr(xc)))

    def qcd_eig_derivative(self, X, nvec, V):
        Xh = np.ascontiguousarray(np.asarray(X, dtype=np.complex128)).view(np.float64)
        out = np.zeros(int(nvec), dtype=np.float64)
        self._check(_lib.qcd_eig_derivative(self.h, Xh.ctypes.data_as(_DP), int(nvec), _ptr(V),
                                            out.ctypes.data_as(_DP)))
        return out

    def qcd_eig_force(self, nvec, V, F):
        return self._check(_lib.qcd_eig_force(self.h, int(nvec), _ptr(V), _ptr(F)))

    def qcd_bilinear_force(self, nvec, G, Psi, grad, F):
        return self._check(_lib.qcd_bilinear_force(self.h, int(nvec), _ptr(G), _ptr(Psi), int(grad), _ptr(F)))

    def qcd_local_coherence(self, nvec, V):
        out = np.zeros(int(nvec), dtype=np.float64)
        self._check(_lib.qcd_local_coherence(self.h, int(nvec), _ptr(V), out.ctypes.data_as(_DP)))
        return out

    def qcd_mg_prolong(self, prec, nrhs, xc, x):
        return self._check(_lib.qcd_mg_prolong(self.h, prec, nrhs, _ptr(xc), _ptr(x)))

    def qcd_selftest_wait_limit(self):
        """Raw status of the bounded-wait self-test (QCD_ETIMEOUT expected)."""
        return _lib.qcd_selftest_wait_limit(self.h)

    def qcd_coarse_apply(self, op, prec, nrhs, x, y, tau):
        t, tp = _dbl(tau)
        return self._check(_lib.qcd_coarse_apply(self.h, op, prec, nrhs, _ptr(x), _ptr(y), tp))

    def qcd_mg_get_P(self):
        info = self.qcd_mg_info()
        n = info["coarse_sites"] * 2 * info["nv"] * info["block_sites"] * 6
        out = np.zeros(n, dtype=np.complex128)
        self._check(_lib.qcd_mg_get_P(self.h, out.view(np.float64).ctypes.data_as(_DP)))
        return out

    def qcd_mg_get_coarse(self):
        info = self.qcd_mg_info()
        nc = 2 * info["nv"]
        out = np.zeros(info["coarse_sites"] * 9 * nc * nc, dtype=np.complex128)
        self._check(_lib.qcd_mg_get_coarse(self.h, out.view(np.float64).ctypes.data_as(_DP)))
        return out.reshape(info["coarse_sites"], 9, nc, nc)

    def qcd_mg_info2(self):
        out = (ctypes.c_int * 8)()
        self._check(_lib.qcd_mg_info2(self.h, out))
        return dict(sites=out[0], nv2=out[1], dims=tuple(out[2:6]), aggregate_sites=out[6], nv1=out[7])

    def qcd_mg_get_P2(self):
        i = self.qcd_mg_info2()
        out = np.zeros(i["sites"] * 2 * i["nv2"] * i["aggregate_sites"] * i["nv1"], dtype=np.complex128)
        self._check(_lib.qcd_mg_get_P2(self.h, out.view(np.float64).ctypes.data_as(_DP)))
        return out.reshape(i["sites"], 2, i["nv2"], i["aggregate_sites"], i["nv1"])

    def qcd_mg_get_coarse2(self):
        i = self.qcd_mg_info2()
        nc = 2 * i["nv2"]
        out = np.zeros(i["sites"] * 9 * nc * nc, dtype=np.complex128)
        self._check(_lib.qcd_mg_get_coarse2(self.h, out.view(np.float64).ctypes.data_as(_DP)))
        return out.reshape(i["sites"], 9, nc, nc)

    def qcd_projected_eig(self, G, H, extraction=QCD_EXTRACT_HARMONIC):
        """(theta, S) of the projected eigenproblem (G, H: m x m complex matrices)."""
        H = np.asfortranarray(np.asarray(H, dtype=np.complex128))
        m = H.shape[0]
        Gf = None if G is None else np.asfortranarray(np.asarray(G, dtype=np.complex128))
        theta = np.zeros(m, dtype=np.float64)
        Gflat = None if Gf is None else np.ascontiguousarray(Gf.reshape(-1, order='F'))
        gp = None if Gflat is None else Gflat.view(np.float64).ctypes.data_as(_DP)
        Hflat = np.ascontiguousarray(H.reshape(-1, order='F'))
        Sflat = np.zeros(m * m, dtype=np.complex128)
        self._check(_lib.qcd_projected_eig(self.h, m, gp, Hflat.view(np.float64).ctypes.data_as(_DP), int(extraction),
                                           theta.ctypes.data_as(_DP), Sflat.view(np.float64).ctypes.data_as(_DP)))
        return theta, Sflat.reshape(m, m, order='F')

    def qcd_sap(self, op, prec, nrhs, b, x, tau, sweeps, block_tol):
        t, tp = _dbl(tau)
        return self._check(_lib.qcd_sap(self.h, op, prec, nrhs, _ptr(b), _ptr(x), tp, int(sweeps), float(block_tol)))

    def qcd_sap_static(self, op, prec, nrhs, b, x, tau, sweeps, block_tol):
        t, tp = _dbl(tau)
        return self._check(_lib.qcd_sap_static(self.h, op, prec, nrhs, _ptr(b), _ptr(x), tp, int(sweeps),
                                               float(block_tol)))

    def qcd_mg_cycle(self, op, prec, nrhs, b, x, tau):
        t, tp = _dbl(tau)
        return self._check(_lib.qcd_mg_cycle(self.h, op, prec, nrhs, _ptr(b), _ptr(x), tp))
