"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/qcd.h declares (no GPU needed, no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qcd.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qcd_[A-Za-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2004_08146_gb300 import build
    path = build.LIB
    if not os.path.exists(path):
        build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("qcd_set_gauge", "qcd_apply_Q", "qcd_mg_setup", "qcd_mg_update_from_eigvecs",
                     "qcd_shifted_solve", "qcd_eigs", "qcd_shifted_solve_batched", "qcd_last_error",
                     "qcd_create", "qcd_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2004_08146_gb300 import qcd
    assert set(_declared()) == set(qcd.EXPORTED)


def test_default_params_are_table_2():
    from paper_2004_08146_gb300 import qcd
    p = qcd.default_params()
    assert (p.setup_iters, p.nu, p.inner_maxiter, p.m_min, p.m_max) == (6, 4, 5, 30, 50)
    assert p.inner_tol == 0.1 and p.coarse_tol == 0.5
    assert p.sap_block_iters == 10 and p.sap_block_tol == 0.1


def test_create_rejects_bad_params():
    from paper_2004_08146_gb300 import qcd
    p = qcd.default_params(m_min=40, m_max=30)
    with pytest.raises(qcd.QcdError):
        qcd.Context(params=p)


def test_calls_without_gauge_fail_cleanly():
    """Argument and state errors come back as status codes, not crashes
    (no device work is issued before the checks)."""
    from paper_2004_08146_gb300 import qcd
    ctx = qcd.Context()
    with pytest.raises(qcd.QcdError) as e:
        ctx.qcd_apply_Q(0, 0, 0.0)
    assert e.value.code == qcd.QCD_ENOTSETUP
    with pytest.raises(qcd.QcdError) as e:
        ctx.qcd_mg_setup(0, (2, 2, 2, 2))
    assert e.value.code == qcd.QCD_EINVAL
    for call in (lambda: ctx.qcd_eig_force(1, 0, 0), lambda: ctx.qcd_local_coherence(1, 0),
                 ctx.qcd_mg_info2, ctx.qcd_mg_get_P2, ctx.qcd_mg_get_coarse2):
        with pytest.raises(qcd.QcdError) as e:
            call()
        assert e.value.code in (qcd.QCD_ENOTSETUP, qcd.QCD_EINVAL)
    ctx.close()


@pytest.mark.parametrize("bad", [dict(extraction=2), dict(update_every=-1), dict(block=0), dict(block=33),
                                 dict(m_max=106, block=8), dict(m_max=112), dict(sap_block_iters=0), dict(sap_block_iters=33),
                                 dict(levels=4), dict(levels=1), dict(nv2=0), dict(nv2=33),
                                 dict(agg2=(2, 0, 2, 2)), dict(nu2=-1), dict(coarse_layout=4),
                                 dict(coarse_layout=-1), dict(coarse_tensor=2), dict(sap_half=-1),
                                 dict(confirm=-1), dict(confirm=1025), dict(coarse_ctas=-1), dict(guard=-1)])
def test_create_rejects_each_bad_field(bad):
    """Parameter validation happens in qcd_create, on the host, before any GPU work."""
    from paper_2004_08146_gb300 import qcd
    with pytest.raises(qcd.QcdError) as e:
        qcd.Context(params=qcd.default_params(**bad))
    assert e.value.code == qcd.QCD_EINVAL


def test_basis_cap_accepts_the_large_workloads():
    """m_max 50 (Table 2) with 16 or 32 targets per iteration fits the basis
    cap of 112 (m_max + block <= 112)."""
    from paper_2004_08146_gb300 import qcd
    for block in (16, 32):
        qcd.Context(params=qcd.default_params(m_max=50, block=block)).close()
    qcd.Context(params=qcd.default_params(m_max=80, block=32)).close()


def test_default_params_method_variants():
    """Defaults: harmonic Ritz extraction, interpolation update after every lock
    (Algorithm 2), Rayleigh-quotient shift, two targets per outer iteration."""
    from paper_2004_08146_gb300 import qcd
    p = qcd.default_params()
    assert p.extraction == qcd.QCD_EXTRACT_HARMONIC and p.update_every == 1
    assert p.shift_rho == 1 and p.block == 2
    assert p.levels == 2 and p.nv2 == 8 and tuple(p.agg2) == (2, 2, 2, 2) and p.nu2 == 2


@pytest.mark.parametrize("dims,m0,csw", [((1, 4, 4, 4), -0.2, 1.0), ((4, 4, 4, 5000), -0.2, 1.0),
                                         ((4, 4, 4, 4), float("nan"), 1.0), ((4, 4, 4, 4), -0.2, float("inf"))])
def test_set_gauge_rejects_bad_lattice_and_couplings(dims, m0, csw):
    """Extents outside [2, 4096] and non-finite m0 or c_sw come back as EINVAL
    before any device work (the gauge array is only a placeholder)."""
    import numpy as np
    from paper_2004_08146_gb300 import qcd
    ctx = qcd.Context()
    U = np.zeros((2, 4, 3, 3), dtype=np.complex128)
    with pytest.raises(qcd.QcdError) as e:
        ctx.qcd_set_gauge(U, dims, m0, csw)
    assert e.value.code == qcd.QCD_EINVAL
    ctx.close()
