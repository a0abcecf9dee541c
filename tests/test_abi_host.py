"""The C ABI without a GPU: the library loads, exports every symbol that
include/sfac.h declares, rejects bad arguments on the host, and its host-only
FP64 precompute agrees with the oracle's dense matrices."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2209_08437_gb300 as S
from oracle import sfac_oracle as O
from tests.conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    return S.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sfac.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sfac_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert {"sfac_plan_create", "sfac_plan_destroy", "sfac_step", "sfac_solve",
            "sfac_last_error"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_params_struct_layout():
    assert ctypes.sizeof(S.SfacParams) == 80
    assert S.SfacParams.alpha.offset == 16 and S.SfacParams.prec.offset == 72


def test_version(lib):
    assert S.sfac_version() >= 100


@pytest.mark.parametrize("kw,status", [
    (dict(n=(64, 64), alpha=(1.0, 1.5), eps=0.1, tau=0.01), S.sfac.SFAC_EINVAL),
    (dict(n=(64, 64), alpha=(1.5, 2.0), eps=0.1, tau=0.01), S.sfac.SFAC_EINVAL),
    (dict(n=(64, 64), alpha=(1.5, 1.5), eps=0.0, tau=0.01), S.sfac.SFAC_EINVAL),
    (dict(n=(64, 64), alpha=(1.5, 1.5), eps=0.1, tau=-1.0), S.sfac.SFAC_EINVAL),
    (dict(n=(64, 64), alpha=(1.5, 1.5), eps=0.1, tau=0.01, a=1.0, b=1.0), S.sfac.SFAC_EINVAL),
    (dict(n=(64, 0), alpha=(1.5, 1.5), eps=0.1, tau=0.01), S.sfac.SFAC_EINVAL),
    (dict(n=(3000, 64), alpha=(1.5, 1.5), eps=0.1, tau=0.01), S.sfac.SFAC_EUNSUPPORTED),
    (dict(n=(1, 64), alpha=(1.5, 1.5), eps=0.1, tau=0.01), S.sfac.SFAC_EUNSUPPORTED),
    (dict(n=(8192, 64), alpha=(1.5, 1.5), eps=0.1, tau=0.01), S.sfac.SFAC_EUNSUPPORTED),
])
def test_plan_create_rejects_on_host(lib, kw, status):
    """These fail in the host-side checks, before any CUDA call."""
    p = S.make_params(**kw)
    out = ctypes.c_void_p(123)
    st = lib.sfac_plan_create(ctypes.byref(p), None, ctypes.byref(out))
    assert st == status
    assert out.value is None
    assert S.sfac_last_error() != ""


def test_null_arguments(lib):
    assert lib.sfac_plan_create(None, None, None) == S.sfac.SFAC_EINVAL
    assert lib.sfac_step(None, None, 1, None) == S.sfac.SFAC_EINVAL
    assert lib.sfac_solve(None, None, 1.0, None) == S.sfac.SFAC_EINVAL
    assert lib.sfac_step_host(None, None, 1, None) == S.sfac.SFAC_EINVAL
    assert lib.sfac_plan_destroy(None) == S.sfac.SFAC_OK
    p = S.make_params((8, 8), (1.5, 1.5), 0.1, 0.01)
    assert lib.sfac_plan_tables(ctypes.byref(p), 2, None, None, None, None) == S.sfac.SFAC_EINVAL
    p.reserved = 1
    assert lib.sfac_plan_tables(ctypes.byref(p), 0, None, None, None, None) == S.sfac.SFAC_EINVAL


def test_host_checks_of_the_newer_entry_points(lib):
    """Argument errors of the probe, the server's wait-limit hook and the
    server round are caught on the host, before any CUDA call."""
    vp = ctypes.c_void_p
    assert lib.sfac_probe_fma(3, 1, 1, vp(16), None) == S.sfac.SFAC_EINVAL
    assert lib.sfac_probe_fma(0, 0, 1, vp(16), None) == S.sfac.SFAC_EINVAL
    assert lib.sfac_probe_fma(1, 1, 0, vp(16), None) == S.sfac.SFAC_EINVAL
    assert lib.sfac_probe_fma(2, 1, 1, None, None) == S.sfac.SFAC_EINVAL
    assert lib.sfac_probe_jq(7, vp(16), vp(16), 4, 0.9, 0.1, None) == S.sfac.SFAC_EINVAL
    assert lib.sfac_probe_jq(S.SFAC_FP64, vp(16), vp(16), -1, 0.9, 0.1, None) == S.sfac.SFAC_EINVAL
    assert lib.sfac_probe_jq(S.SFAC_FP64, None, vp(16), 4, 0.9, 0.1, None) == S.sfac.SFAC_EINVAL
    assert lib.sfac_probe_jq(S.SFAC_FP32, vp(16), vp(16), 4, 0.0, 1.0, None) == S.sfac.SFAC_EINVAL
    assert lib.sfac_probe_jq(S.SFAC_FP32, vp(16), vp(16), 4, 1.5, -0.5, None) == S.sfac.SFAC_EINVAL
    assert lib.sfac_probe_jq(S.SFAC_FP64, None, None, 0, 0.9, 0.1, None) == S.sfac.SFAC_OK
    route = ctypes.c_int(9)
    assert lib.sfac_plan_host_route(None, vp(16), 1, ctypes.byref(route)) == S.sfac.SFAC_EINVAL
    assert route.value == 9
    assert lib.sfac_server_set_wait_limit(None, 10, -1) == S.sfac.SFAC_EINVAL
    launched = ctypes.c_int(7)
    assert lib.sfac_server_round(None, 4, 0, None, ctypes.byref(launched)) == S.sfac.SFAC_EINVAL
    assert launched.value == 0
    n = ctypes.c_int(5)
    assert lib.sfac_server_wait(None, None, None, 0, ctypes.byref(n)) == S.sfac.SFAC_EINVAL


@pytest.mark.parametrize("n,alpha,eps,tau", [(8, 1.3, 0.1, 0.01), (64, 1.7, 0.05, 1e-3),
                                             (63, 1.5, 0.1, 0.02), (256, 1.2, 0.08, 2e-3),
                                             (1024, 1.3, 0.05, 1e-3)])
def test_host_precompute_matches_oracle(n, alpha, eps, tau):
    """The library's FP64 tables (computed without a GPU) against the oracle:
    b_k against the dense B, and the spectra of Remark 1 against a dense
    symmetric eigensolve of the oracle's C and S."""
    p = S.make_params((n,), (alpha,), eps, tau)
    lam, mu, bcol, jq = S.sfac_plan_tables(p, 0)
    h = 2.0 / (n + 1)
    B = O.matrix_B(alpha, eps, h, n)
    np.testing.assert_allclose(bcol, B[:, 0], rtol=1e-13, atol=1e-13 * abs(B[0, 0]))
    C, Sm = O.split_CS(B)
    scale = abs(B[0, 0])
    np.testing.assert_allclose(np.sort(lam), np.linalg.eigvalsh(C), rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(np.sort(mu), np.linalg.eigvalsh(Sm), rtol=0, atol=1e-13 * scale)
    # ordering: lambda_j pairs with the DFT frequency j, mu_j with the twisted one
    np.testing.assert_allclose(lam, O.circulant_eigenvalues(C[:, 0]).real, atol=1e-13 * scale)
    np.testing.assert_allclose(mu, O.skew_circulant_eigenvalues(Sm[:, 0]).real, atol=1e-13 * scale)
    np.testing.assert_allclose(jq, [np.exp(-tau), -np.expm1(-tau), np.exp(-2 * tau),
                                    -np.expm1(-2 * tau)], rtol=1e-14)
