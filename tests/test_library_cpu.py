"""CPU checks of libzolo: it builds, loads, exports every symbol of include/zolo.h,
its host-side coefficient module agrees with the oracle and Table 1, and illegal
arguments are rejected before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import zolo_oracle as zo
from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "zolo.h")


@pytest.fixture(scope="module")
def zb():
    from paper_1806_06204_gb300 import build
    build.build()
    from paper_1806_06204_gb300 import binding
    return binding


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(zolo_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(zb):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(zb.LIB, name), name
    assert sorted(zb.EXPORTED) == names


def test_coefficients_match_oracle(zb):
    for ell in [1e-16, 1e-12, 1e-8, 1e-4, 1e-2, 0.1, 0.5, 0.9, 0.999, 1.0]:
        for r in range(1, 9):
            c, a, mh, gap = zb.coefficients(ell, r)
            co = zo.zolotarev_coeffs(ell, r)
            assert np.allclose(c, co.c, rtol=2e-14, atol=0), (ell, r)
            assert np.allclose(a, co.a, rtol=1e-12, atol=0), (ell, r)
            assert mh == pytest.approx(co.Mhat, rel=1e-14)
            assert gap == pytest.approx(zo.one_minus_zhat_at_ell(co), rel=1e-12, abs=1e-300)


def test_schedule_reproduces_table1(zb):
    from tests.test_oracle_coefficients import read_table1
    kappas, table = read_table1()
    for r, row in table.items():
        got = [len(zb.schedule(1.0 / k, r)[0]) - 1 for k in kappas]
        assert got == row, (r, got, row)


def test_schedule_r_choice_and_switch_match_oracle(zb):
    for kappa in [1.5, 10, 1e2, 1e4, 1e8, 1e12, 1e16]:
        ells, qr, r = zb.schedule(1.0 / kappa, 0)
        assert r == zo.choose_r(1.0 / kappa)
        oe = zo.ell_schedule(1.0 / kappa, r)
        assert np.allclose(ells, oe, rtol=1e-14, atol=1e-16)
        assert qr == [zo.uses_qr(zo.zolotarev_coeffs(e, r), e) for e in oe[:-1]]
    # a measured r belongs to a handle: the host-only schedule refuses it
    with pytest.raises(zb.ZoloError):
        zb.schedule(1e-8, zb.ZOLO_R_TUNED)


def test_illegal_arguments_rejected_before_device_work(zb):
    fake = ctypes.c_void_p(1)   # never dereferenced: validation fails first
    o = zb.opts(beta=1e-3)
    info = zb.ZoloInfo()
    P = ctypes.c_void_p(16)
    call = lambda *a: zb.LIB.zolo_pd(*a, ctypes.byref(info), None)
    assert zb.LIB.zolo_pd(None, P, 4, 4, 4, P, 4, P, 4, ctypes.byref(o), ctypes.byref(info), None) == -1
    assert call(fake, None, 4, 4, 4, P, 4, P, 4, ctypes.byref(o)) == -2
    assert call(fake, P, 3, 4, 4, P, 4, P, 4, ctypes.byref(o)) == -3
    assert call(fake, P, 4, 0, 4, P, 4, P, 4, ctypes.byref(o)) == -4
    assert call(fake, P, 4, 4, 3, P, 4, P, 4, ctypes.byref(o)) == -5
    assert call(fake, P, 4, 4, 4, P, 3, P, 4, ctypes.byref(o)) == -7
    assert call(fake, P, 4, 4, 4, P, 4, P, 3, ctypes.byref(o)) == -9
    # beta <= 0 asks for the device estimate, so it is legal; -inf is not finite
    for bad in [dict(beta=float("-inf")), dict(beta=1e-3, r=9), dict(beta=1e-3, r=-2), dict(beta=2.0, alpha=1.0),
                dict(beta=1e-3, max_iter=0), dict(beta=float("nan"))]:
        ob = zb.opts(**bad)
        assert call(fake, P, 4, 4, 4, P, 4, P, 4, ctypes.byref(ob)) == -10, bad
    assert zb.LIB.zolo_coefficients(0.0, 3, None, None, None, None) == -1
    assert zb.LIB.zolo_coefficients(0.5, 9, None, None, None, None) == -2


def test_workspace_bytes_query(zb):
    # host-only: the workspace a call keeps, from the same layout the call carves
    m, n = 3000, 1000
    f = lambda **k: zb.workspace_bytes(m, n, **k)
    b8 = f(r=8)
    # at least X, X_next, S (m x n), M (n x n) and, per shift, the stacked W
    # ((m + n) x n) and the reflectors V ((m + 128) x n)
    floor = 8 * (3 * m * n + n * n + 8 * ((m + n) * n + (m + 128) * n))
    assert floor <= b8 <= 1.25 * floor + (1 << 20)
    assert f(r=1) < f(r=4) < b8 == f(r=0) == f(r=zb.ZOLO_R_TUNED)
    assert f(r=8, svd=True) > b8
    assert f(r=8, prec=zb.ZOLO_SPLIT_BF16) > b8
    assert zb.workspace_bytes(16384, 16384, 8, zb.ZOLO_SPLIT_BF16) < 100e9
    import ctypes
    out = ctypes.c_uint64()
    call = zb.LIB.zolo_workspace_bytes
    assert call(10, 20, 1, 0, 0, ctypes.byref(out)) == -1       # m < n
    assert call(10, 0, 1, 0, 0, ctypes.byref(out)) == -2
    assert call(10, 10, 9, 0, 0, ctypes.byref(out)) == -3
    assert call(10, 10, -2, 0, 0, ctypes.byref(out)) == -3
    assert call(10, 10, 1, 5, 0, ctypes.byref(out)) == -4
    assert call(10, 10, 1, 0, 2, ctypes.byref(out)) == -5
    assert call(10, 10, 1, 0, 0, None) == -6


def test_debug_stall_rejects_bad_arguments_without_a_device(zb):
    assert zb.LIB.zolo_debug_stall(None, zb.ZOLO_STALL_SPLIT_GEMM, 1000) == -1


def test_library_coefficients_against_mpmath_directly(zb):
    """The library's coefficient module pinned to mpmath's elliptic functions at
    50 digits on its own, not only through the oracle: c_i (Eq. 7), a_j as the
    partial-fraction residues of Eq. (8) (Theorem 1), M_hat (Eq. 8) and the gap
    1 - Zhat(l; l)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    worst = {"c": 0.0, "a": 0.0, "M": 0.0, "gap": 0.0}
    for ell in [1e-16, 1e-12, 1e-8, 1e-4, 1e-2, 0.1, 0.5, 0.9, 0.999]:
        for r in (1, 2, 4, 6, 8):
            c, a, mh, gap = zb.coefficients(ell, r)
            L = mp.mpf(ell)
            m = 1 - L * L
            Kp = mp.ellipk(m)
            cr = [L * L * (mp.ellipfun("sn", i * Kp / (2 * r + 1), m=m) /
                           mp.ellipfun("cn", i * Kp / (2 * r + 1), m=m)) ** 2
                  for i in range(1, 2 * r + 1)]
            M = mp.mpf(1)
            for j in range(r):
                M *= (1 + cr[2 * j]) / (1 + cr[2 * j + 1])
            # residue of M x prod (x^2 + c_2k) / prod (x^2 + c_2k-1) at x^2 = -c_2j-1,
            # divided by M: a_j (Eq. 9)
            ar = []
            for j in range(r):
                num = mp.mpf(1)
                den = mp.mpf(1)
                for k in range(r):
                    num *= cr[2 * k + 1] - cr[2 * j]
                    if k != j:
                        den *= cr[2 * k] - cr[2 * j]
                ar.append(num / den)
            z = M * L
            for j in range(r):
                z *= (L * L + cr[2 * j + 1]) / (L * L + cr[2 * j])
            worst["c"] = max(worst["c"], max(float(abs((ci - x) / x)) for ci, x in zip(c, cr)))
            worst["a"] = max(worst["a"], max(float(abs((ai - x) / x)) for ai, x in zip(a, ar)))
            worst["M"] = max(worst["M"], float(abs((mh - M) / M)))
            g = 1 - z
            if g > mp.mpf(10) ** -30:
                worst["gap"] = max(worst["gap"], float(abs((gap - g) / g)))
    # measured: c 5.8e-15, a 9.6e-15, M 1.6e-15, gap 3.9e-15
    assert worst["c"] < 2e-14 and worst["M"] < 1e-14, worst
    assert worst["a"] < 5e-14 and worst["gap"] < 2e-14, worst
