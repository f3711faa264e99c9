"""Pins for the oracle's Zolotarev coefficients and l-schedule (Eqs. 7-10, Table 1).

Each pin comes from something other than the oracle's own formulas: the numbers
the paper prints (Table 1), an independent closed form (the r = 1 case is the
QDWH step of Nakatsukasa, Bai and Gygi), a high-precision library evaluation of
the elliptic functions (mpmath), and properties the Zolotarev function must have
(Theorem 1's identity, equioscillation, ordering of the coefficients).
"""
import math
import os

import numpy as np
import pytest

from oracle import zolo_oracle as zo
from tests.conftest import GOLDEN

ELLS = [1e-16, 1e-12, 1e-8, 1e-5, 1e-3, 0.01, 0.1, 0.3, 0.5, 0.8, 0.95, 0.999]


def read_table1():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "table1_iterations.txt"))
            if ln.strip() and not ln.startswith("#")]
    kappas = [float(x) for x in rows[0][1:]]
    table = {int(r[0][1:]): [int(x) for x in r[1:]] for r in rows[1:]}
    return kappas, table


def test_table1_reproduced_all_96_cells():
    kappas, table = read_table1()
    assert len(kappas) == 12 and sorted(table) == list(range(1, 9))
    got = {r: [zo.iterations_needed(k, r) for k in kappas] for r in table}
    bad = [(r, kappas[i], got[r][i], table[r][i]) for r in table for i in range(12)
           if got[r][i] != table[r][i]]
    assert not bad, f"cells differing from Table 1 (r, kappa, oracle, paper): {bad}"


def test_r1_equals_dwh_closed_form():
    # Zhat_3(x) = M x (x^2 + c2)/(x^2 + c1) against x (a + b x^2)/(1 + c x^2):
    # c1 = 1/c, c2 = a/b, M = b/c.
    for ell in [1e-12, 1e-8, 1e-4, 1e-2, 0.1, 0.5, 0.9]:
        a, b, c = zo.dwh_closed_form(ell)
        co = zo.zolotarev_coeffs(ell, 1)
        assert co.c[0] == pytest.approx(1.0 / c, rel=1e-11)
        assert co.c[1] == pytest.approx(a / b, rel=1e-11)
        assert co.Mhat == pytest.approx(b / c, rel=1e-11)


def test_coefficients_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    worst = 0.0
    for ell in ELLS:
        for r in (1, 2, 3, 5, 8):
            co = zo.zolotarev_coeffs(ell, r)
            L = mp.mpf(ell)
            m = 1 - L * L                       # parameter m = l'^2 (modulus l')
            Kp = mp.ellipk(m)
            assert float(Kp) == pytest.approx(zo.K_complement(ell), rel=1e-14)
            for i in range(1, 2 * r + 1):
                u = i * Kp / (2 * r + 1)
                ref = L * L * (mp.ellipfun("sn", u, m=m) / mp.ellipfun("cn", u, m=m)) ** 2
                worst = max(worst, float(abs((co.c[i - 1] - ref) / ref)))
    assert worst < 5e-14, worst


def test_theorem1_partial_fraction_identity():
    # Eq. (8) (product form) equals Eq. (9) (partial fractions) with a_j of Eq. (10).
    for ell in ELLS:
        for r in range(1, 9):
            co = zo.zolotarev_coeffs(ell, r)
            x = np.geomspace(ell, 1.0, 400)
            p, q = zo.zhat(x, co), zo.zhat_partial_fraction(x, co)
            assert np.max(np.abs(p - q) / np.abs(p)) < 1e-12, (ell, r)


def test_coefficient_signs_and_ordering():
    for ell in ELLS:
        for r in range(1, 9):
            co = zo.zolotarev_coeffs(ell, r)
            assert np.all(co.c > 0) and np.all(np.diff(co.c) > 0)
            assert np.all(co.a > 0) and co.Mhat > 0


def test_equioscillation_on_interval():
    # Zhat maps [l, 1] into [Zhat(l), 1], touching 1 at r interior points and at
    # x = 1, and Zhat(l) at r interior points and at x = l: 2r + 2 alternation points.
    for ell in [1e-8, 1e-4, 1e-2, 0.2]:
        for r in (1, 2, 4, 8):
            co = zo.zolotarev_coeffs(ell, r)
            if zo.one_minus_zhat_at_ell(co) < 1e-7:
                continue                       # amplitude below what sampling resolves
            x = np.geomspace(ell, 1.0, 200001)
            z = zo.zhat(x, co)
            lo = float(zo.zhat(ell, co))
            assert z.max() <= 1.0 + 1e-13
            assert z.min() >= lo - 1e-13 * max(1.0, lo)
            # local extrema of the sampled curve, endpoints included
            dz = np.sign(np.diff(z))
            turns = np.nonzero(dz[1:] != dz[:-1])[0] + 1
            ext = np.concatenate([[0], turns, [len(x) - 1]])
            vals = z[ext]
            assert len(ext) == 2 * r + 2, (ell, r, len(ext))
            hi_pts, lo_pts = vals[1::2], vals[0::2]
            assert np.allclose(hi_pts, 1.0, atol=1e-6), (ell, r, hi_pts)
            assert np.allclose(lo_pts, lo, rtol=1e-6, atol=1e-9), (ell, r, lo_pts, lo)


def test_gap_formula_against_direct_and_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    for ell in [1e-10, 1e-4, 0.01, 0.1, 0.5, 0.9]:
        for r in (1, 3, 6, 8):
            co = zo.zolotarev_coeffs(ell, r)
            gap = zo.one_minus_zhat_at_ell(co)
            direct = 1.0 - float(zo.zhat(ell, co))
            if direct > 1e-6:
                assert gap == pytest.approx(direct, rel=1e-9)
            # the same gap from mpmath's elliptic functions at 60 digits
            L = mp.mpf(ell)
            m = 1 - L * L
            Kp = mp.ellipk(m)
            c = [L * L * (mp.ellipfun("sn", i * Kp / (2 * r + 1), m=m)
                          / mp.ellipfun("cn", i * Kp / (2 * r + 1), m=m)) ** 2
                 for i in range(1, 2 * r + 1)]
            M = mp.mpf(1)
            for j in range(r):
                M *= (1 + c[2 * j]) / (1 + c[2 * j + 1])
            z = M * L
            for j in range(r):
                z *= (L * L + c[2 * j + 1]) / (L * L + c[2 * j])
            ref = 1 - z
            if ref > mp.mpf("1e-300"):
                assert gap == pytest.approx(float(ref), rel=1e-10), (ell, r)


def test_choose_r_is_smallest_with_two_iterations():
    for kappa in [1.5, 10, 1e2, 1e4, 1e6, 1e8, 1e10, 1e12]:
        r = zo.choose_r(1.0 / kappa)
        assert len(zo.ell_schedule(1.0 / kappa, r)) - 1 <= 2
        if r > 1:
            assert len(zo.ell_schedule(1.0 / kappa, r - 1)) - 1 > 2


def test_qr_then_cholesky_switch_on_workloads():
    # kappa 1e8 r=3: QR then two Cholesky passes; kappa 1e12 r=8 and 1e6 r=6: QR then Cholesky.
    for kappa, r, want in [(1e8, 3, [True, False, False]), (1e12, 8, [True, False]),
                           (1e6, 6, [True, False]), (1e16, 8, [True, False])]:
        ells = zo.ell_schedule(1.0 / kappa, r)
        got = [zo.uses_qr(zo.zolotarev_coeffs(e, r), e) for e in ells[:-1]]
        assert got == want, (kappa, r, got)


# --- planted mistakes: each plausible misreading must fail one of the pins -------

def test_printed_eq10_product_breaks_theorem1(monkeypatch):
    real = zo.zolotarev_coeffs

    def printed(ell, r):
        co = real(ell, r)
        c_odd, c_even = co.c[0::2], co.c[1::2]
        co.a = np.array([-np.prod(c_odd[j] - c_even)
                         * np.prod([c_odd[j] - c_odd[k] for k in range(r) if k != j])
                         for j in range(r)])
        return co
    co = printed(0.01, 3)
    x = np.geomspace(0.01, 1.0, 50)
    assert np.max(np.abs(zo.zhat(x, co) - zo.zhat_partial_fraction(x, co))) > 1e-3


def test_printed_ell_update_breaks_table1(monkeypatch):
    def printed_gap(co):
        ell = co.ell
        z = co.Mhat * ell
        for j in range(co.r):
            z *= (ell + co.c[2 * j + 1]) / (ell * ell + co.c[2 * j])
        return 1.0 - min(1.0, z)
    monkeypatch.setattr(zo, "one_minus_zhat_at_ell", printed_gap)
    kappas, table = read_table1()
    got = {r: [zo.iterations_needed(k, r) for k in kappas] for r in table}
    assert any(got[r] != table[r] for r in table)


def test_modulus_read_as_parameter_breaks_mpmath_pin():
    # sn/cn at modulus l' versus at parameter l' (modulus sqrt(l')): c_i differ.
    ell, r = 0.1, 3
    co = zo.zolotarev_coeffs(ell, r)
    alt = zo.zolotarev_coeffs(math.sqrt(1.0 - math.sqrt(1.0 - ell * ell)), r)
    assert np.max(np.abs(co.c - alt.c) / co.c) > 1e-3
