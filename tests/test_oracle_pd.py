"""Pins for the oracle's Zolo-PD and Zolo-SVD (Eqs. 11-12, Algorithms 1-2).

One iteration is checked against the closed form of Theorem 2 built from the
generator's own U, sigma, V; the full decomposition against the invariants that
define it (Q_p^T Q_p = I, H symmetric positive semidefinite, A = Q_p H), against
the polar factor U V^T, and the SVD against the generator's sigma and brute force."""
import math

import numpy as np
import pytest

from oracle import zolo_oracle as zo
from paper_1806_06204_gb300 import synth


def closed_form_step(sm, alpha, co):
    # Theorem 2: Zhat(X) = U diag(Zhat(sigma_i / alpha)) V^T
    return (sm.U * zo.zhat(sm.sigma / alpha, co)) @ sm.V.T


@pytest.mark.parametrize("kappa,r", [(1e4, 3), (1e8, 6), (1e12, 8)])
def test_qr_step_equals_theorem2_closed_form(kappa, r):
    sm = synth.square_geometric(24, kappa, seed=11)
    co = zo.zolotarev_coeffs(1.0 / kappa, r)
    X1 = zo.zolo_step_qr(sm.A / 1.0, co)
    ref = closed_form_step(sm, 1.0, co)
    # rounding in the smallest singular directions is amplified by ~Zhat(l)/l
    amp = float(zo.zhat(1.0 / kappa, co)) * kappa
    assert np.linalg.norm(X1 - ref) / np.linalg.norm(ref) < 1e-13 + 20 * zo.EPS * amp
    # and the explicit-inverse form of Eq. (11), for the well conditioned case
    if kappa <= 1e4:
        X = sm.A
        S = sum(co.a[j] * X @ np.linalg.inv(X.T @ X + co.c[2 * j] * np.eye(24)) for j in range(r))
        assert np.linalg.norm(X1 - co.Mhat * (X + S)) / np.linalg.norm(X1) < 1e-9


@pytest.mark.parametrize("kappa,r", [(2.0, 3), (10.0, 4), (50.0, 8)])
def test_cholesky_step_equals_theorem2_closed_form(kappa, r):
    sm = synth.tall_uniform(40, 16, lo=1.0 / kappa, seed=12)
    co = zo.zolotarev_coeffs(1.0 / kappa, r)
    X1 = zo.zolo_step_chol(sm.A, co)
    ref = closed_form_step(sm, 1.0, co)
    assert np.linalg.norm(X1 - ref) / np.linalg.norm(ref) < 1e-13


def test_transposed_q2_breaks_theorem2():
    # planted mistake: Q_{j1} Q_{j2} instead of Q_{j1} Q_{j2}^T
    sm = synth.square_geometric(16, 1e4, seed=13)
    co = zo.zolotarev_coeffs(1e-4, 3)
    X, n = sm.A, 16
    S = np.zeros_like(X)
    for j in range(3):
        W = np.vstack([X, math.sqrt(co.c[2 * j]) * np.eye(n)])
        refl, _ = zo.householder_qr(W)
        Q = zo.thin_q(refl, 2 * n, n)
        S += co.a[j] / math.sqrt(co.c[2 * j]) * (Q[:n] @ Q[n:])
    bad = co.Mhat * (X + S)
    assert np.linalg.norm(bad - closed_form_step(sm, 1.0, co)) > 1e-3


def test_pd_invariants_256_kappa_1e8():
    sm = synth.square_geometric(256, 1e8, seed=1000)
    Qp, H, info = zo.zolo_pd(sm.A, 1.0, sm.sigma[-1], r=3)
    assert info.iters == 3 and info.used_qr == [True, False, False]
    assert zo.orthogonality(Qp) < 1e-13
    assert zo.backward_error_pd(sm.A, Qp, H) < 1e-13
    assert np.array_equal(H, H.T)
    assert np.linalg.eigvalsh(H).min() > -1e-13
    # polar factor of a full-rank A is U V^T; conditioning ~ 1/(sigma_{n-1} + sigma_n)
    assert np.linalg.norm(Qp - sm.U @ sm.V.T) < 1e-14 * 1e8 * 16


def test_pd_tall_and_ell_schedule():
    sm = synth.tall_uniform(300, 120, lo=1e-6, seed=3000)
    Qp, H, info = zo.zolo_pd(sm.A, 1.0, 1e-6, r=6)
    assert info.iters == 2 and info.used_qr == [True, False]
    assert zo.orthogonality(Qp) < 1e-13 and zo.backward_error_pd(sm.A, Qp, H) < 1e-13
    assert 1.0 - info.ells[-1] <= 1e-15


def test_posteriori_test_adds_the_papers_extra_iteration():
    # Section 4 reports one iteration more than Table 1; the literal test of
    # Algorithm 1 step (d) does that for kappa 1e12, r 8 (delta_2 ~ 0.23 > eps^(1/17)).
    sm = synth.square_geometric(64, 1e12, seed=7)
    _, _, a = zo.zolo_pd(sm.A, 1.0, sm.sigma[-1], r=8)
    Qp, H, b = zo.zolo_pd(sm.A, 1.0, sm.sigma[-1], r=8, posteriori=True)
    assert a.iters == 2 and b.iters == 3 and b.extra_iters == 1
    assert b.delta[-1] < zo.EPS ** (1.0 / 17)
    assert zo.backward_error_pd(sm.A, Qp, H) < 1e-13


def test_alpha_above_sigma_max_and_default_r():
    sm = synth.square_geometric(48, 1e5, seed=21)
    Qp, H, info = zo.zolo_pd(sm.A, 3.0, sm.sigma[-1] / 2.0)
    assert info.r == zo.choose_r(sm.sigma[-1] / 6.0)
    assert zo.orthogonality(Qp) < 1e-13 and zo.backward_error_pd(sm.A, Qp, H) < 1e-13


def test_newton_schulz_restores_orthogonality_at_kappa_1e16():
    sm = synth.square_geometric(128, 1e16, seed=1000)
    Qp, H, _ = zo.zolo_pd(sm.A, 1.0, 1e-16, r=8)
    Qn, Hn, _ = zo.zolo_pd(sm.A, 1.0, 1e-16, r=8, ns_steps=1)
    assert zo.orthogonality(Qp) > 1e-13          # sigma at rounding level costs orthogonality
    assert zo.orthogonality(Qn) < 1e-14
    assert zo.backward_error_pd(sm.A, Qn, Hn) < 1e-13


@pytest.mark.parametrize("n,kappa,r", [(256, 1e8, 3), (128, 1e12, 8)])
def test_svd_against_generator_sigma(n, kappa, r):
    sm = synth.square_geometric(n, kappa, seed=1000)
    U, S, V, _ = zo.zolo_svd(sm.A, 1.0, sm.sigma[-1], r=r)
    assert np.max(np.abs(S - sm.sigma)) <= 1e-12 * sm.sigma[0]
    assert np.all(np.diff(S) <= 0)
    assert zo.svd_residual(sm.A, U, S, V) < 1e-13
    assert zo.orthogonality(U) < 1e-13 and zo.orthogonality(V) < 1e-13


def test_svd_against_brute_force_one_sided_jacobi():
    sm = synth.make_matrix(20, 14, np.geomspace(1, 1e-4, 14), seed=31)
    U, S, V, _ = zo.zolo_svd(sm.A, 1.0, 1e-4)
    Ub, Sb, Vb = zo.one_sided_jacobi_svd(sm.A)
    assert np.max(np.abs(S - Sb)) < 1e-14
    # singular vectors up to sign (distinct singular values)
    assert np.allclose(np.abs(np.sum(U * Ub, axis=0)), 1.0, atol=1e-9)
    assert np.allclose(np.abs(np.sum(V * Vb, axis=0)), 1.0, atol=1e-9)


@pytest.mark.parametrize("qr,kappa", [(True, 1e6), (False, 20.0)])
def test_group_terms_each_equal_the_closed_form_term(qr, kappa):
    # Algorithm 3 step 4(c): group j forms T_j = a_j X (X^T X + c_{2j-1} I)^{-1}
    # (Theorem 2), which on X = U diag(sigma) V^T is U diag(a_j sigma / (sigma^2 + c)) V^T
    sm = synth.square_geometric(20, kappa, seed=14) if qr else synth.tall_uniform(30, 12, 1 / kappa, 15)
    r = 5
    co = zo.zolotarev_coeffs(1.0 / kappa, r)
    for j in range(r):
        c = co.c[2 * j]
        ref = (sm.U * (co.a[j] * sm.sigma / (sm.sigma ** 2 + c))) @ sm.V.T
        got = zo.group_terms(sm.A, co, [j], qr)
        tol = 1e-13 if not qr else 1e-13 + 50 * zo.EPS * kappa
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol, j


@pytest.mark.parametrize("qr", [True, False])
def test_groups_of_a_partition_sum_to_the_whole_step(qr):
    # Algorithm 3 step 4(d): the sum over the groups is the one-process step
    sm = synth.tall_uniform(28, 12, 1e-2 if not qr else 1e-6, seed=16)
    ell = float(sm.sigma[-1])
    co = zo.zolotarev_coeffs(ell, 7)
    whole = zo.zolo_step_qr(sm.A, co) if qr else zo.zolo_step_chol(sm.A, co)
    for parts in ([range(7)], [range(0, 3), range(3, 7)], [range(0, 2), range(2, 4), range(4, 6),
                                                          range(6, 7)]):
        S = sum(zo.group_terms(sm.A, co, p, qr) for p in parts)
        got = co.Mhat * (sm.A + S)
        assert np.linalg.norm(got - whole) / np.linalg.norm(whole) < 1e-14
    # a partition that drops a shift is caught
    S = zo.group_terms(sm.A, co, range(0, 6), qr)
    assert np.linalg.norm(co.Mhat * (sm.A + S) - whole) / np.linalg.norm(whole) > 1e-6
