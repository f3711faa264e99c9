"""Pins for the oracle's dense kernels against textbook/library routines (numpy/LAPACK)."""
import math

import numpy as np
import pytest

from oracle import zolo_oracle as zo


def rng(seed=0):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("p,n", [(7, 3), (40, 17), (64, 64), (97, 41)])
def test_householder_qr_matches_lapack(p, n):
    W = rng(p * n).standard_normal((p, n))
    refl, R = zo.householder_qr(W)
    Q = zo.thin_q(refl, p, n)
    Qn, Rn = np.linalg.qr(W)
    # unique up to the signs of R's rows
    d = np.sign(np.diag(R)) * np.sign(np.diag(Rn))
    assert np.allclose(R, d[:, None] * Rn, atol=1e-12 * np.abs(Rn).max())
    assert np.allclose(Q, Qn * d, atol=1e-12)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) < 1e-13
    assert np.linalg.norm(Q @ R - W) < 1e-13 * np.linalg.norm(W)


def test_householder_vector_zero_tail():
    v, tau, beta = zo.householder_vector(np.array([3.0, 0.0, 0.0]))
    assert tau == 0.0 and beta == 3.0 and v[0] == 1.0


def test_cholesky_and_solves_match_lapack():
    X = rng(3).standard_normal((50, 20))
    Z = X.T @ X + 0.3 * np.eye(20)
    R = zo.cholesky_upper(Z)
    assert np.allclose(R, np.linalg.cholesky(Z).T, atol=1e-12)
    Y = zo.solve_right_upper(X, R)
    assert np.allclose(Y, np.linalg.solve(R.T, X.T).T, atol=1e-12)
    W = zo.solve_right_upper_transpose(Y, R)
    assert np.allclose(W, X @ np.linalg.inv(Z), atol=1e-11)


def test_cholesky_breakdown_raises():
    with pytest.raises(np.linalg.LinAlgError):
        zo.cholesky_upper(np.array([[1.0, 2.0], [2.0, 1.0]]))


@pytest.mark.parametrize("n", [1, 2, 9, 40])
def test_eigh_matches_lapack(n):
    g = rng(n)
    Q, _ = np.linalg.qr(g.standard_normal((n, n)))
    lam = np.geomspace(1.0, 1e-9, n)
    H = (Q * lam) @ Q.T
    H = 0.5 * (H + H.T)
    got, V = zo.jacobi_eigh(H)
    order = np.argsort(-got)
    got, V = got[order], V[:, order]
    ref, Vn = np.linalg.eigh(H)
    ref, Vn = ref[::-1], Vn[:, ::-1]
    assert np.max(np.abs(got - ref)) < 1e-14
    assert np.linalg.norm(V.T @ V - np.eye(n)) < 1e-13
    assert np.linalg.norm(H - (V * got) @ V.T) < 1e-14 * n
    # eigenvectors of well separated eigenvalues agree up to sign
    assert np.allclose(np.abs(np.sum(V * Vn, axis=0))[lam > 1e-6], 1.0, atol=1e-8)


def test_eigh_semidefinite_falls_back_to_shift():
    Q, _ = np.linalg.qr(rng(5).standard_normal((12, 12)))
    lam = np.concatenate([np.linspace(1, 0.1, 10), [0.0, -1e-17]])
    H = (Q * lam) @ Q.T
    got, V = zo.jacobi_eigh(0.5 * (H + H.T))
    assert np.max(np.abs(np.sort(got) - np.sort(lam))) < 1e-14


@pytest.mark.parametrize("m,n", [(5, 5), (12, 7), (30, 30)])
def test_one_sided_jacobi_svd_matches_lapack(m, n):
    A = rng(m + n).standard_normal((m, n))
    U, S, V = zo.one_sided_jacobi_svd(A)
    assert np.allclose(S, np.linalg.svd(A, compute_uv=False), atol=1e-13)
    assert np.linalg.norm(A - (U * S) @ V.T) < 1e-13 * np.linalg.norm(A)
    assert np.linalg.norm(U.T @ U - np.eye(n)) < 1e-13


def test_hestenes_odd_column_count():
    X = rng(2).standard_normal((9, 7))
    Y, _ = zo.hestenes_columns(X)
    G = Y.T @ Y
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() < 1e-13
    assert np.allclose(np.sort(np.linalg.norm(Y, axis=0)), np.sort(np.linalg.svd(X, compute_uv=False)))


@pytest.mark.parametrize("m,n,kappa", [(6, 6, 10.0), (40, 25, 1e6), (33, 33, 1e10)])
def test_beta_estimate_closed_form(m, n, kappa):
    # With X0 = A/alpha = QR the singular values of R are those of X0, so
    # ||R^{-1}||_F^2 = sum_i (alpha/sigma_i)^2 and the estimate is
    # (sum_i sigma_i^{-2})^{-1/2} whatever alpha is: sigma_min/sqrt(n) <= beta <= sigma_min.
    r = rng(m * n)
    sig = np.geomspace(1.0, 1.0 / kappa, n) * 3.0
    U, _ = np.linalg.qr(r.standard_normal((m, n)))
    V, _ = np.linalg.qr(r.standard_normal((n, n)))
    A = (U * sig) @ V.T
    want = 1.0 / math.sqrt(np.sum(sig ** -2.0))
    for alpha in (sig.max(), 7.0 * sig.max()):
        got = zo.beta_estimate(A, alpha)
        assert abs(got - want) <= (1e-12 + 10 * zo.EPS * kappa) * want
        assert sig.min() / math.sqrt(n) * (1 - 1e-9) <= got <= sig.min() * (1 + 1e-9)


def test_beta_estimate_diagonal_and_identity():
    d = np.array([4.0, -0.5, 2.0, 0.25])
    assert zo.beta_estimate(np.diag(d), 4.0) == pytest.approx(1.0 / math.sqrt(np.sum(d ** -2.0)),
                                                              rel=1e-15)
    # all singular values equal: the estimate is sigma / sqrt(n), the loosest case
    assert zo.beta_estimate(np.eye(9), 1.0) == pytest.approx(1.0 / 3.0, rel=1e-15)


def test_alpha_bound_exact_cases_and_upper_bound():
    # diagonal: ||A||_1 = ||A||_inf = max |d_i| = ||A||_2, so the Hoelder bound is exact
    d = np.array([0.5, -3.0, 2.0])
    assert zo.alpha_bound(np.diag(d)) == pytest.approx(3.0, rel=1e-15)
    # all ones, m x n: rank one with ||A||_2 = ||A||_F = sqrt(mn) = sqrt(||A||_1 ||A||_inf)
    assert zo.alpha_bound(np.ones((6, 4))) == pytest.approx(math.sqrt(24.0), rel=1e-15)
    # an orthonormal-column matrix: ||A||_2 = 1 while ||A||_F = sqrt(n)
    Q, _ = np.linalg.qr(rng(3).standard_normal((50, 20)))
    b = zo.alpha_bound(Q)
    assert 1.0 - 1e-14 <= b <= math.sqrt(20.0) + 1e-12
    for seed in range(5):
        A = rng(seed).standard_normal((30, 17)) * rng(seed + 9).uniform(0.01, 10, 17)
        assert zo.alpha_bound(A) >= np.linalg.norm(A, 2) * (1 - 1e-14)
        assert zo.alpha_bound(A) <= np.linalg.norm(A) * (1 + 1e-15)


@pytest.mark.parametrize("m,n", [(9, 5), (40, 17), (33, 33)])
def test_stacked_qr_structure_of_section_3_1(m, n):
    # The structure the GPU's structured QR is built on (Section 3.1): for
    # W = [X; sqrt(c) I], the dense Householder QR's k-th reflector is non-zero
    # only on rows k..m+k, and the lower block Q2 of the thin Q is upper triangular
    # (both exactly: the zeros are structural)
    X = rng(m * 7 + n).standard_normal((m, n))
    W = np.vstack([X, math.sqrt(0.37) * np.eye(n)])
    refl, R = zo.householder_qr(W)
    for k, (v, tau) in enumerate(refl):
        rows = np.nonzero(v)[0] + k           # v acts on rows k.. of W
        assert rows.min() == k and rows.max() == m + k
    Q = zo.thin_q(refl, m + n, n)
    assert np.all(np.tril(Q[m:], -1) == 0.0)
    assert np.linalg.norm(Q @ R - W) <= 1e-13 * np.linalg.norm(W)


def test_compact_wy_block_merge():
    # The merge the block T factor is built with: for reflector blocks V1, V2 with
    # I - V1 T1 V1^T and I - V2 T2 V2^T, their product is I - V T V^T with
    # V = [V1 V2] and T = [[T1, -T1 (V1^T V2) T2], [0, T2]]  (Schreiber-Van Loan)
    p, k1, k2 = 30, 6, 5
    refl, _ = zo.householder_qr(rng(21).standard_normal((p, k1 + k2)))
    V = np.zeros((p, k1 + k2))
    taus = []
    for k, (v, tau) in enumerate(refl):
        V[k:, k] = v
        taus.append(tau)

    def t_factor(Vb, tb):
        # I - Vb T Vb^T = H_1 ... H_k, column by column
        k = Vb.shape[1]
        T = np.zeros((k, k))
        for j in range(k):
            T[j, j] = tb[j]
            T[:j, j] = -tb[j] * T[:j, :j] @ (Vb[:, :j].T @ Vb[:, j])
        return T

    V1, V2 = V[:, :k1], V[:, k1:]
    T1, T2 = t_factor(V1, taus[:k1]), t_factor(V2, taus[k1:])
    T = np.block([[T1, -T1 @ (V1.T @ V2) @ T2], [np.zeros((k2, k1)), T2]])
    prod = np.eye(p)
    for k in range(k1 + k2):
        prod = prod @ (np.eye(p) - taus[k] * np.outer(V[:, k], V[:, k]))
    assert np.allclose(np.eye(p) - V @ T @ V.T, prod, atol=1e-14)
    assert np.allclose(T, t_factor(V, taus), atol=1e-14)
