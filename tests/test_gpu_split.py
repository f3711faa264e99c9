"""GPU checks of the split-precision (Ozaki) tensor-core path through the C ABI.

The BF16 form's product of S six-bit slices per operand carries an error of at
most about 2 K 2^-6S max_k|A_ik| max_k|B_kj| per entry (truncation of each
operand after S digits); the FP16 form's eight seven-bit slices (36 slice pairs)
and the FP8 form's eleven five-bit slices (76 slice pairs) reach the same
grade as nine BF16 slices.  Integer matrices whose digits fit are
multiplied exactly.  The full decomposition in either split form must meet the
same invariants as FP64."""
import math

import numpy as np
import pytest

from oracle import zolo_oracle as zo
from paper_1806_06204_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06204_gb300 import build
    build.build()
    from paper_1806_06204_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def handle(zb):
    h = zb.Handle(0)
    yield h
    h.close()


def dev(a):
    import torch
    return torch.from_numpy(np.asfortranarray(a)).cuda()


def opnp(X, t):
    return X.T if t else X


@pytest.mark.parametrize("m,n,k,ta,tb", [(64, 64, 64, 0, 0), (200, 130, 300, 0, 1), (33, 257, 1100, 1, 0),
                                         (129, 65, 2100, 1, 1), (1, 5, 7, 0, 0), (300, 16, 40, 0, 0)])
@pytest.mark.parametrize("prec,S", [(0, 0), (1, 8), (1, 9), (2, 8), (3, 11)])
def test_dgemm_matches_numpy(zb, handle, m, n, k, ta, tb, prec, S):
    rng = np.random.default_rng(m * 7 + n + k)
    A = rng.standard_normal((k, m) if ta else (m, k)) * np.exp(rng.uniform(-3, 3, (1, 1)))
    B = rng.standard_normal((n, k) if tb else (k, n))
    C0 = rng.standard_normal((m, n))
    alpha, beta = 0.7, -1.3
    C = dev(C0)
    zb.zolo_dgemm(handle, dev(A), dev(B), C, alpha=alpha, beta=beta, transA=bool(ta), transB=bool(tb),
                  prec=prec, slices=S)
    ref = alpha * opnp(A, ta) @ opnp(B, tb) + beta * C0
    got = C.cpu().numpy()
    if prec == 0:
        tol = 1e-13 * (np.abs(opnp(A, ta)) @ np.abs(opnp(B, tb)) + np.abs(C0))
    else:
        amax = np.max(np.abs(opnp(A, ta)), axis=1, keepdims=True)
        bmax = np.max(np.abs(opnp(B, tb)), axis=0, keepdims=True)
        bits = 6 * S if prec == 1 else 54   # FP16, FP8: the grade of nine BF16 slices
        tol = 2.0 * k * 2.0 ** (-bits) * abs(alpha) * amax * bmax * 4 + 1e-15 * np.abs(ref) + 1e-300
    assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) / tol)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_split_integer_products_are_exact(zb, handle, prec):
    # entries of at most two digits (|x| < 64: one base-64 or base-128 digit, two
    # base-32 ones, after the row scale): every slice product is an integer sum
    # below 2^24 within a chunk and no level is dropped, so the result is exact
    rng = np.random.default_rng(5)
    A = rng.integers(-63, 64, (256, 1024)).astype(np.float64)
    B = rng.integers(-63, 64, (1024, 192)).astype(np.float64)
    C = zb.zolo_dgemm(handle, dev(A), dev(B), prec=prec, slices=8 if prec < 3 else 0)
    assert np.array_equal(C.cpu().numpy(), A @ B)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_split_nonfinite_rows_and_columns_give_nan(zb, handle, prec):
    # an Inf or NaN leaves no digits to multiply: its row of op(A) or column of
    # op(B) comes out NaN (FP64 gives NaN or Inf there); every other entry is the
    # product as usual
    rng = np.random.default_rng(17)
    A = rng.standard_normal((64, 100))
    B = rng.standard_normal((100, 40))
    A[3, 17] = np.nan
    A[10, 5] = np.inf
    B[7, 2] = -np.inf
    C = zb.zolo_dgemm(handle, dev(A), dev(B), prec=prec).cpu().numpy()
    with np.errstate(invalid="ignore", over="ignore"):
        ref = A @ B
    bad = ~np.isfinite(ref)
    assert np.array_equal(~np.isfinite(C), bad)
    assert np.all(np.isnan(C[bad]))
    ok = ~bad
    # the bound of test_dgemm_matches_numpy (eight 6-bit BF16 slices by default)
    bits = 48 if prec == 1 else 54
    amax = np.where(np.isfinite(A), np.abs(A), 0.0).max(axis=1, keepdims=True)
    bmax = np.where(np.isfinite(B), np.abs(B), 0.0).max(axis=0, keepdims=True)
    tol = 2.0 * 100 * 2.0 ** (-bits) * amax * bmax * 4 + 1e-15 * np.abs(np.where(ok, ref, 0.0))
    assert np.all(np.abs(C[ok] - ref[ok]) <= tol[ok])


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_split_long_k_stays_exact(zb, handle, prec):
    # every digit at its bound over K = 150000 terms: the level sums would overflow
    # the epilogue's int64 in one product; gemm_split cuts K into pieces that fit
    # (114688 terms for BF16 and FP8, 61440 for FP16) and adds them in FP64
    from fractions import Fraction
    K = 150000
    a, b = 0.4999, -0.4999
    A = np.full((8, K), a)
    B = np.full((K, 8), b)
    C = zb.zolo_dgemm(handle, dev(A), dev(B), prec=prec).cpu().numpy()
    ref = float(Fraction(a) * Fraction(b) * K)
    assert np.max(np.abs(C - ref)) <= 1e-14 * abs(ref)


@pytest.mark.parametrize("m,n,kappa,r,form", [(256, 256, 1e8, 3, 1), (300, 160, 1e6, 6, 1),
                                              (384, 384, 1e12, 8, 1), (384, 384, 1e12, 8, 2),
                                              (800, 200, 1e6, 6, 0)])
@pytest.mark.parametrize("prec", [1, 2, 3])
def test_split_pd_meets_invariants_and_matches_oracle(zb, handle, m, n, kappa, r, form, prec):
    # form 2 / the 800 x 200 auto case: Cholesky-form iterations through W = sum_j a_j Z_j^{-1}
    sm = synth.make_matrix(m, n, synth.geometric_sigma(n, kappa), seed=3100 + m)
    beta = float(sm.sigma[-1])
    Qp, H, info = zb.zolo_pd(handle, dev(sm.A), zb.opts(beta=beta, r=r, prec=prec,
                                                         ns_steps=1, chol_form=form))
    Qo, Ho, io = zo.zolo_pd(sm.A, 1.0, beta, r=r, ns_steps=1)
    Qp, H = Qp.cpu().numpy(), H.cpu().numpy()
    assert info.iters == io.iters and info.used_qr == io.used_qr
    assert zo.backward_error_pd(sm.A, Qp, H) <= 1e-13
    assert zo.orthogonality(Qp) <= 1e-13
    assert np.array_equal(H, H.T)
    # H is well conditioned (its perturbation is Qp's times A): FP64's tolerance
    assert np.linalg.norm(H - Ho) <= 1e-13 * np.linalg.norm(Ho)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_split_svd_sigma(zb, handle, prec):
    sm = synth.square_geometric(256, 1e8, seed=1000)
    U, S, V, info = zb.zolo_svd(handle, dev(sm.A), zb.opts(beta=1e-8, r=3, prec=prec,
                                                          ns_steps=1))
    assert np.max(np.abs(S.cpu().numpy() - sm.sigma)) <= 1e-12
