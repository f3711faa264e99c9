"""GPU parity: libzolo through its C ABI against the CPU oracle.

Tolerances: the polar factor is unique for full-rank A but its sensitivity is
~1/(sigma_{n-1} + sigma_n) (relative to ||A||), so Qp is compared entry-wise
within c eps / ((sigma_{n-1} + sigma_n)/alpha); H = sym(Qp^T A) and the singular
values are well conditioned and are compared at ~1e-13.  Every result must also
meet the contract's invariants: ||A - Qp H||_F/||A||_F <= 1e-13,
||Qp^T Qp - I||_F/sqrt(n) <= 1e-13, |sigma_i - sigma_i^oracle| <= 1e-12 sigma_1.
"""
import math

import numpy as np
import pytest

from oracle import zolo_oracle as zo
from paper_1806_06204_gb300 import synth

pytestmark = pytest.mark.gpu

EPS = zo.EPS


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


def host(t):
    return t.cpu().numpy()


def polar_tol(sm, alpha=1.0, c=200.0):
    s = np.sort(sm.sigma)
    gap = s[0] + s[1] if len(s) > 1 else s[0]
    return c * EPS / (gap / alpha)


def check_pd_invariants(A, Qp, H):
    assert zo.orthogonality(Qp) <= 1e-13
    assert zo.backward_error_pd(A, Qp, H) <= 1e-13
    assert np.array_equal(H, H.T)
    assert np.linalg.eigvalsh(H).min() >= -1e-13 * np.linalg.norm(A, 2)


# --------------------------------------------------------------- one iteration

@pytest.mark.parametrize("m,n,kappa,r", [(64, 64, 1e6, 4), (97, 61, 1e10, 8), (40, 40, 1e2, 2),
                                         (130, 70, 1e4, 3)])
def test_one_qr_iteration_matches_oracle(zb, handle, m, n, kappa, r):
    # force the QR form (Eq. 12) and stop after one iteration
    sm = synth.make_matrix(m, n, synth.geometric_sigma(n, kappa), seed=2000 + m)
    o = zb.opts(beta=1.0 / kappa, r=r, max_iter=1, force_qr=1)
    X1, _, info = zb.zolo_pd(handle, dev(sm.A), o)
    co = zo.zolotarev_coeffs(1.0 / kappa, r)
    ref = zo.zolo_step_qr(sm.A, co)
    amp = float(zo.zhat(1.0 / kappa, co)) * kappa
    err = np.linalg.norm(host(X1) - ref) / np.linalg.norm(ref)
    assert info.iters == 1 and info.used_qr == [True]
    assert err < 1e-13 + 50 * EPS * amp, err


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("m,n,kappa,r", [(64, 64, 5.0, 3), (200, 65, 20.0, 5), (33, 1, 1.5, 1),
                                         (129, 129, 50.0, 8), (300, 130, 30.0, 2)])
def test_one_cholesky_iteration_matches_oracle(zb, handle, m, n, kappa, r, form):
    # form 1: the triangular solves of Algorithm 1 (d); form 2: X sum_j a_j Z_j^{-1}
    # through explicit R_j^{-1} (the same rational function of X^T X)
    sm = synth.make_matrix(m, n, synth.geometric_sigma(n, kappa), seed=2100 + m)
    o = zb.opts(beta=1.0 / kappa, r=r, max_iter=1, force_qr=0, chol_form=form)
    X1, _, info = zb.zolo_pd(handle, dev(sm.A), o)
    co = zo.zolotarev_coeffs(1.0 / kappa, r)
    ref = zo.zolo_step_chol(sm.A, co)
    assert info.iters == 1 and info.used_qr == [False]
    assert np.linalg.norm(host(X1) - ref) / np.linalg.norm(ref) < 1e-13


# ------------------------------------------------------------------ full PD

@pytest.mark.parametrize("m,n,kappa,r", [(256, 256, 1e8, 3), (300, 120, 1e6, 6), (128, 128, 1e12, 8),
                                         (77, 77, 1e2, 0), (1, 1, 1.0, 1), (65, 33, 1e4, 0),
                                         # r = 1 is the dynamically weighted Halley step: QDWH-PD
                                         (256, 256, 1e8, 1), (120, 80, 1e12, 1)])
def test_pd_matches_oracle(zb, handle, m, n, kappa, r):
    sm = synth.make_matrix(m, n, synth.geometric_sigma(n, kappa), seed=1000 + m + n)
    beta = float(sm.sigma[-1])
    Qp, H, info = zb.zolo_pd(handle, dev(sm.A), zb.opts(beta=beta, r=r))
    Qo, Ho, io = zo.zolo_pd(sm.A, 1.0, beta, r=r)
    Qp, H = host(Qp), host(H)
    assert info.r == io.r and info.iters == io.iters and info.used_qr == io.used_qr
    assert np.allclose(info.ell, io.ells, rtol=1e-14, atol=1e-15)
    check_pd_invariants(sm.A, Qp, H)
    assert np.linalg.norm(H - Ho) <= 1e-13 * np.linalg.norm(Ho)
    assert np.linalg.norm(Qp - Qo) <= polar_tol(sm) * math.sqrt(n)
    # per-iteration relative changes agree (the a-posteriori quantity of Algorithm 1);
    # late, small deltas are carried by the smallest singular directions, whose
    # iterates differ by about eps * kappa between two correct runs
    assert np.allclose(info.delta, io.delta, rtol=max(1e-6, 10 * EPS * kappa), atol=1e-13)


@pytest.mark.parametrize("m,n,kappa,r", [(6400, 48, 1e6, 3), (7000, 33, 1e10, 2),
                                         (2500, 40, 1e8, 4)])
def test_tall_panels_in_global_memory_match_oracle(zb, handle, m, n, kappa, r):
    # m + 32 > 8 x 768 rows: the QR panels run in the cluster kernel that keeps the
    # panel in global memory (512 threads per CTA); 2500 rows: the shared-memory
    # cluster kernel with more rows per CTA than threads; two panels, the last ragged
    sm = synth.make_matrix(m, n, synth.geometric_sigma(n, kappa), seed=4000 + m + n)
    beta = float(sm.sigma[-1])
    Qp, H, info = zb.zolo_pd(handle, dev(sm.A), zb.opts(beta=beta, r=r))
    Qo, Ho, io = zo.zolo_pd(sm.A, 1.0, beta, r=r)
    Qp, H = host(Qp), host(H)
    assert info.iters == io.iters and info.used_qr == io.used_qr and io.used_qr[0]
    check_pd_invariants(sm.A, Qp, H)
    assert np.linalg.norm(H - Ho) <= 1e-13 * np.linalg.norm(Ho)
    assert np.linalg.norm(Qp - Qo) <= polar_tol(sm) * math.sqrt(n)


@pytest.mark.parametrize("m,n,kappa,r,form", [(700, 200, 1e6, 6, 0), (256, 256, 1e12, 8, 2),
                                              (520, 130, 1e8, 2, 2), (190, 190, 1e4, 3, 1)])
def test_pd_inverse_cholesky_form_matches_oracle(zb, handle, m, n, kappa, r, form):
    # 700 x 200 with r = 6: the flop model picks the inverse form by itself
    sm = synth.make_matrix(m, n, synth.geometric_sigma(n, kappa), seed=3000 + m + n)
    beta = float(sm.sigma[-1])
    Qp, H, info = zb.zolo_pd(handle, dev(sm.A), zb.opts(beta=beta, r=r, chol_form=form))
    Qo, Ho, io = zo.zolo_pd(sm.A, 1.0, beta, r=r)
    Qp, H = host(Qp), host(H)
    assert info.iters == io.iters and info.used_qr == io.used_qr and not all(io.used_qr)
    assert info.chol_form == (form or 2)
    check_pd_invariants(sm.A, Qp, H)
    assert np.linalg.norm(H - Ho) <= 1e-13 * np.linalg.norm(Ho)
    assert np.linalg.norm(Qp - Qo) <= polar_tol(sm) * math.sqrt(n)


@pytest.mark.parametrize("m,n,kind", [(96, 96, "dense"), (300, 40, "dense"), (700, 513, "dense"),
                                      (96, 96, "diag"), (300, 40, "diag"), (700, 513, "diag")])
def test_pd_alpha_from_norm_bound(zb, handle, m, n, kind):
    # alpha <= 0: min(||A||_F, sqrt(||A||_1 ||A||_inf)).  The Frobenius norm is the
    # smaller for the dense matrices, the Hoelder bound for the nearly diagonal ones;
    # 700 x 513 spans several 256-column chunks of the row sums and a ragged last one
    sig = 3.0 * synth.geometric_sigma(n, 1e5)
    if kind == "dense":
        A = synth.make_matrix(m, n, sig, seed=77 + n).A
    else:
        A = np.zeros((m, n))
        A[:n, :n] = np.diag(sig)
        A += 1e-7 / math.sqrt(m) * np.random.default_rng(n).standard_normal((m, n))
    fro = np.linalg.norm(A)
    holder = math.sqrt(np.abs(A).sum(axis=0).max() * np.abs(A).sum(axis=1).max())
    assert (holder < fro) == (kind == "diag")
    Qp, H, info = zb.zolo_pd(handle, dev(A), zb.opts(beta=1e-5, alpha=0.0, r=5))
    check_pd_invariants(A, host(Qp), host(H))
    alpha = zo.alpha_bound(A)
    assert alpha >= np.linalg.norm(A, 2)
    assert info.ell[0] == pytest.approx(1e-5 / alpha, rel=1e-13)


@pytest.mark.parametrize("m,n,kappa", [(256, 256, 1e8), (300, 120, 1e12), (129, 129, 10.0),
                                       (200, 33, 1e4)])
def test_beta_estimated_on_device(zb, handle, m, n, kappa):
    # beta <= 0: the library estimates beta = alpha / ||R^{-1}||_F from a QR of A/alpha;
    # the closed form is (sum_i sigma_i^{-2})^{-1/2}, between sigma_min/sqrt(n) and sigma_min
    sm = synth.make_matrix(m, n, synth.geometric_sigma(n, kappa), seed=2000 + m + n)
    alpha = float(sm.sigma.max())
    Qp, H, info = zb.zolo_pd(handle, dev(sm.A), zb.opts(beta=0.0, alpha=alpha))
    assert info.status == 0
    beta = info.ell[0] * alpha
    want = zo.beta_estimate(sm.A, alpha)
    rel = 1e-10 + 100 * EPS * kappa
    assert beta == pytest.approx(want, rel=rel)
    s = np.sort(sm.sigma)
    assert beta == pytest.approx(1.0 / math.sqrt(np.sum(s ** -2.0)), rel=rel)
    assert s[0] / math.sqrt(n) * (1 - rel) <= beta <= s[0] * (1 + rel)
    Qp, H = host(Qp), host(H)
    check_pd_invariants(sm.A, Qp, H)
    Qo, Ho, io = zo.zolo_pd(sm.A, alpha, want)
    assert info.r == io.r and info.iters == io.iters
    assert np.linalg.norm(H - Ho) <= 1e-13 * np.linalg.norm(Ho)
    assert np.linalg.norm(Qp - Qo) <= polar_tol(sm, alpha) * math.sqrt(n)


def test_beta_estimated_with_alpha_bound(zb, handle):
    sm = synth.make_matrix(160, 96, synth.geometric_sigma(96, 1e6), seed=31)
    A = 5.0 * sm.A
    Qp, H, info = zb.zolo_pd(handle, dev(A), zb.opts(beta=-1.0, alpha=0.0))
    alpha = zo.alpha_bound(A)
    assert info.ell[0] * alpha == pytest.approx(zo.beta_estimate(A, alpha), rel=1e-8)
    check_pd_invariants(A, host(Qp), host(H))


def test_posteriori_mode_matches_oracle(zb, handle):
    sm = synth.square_geometric(128, 1e12, seed=8)
    Qp, H, info = zb.zolo_pd(handle, dev(sm.A), zb.opts(beta=1e-12, r=8, posteriori=True))
    _, _, io = zo.zolo_pd(sm.A, 1.0, 1e-12, r=8, posteriori=True)
    assert info.iters == io.iters == 3 and info.used_qr == [True, False, False]
    check_pd_invariants(sm.A, host(Qp), host(H))


def test_newton_schulz_step_at_kappa_1e16(zb, handle):
    sm = synth.square_geometric(128, 1e16, seed=1000)
    Qp, H, _ = zb.zolo_pd(handle, dev(sm.A), zb.opts(beta=1e-16, r=8, ns_steps=1))
    Qo, Ho, _ = zo.zolo_pd(sm.A, 1.0, 1e-16, r=8, ns_steps=1)
    Qp, H = host(Qp), host(H)
    assert zo.orthogonality(Qp) < 1e-14
    assert zo.backward_error_pd(sm.A, Qp, H) < 1e-13
    assert np.linalg.norm(H - Ho) <= 1e-13 * np.linalg.norm(Ho)


def test_cholesky_breakdown_falls_back_to_qr(zb, handle):
    # the Cholesky form forced on kappa 1e12: Z_1 = X^T X + c_1 I with c_1 ~ 1e-23
    # is numerically indefinite; the iteration is redone in the QR form.
    sm = synth.square_geometric(128, 1e12, seed=9)
    Qp, H, info = zb.zolo_pd(handle, dev(sm.A), zb.opts(beta=1e-12, r=8, force_qr=0))
    assert info.chol_fallbacks >= 1 and info.used_qr[0]
    check_pd_invariants(sm.A, host(Qp), host(H))


def test_nonfinite_input_reported(zb, handle):
    A = synth.square_geometric(32, 10.0, seed=3).A.copy(order="F")
    A[5, 7] = np.nan
    _, _, info = zb.zolo_pd(handle, dev(A), zb.opts(beta=0.1, r=2), check=False)
    assert info.status == 1   # ZOLO_ENONFINITE


def test_user_stream_and_leading_dimensions(zb, handle):
    import torch
    sm = synth.make_matrix(70, 50, synth.geometric_sigma(50, 1e3), seed=4)
    big = torch.zeros((60, 90), dtype=torch.float64, device="cuda").t()   # 90 x 60, ld 90
    big[:70, :50] = torch.from_numpy(sm.A).cuda()
    A = big[:70, :50]
    Qb = torch.full((55, 80), 7.0, dtype=torch.float64, device="cuda").t()
    Hb = torch.full((52, 61), 7.0, dtype=torch.float64, device="cuda").t()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        zb.zolo_pd(handle, A, zb.opts(beta=1e-3, r=4), Qp=Qb[:70, :50], H=Hb[:50, :50], stream=s)
    torch.cuda.synchronize()
    Qp, H = host(Qb[:70, :50]), host(Hb[:50, :50])
    check_pd_invariants(sm.A, Qp, H)
    assert np.all(host(Qb)[70:, :] == 7.0) and np.all(host(Hb)[50:, :] == 7.0)


# ------------------------------------------------------------------ SVD

def test_svd_with_a_cluster_of_equal_singular_values(zb, handle):
    # 16 equal singular values: the eigensolver's simultaneous step meets large
    # angles there and must fall back to exact rotations; the cluster's singular
    # vectors are only defined up to a rotation, so invariants are checked
    n = 160
    sig = np.sort(np.r_[np.geomspace(1.0, 1e-6, n - 16), np.full(16, 1e-2)])[::-1].copy()
    sm = synth.make_matrix(n, n, sig, seed=1177)
    U, S, V, info = zb.zolo_svd(handle, dev(sm.A), zb.opts(beta=float(sig[-1])))
    U, S, V = host(U), host(S), host(V)
    assert np.max(np.abs(S - sm.sigma)) <= 1e-12 * sm.sigma[0]
    assert zo.svd_residual(sm.A, U, S, V) <= 1e-13 * math.sqrt(n)
    assert zo.orthogonality(U) <= 1e-13 and zo.orthogonality(V) <= 1e-13


@pytest.mark.parametrize("m,n,kappa,r", [(256, 256, 1e8, 3), (150, 90, 1e6, 0), (31, 31, 1e3, 2)])
def test_svd_matches_oracle(zb, handle, m, n, kappa, r):
    sm = synth.make_matrix(m, n, synth.geometric_sigma(n, kappa), seed=1100 + m)
    beta = float(sm.sigma[-1])
    U, S, V, info = zb.zolo_svd(handle, dev(sm.A), zb.opts(beta=beta, r=r))
    Uo, So, Vo, _ = zo.zolo_svd(sm.A, 1.0, beta, r=r)
    U, S, V = host(U), host(S), host(V)
    assert np.max(np.abs(S - So)) <= 1e-12 * So[0]
    assert np.max(np.abs(S - sm.sigma)) <= 1e-12 * sm.sigma[0]
    assert zo.svd_residual(sm.A, U, S, V) <= 1e-13 * math.sqrt(n)
    assert zo.orthogonality(U) <= 1e-13 and zo.orthogonality(V) <= 1e-13
    # singular vectors of well separated singular values agree up to sign
    gap = np.minimum(np.abs(np.diff(np.r_[np.inf, So])), np.abs(np.diff(np.r_[So, -np.inf])))
    sep = gap > 1e-3 * So[0]
    assert np.allclose(np.abs(np.sum(U * Uo, axis=0))[sep], 1.0, atol=1e-9)
    assert np.allclose(np.abs(np.sum(V * Vo, axis=0))[sep], 1.0, atol=1e-9)


@pytest.mark.parametrize("n,kappa", [(520, 1e8), (700, 1e12)])
def test_svd_past_the_row_split_of_the_fp32_sweeps(zb, handle, n, kappa):
    # from n = 512 the FP32 Jacobi sweeps give each block pair two blocks, one
    # per half of the rows (520: a ragged second half of 4 rows past a 256-row
    # chunk); checked against the singular values and vectors the matrix was
    # built from, which hold at any size
    sm = synth.make_matrix(n, n, synth.geometric_sigma(n, kappa), seed=1300 + n)
    U, S, V, info = zb.zolo_svd(handle, dev(sm.A), zb.opts(beta=float(sm.sigma[-1])))
    U, S, V = host(U), host(S), host(V)
    assert np.max(np.abs(S - sm.sigma)) <= 1e-12 * sm.sigma[0]
    assert zo.svd_residual(sm.A, U, S, V) <= 1e-13 * math.sqrt(n)
    assert zo.orthogonality(U) <= 1e-13 and zo.orthogonality(V) <= 1e-13
    # vectors of singular values separated by 1e-3 sigma_1 agree up to sign
    So = sm.sigma
    gap = np.minimum(np.abs(np.diff(np.r_[np.inf, So])), np.abs(np.diff(np.r_[So, -np.inf])))
    sep = gap > 1e-3 * So[0]
    assert sep.sum() >= 10
    assert np.allclose(np.abs(np.sum(U * sm.U, axis=0))[sep], 1.0, atol=1e-9)
    assert np.allclose(np.abs(np.sum(V * sm.V, axis=0))[sep], 1.0, atol=1e-9)


def test_host_entry_points_match_device_ones(zb, handle):
    sm = synth.square_geometric(100, 1e6, seed=5)
    o = zb.opts(beta=1e-6, r=5)
    Qd, Hd, _ = zb.zolo_pd(handle, dev(sm.A), o)
    Qh = np.zeros((100, 100), order="F")
    Hh = np.zeros((100, 100), order="F")
    zb.zolo_pd_host(handle, np.asfortranarray(sm.A), o, Qh, Hh)
    assert np.array_equal(Qh, host(Qd)) and np.array_equal(Hh, host(Hd))
    U = np.zeros((100, 100), order="F")
    V = np.zeros((100, 100), order="F")
    S = np.zeros(100)
    zb.zolo_svd_host(handle, np.asfortranarray(sm.A), o, U, S, V)
    assert np.max(np.abs(S - sm.sigma)) < 1e-12
