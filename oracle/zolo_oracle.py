"""Plain FP64 CPU oracle for Zolo-PD and Zolo-SVD (Li, Liu, Du, arxiv 1806.06204).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
baseline may import this module; the product path (the CUDA library and its
Python binding) never calls it and shares no code with it.

It restates the paper's method step by step in the paper's order and notation:

* Eq. (7)  c_i = l^2 sn^2(iK'/(2r+1); l') / cn^2(iK'/(2r+1); l'),  l' = sqrt(1-l^2)
* Eq. (8)  scaled Zolotarev function Zhat and M_hat
* Eq. (9), (10)  partial-fraction form and its weights a_j
* Eq. (12) inverse-free QR form of one iteration
* Algorithm 1 step (d): the Cholesky form of one iteration
* Algorithm 1 step (c): the update l := Zhat(l; l)
* Table 1: iterations needed for Zhat^(k)([l, 1]) to lie in [1 - 1e-15, 1]
* Algorithm 1 step 5: H = (Qp^T A + (Qp^T A)^T) / 2
* Algorithm 2: SVD from the polar decomposition and an eigendecomposition of H

Readings of passages that are garbled or silent (each is pinned by a test):

* Eq. (10) prints the two products multiplied; the partial-fraction residue is
  their quotient:  a_j = -prod_k (c_{2j-1} - c_{2k}) / prod_{k != j} (c_{2j-1} - c_{2k-1}).
* Algorithm 1 step (c) prints (l + c_{2j}) in the numerator; Eq. (8) evaluated at
  x = l gives (l^2 + c_{2j}), which is what is used.
* sn, cn take the modulus l' (parameter m = l'^2), as the integrand of K' shows.
* "L = Chol(Z)" with X L^{-1} L^{-*} is only right for the upper factor R with
  Z = R^T R; the oracle computes T_j = a_j (X R^{-1}) R^{-T}.
* The switch from the QR form to the Cholesky form is not stated for Zolo-PD; as
  in QDWH (Section 2.1, Cholesky once c_k <= 100, i.e. kappa(Z) <= 101), the
  Cholesky form is used once the bound kappa(Z_1) <= (1 + c_1)/(l^2 + c_1) is at
  most 100.
* Iterations follow the a-priori l-recurrence of Table 1; the a-posteriori test of
  Algorithm 1 step (d) adds iterations only if the last change still exceeds
  eps^(1/(2r+1)).
* The eigensolver (ELPA in the paper, Algorithm 2 step 2) is replaced by one-sided
  (Hestenes) Jacobi on the Cholesky factor of H, in the round-robin ordering
  (Golub & Van Loan, Matrix Computations, Sections 8.5.4-8.6.3): any method that
  returns H = V diag(lam) V^T is a valid step 2, and this one converges in a few
  sweeps on geometric spectra.

The elliptic functions are evaluated with the arithmetic-geometric-mean method
(Abramowitz & Stegun 16.4 and 17.6) after the Jacobi imaginary transformation
(A&S 16.20.1, sc(u | 1-m) = -i sn(iu | m)), so that no step cancels when l is
tiny.  Nothing here is blocked, fused or reordered beyond what the paper states;
numpy's matrix product is the only library step.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

EPS = float(np.finfo(np.float64).eps)      # 2^-52
TABLE1_TOL = 1e-15                        # Table 1: Zhat^(k)([l,1]) in [1 - 1e-15, 1]


# ---------------------------------------------------------------------------
# Elliptic integral and Jacobi functions (A&S 16.4, 16.20.1, 17.6)
# ---------------------------------------------------------------------------

def agm(a: float, b: float) -> float:
    """Arithmetic-geometric mean of a, b > 0."""
    for _ in range(200):
        if abs(a - b) <= 2.0 * EPS * a:
            break
        a, b = 0.5 * (a + b), math.sqrt(a * b)
    return 0.5 * (a + b)


def K_complement(ell: float) -> float:
    """K' = K(l') for the modulus l' = sqrt(1 - l^2): pi / (2 AGM(1, l)) (A&S 17.6)."""
    return math.pi / (2.0 * agm(1.0, ell))


def _asinh_x_sinh(x: float, psi: float) -> float:
    """asinh(x * sinh(psi)) for x > 0, psi >= 0, without overflow for large psi."""
    if psi < 30.0:
        return math.asinh(x * math.sinh(psi))
    # ln(x sinh psi) = ln x + psi - ln 2 + log1p(-e^{-2 psi});  asinh(y) = ln(2y) + ln((1 + sqrt(1 + y^-2))/2)
    log_y = math.log(x) + psi - math.log(2.0) + math.log1p(-math.exp(-2.0 * psi))
    inv_y2 = math.exp(-2.0 * log_y) if log_y < 300.0 else 0.0
    return math.log(2.0) + log_y + math.log(0.5 * (1.0 + math.sqrt(1.0 + inv_y2)))


def sc_complement(u: float, ell: float) -> float:
    """sc(u; l') = sn/cn at modulus l' = sqrt(1 - l^2), for 0 <= u <= K'/2.

    (The truncated AGM recurrence below grows like exp(2 psi) and loses accuracy
    past the half period; larger arguments go through the reflection in
    `c_coefficient`.)

    Imaginary transformation: sc(u; l') = -i sn(iu; l).  sn at modulus l by the
    AGM scale a_0 = 1, b_0 = l', c_0 = l (A&S 16.4).  With the phase phi_n = i psi_n
    the backward recurrence stays real:
        psi_N = 2^N a_N u,   psi_{n-1} = (psi_n + asinh((c_n / a_n) sinh psi_n)) / 2,
    and sc = sinh(psi_0).
    """
    ellp = math.sqrt((1.0 - ell) * (1.0 + ell))
    if ellp == 0.0:                      # l = 1: modulus 0, sc = tan
        return math.tan(u)
    a, b, c = 1.0, ellp, ell
    an, cn = [a], [c]
    for _ in range(60):
        if c <= EPS * a:
            break
        a_next = 0.5 * (a + b)
        b = math.sqrt(a * b)
        c = c * c / (4.0 * a_next)       # = (a - b)/2 without cancellation
        a = a_next
        an.append(a)
        cn.append(c)
    N = len(an) - 1
    psi = (2.0 ** N) * an[N] * u
    for n in range(N, 0, -1):
        psi = 0.5 * (psi + _asinh_x_sinh(cn[n] / an[n], psi))
    return math.sinh(psi)


# ---------------------------------------------------------------------------
# Zolotarev coefficients, Eqs. (7), (8), (10)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Coeffs:
    ell: float
    r: int
    c: np.ndarray      # c_1 .. c_{2r}   (c[i-1] = c_i)
    a: np.ndarray      # a_1 .. a_r
    Mhat: float


def c_coefficient(i: int, r: int, ell: float, Kp: float) -> float:
    """c_i of Eq. (7) at u_i = i K'/(2r+1).

    For u_i <= K'/2 directly: c_i = l^2 sc^2(u_i; l').  Beyond it, the quarter-period
    reflection sc(K' - v; l') = 1 / (l sc(v; l')) (A&S 16.8) with v = K' - u_i gives
    c_i = 1 / sc^2(v; l'), so every evaluation has an argument of at most K'/2."""
    if 2 * i <= 2 * r + 1:
        u = i * Kp / (2 * r + 1)
        return ell * ell * sc_complement(u, ell) ** 2
    v = (2 * r + 1 - i) * Kp / (2 * r + 1)
    return 1.0 / sc_complement(v, ell) ** 2


def zolotarev_coeffs(ell: float, r: int) -> Coeffs:
    """c_i (Eq. 7), M_hat (Eq. 8) and a_j (Eq. 10, read as a quotient)."""
    assert 0.0 < ell <= 1.0 and r >= 1
    Kp = K_complement(ell)
    c = np.array([c_coefficient(i, r, ell, Kp) for i in range(1, 2 * r + 1)])
    c_odd = c[0::2]        # c_1, c_3, ..., c_{2r-1}
    c_even = c[1::2]       # c_2, c_4, ..., c_{2r}
    Mhat = float(np.prod((1.0 + c_odd) / (1.0 + c_even)))
    a = np.empty(r)
    for j in range(r):
        num = np.prod(c_odd[j] - c_even)
        den = np.prod([c_odd[j] - c_odd[k] for k in range(r) if k != j])
        a[j] = -num / den
    return Coeffs(ell=ell, r=r, c=c, a=a, Mhat=Mhat)


def zhat(x, co: Coeffs):
    """Product form, Eq. (8): M_hat x prod_j (x^2 + c_{2j}) / (x^2 + c_{2j-1})."""
    x = np.asarray(x, dtype=np.float64)
    out = co.Mhat * x
    for j in range(co.r):
        out = out * (x * x + co.c[2 * j + 1]) / (x * x + co.c[2 * j])
    return out


def zhat_partial_fraction(x, co: Coeffs):
    """Partial-fraction form, Eq. (9): M_hat x (1 + sum_j a_j / (x^2 + c_{2j-1}))."""
    x = np.asarray(x, dtype=np.float64)
    s = np.ones_like(x)
    for j in range(co.r):
        s = s + co.a[j] / (x * x + co.c[2 * j])
    return co.Mhat * x * s


def one_minus_zhat_at_ell(co: Coeffs) -> float:
    """1 - Zhat(l; l), the gap that Table 1 compares with 1e-15, without cancellation.

    On [l, 1], Zhat <= 1 touches 1 at x = 1 and at r interior maxima
    xi_m = l / dn((2m-1)K'/(2r+1); l'), which by Eq. (7) is
    xi_m^2 = (l^2 + c_{2m-1}) / (1 + c_{2m-1}).  The numerator of 1 - Zhat(x)
    (Eq. (8) over a common denominator, degree 2r+1, leading coefficient -M_hat)
    therefore factors as M_hat (1 - x) prod_m (x - xi_m)^2, and
        1 - Zhat(l) = M_hat (1 - l) prod_m (xi_m - l)^2 / prod_m (l^2 + c_{2m-1}),
    with xi_m - l = c_{2m-1} l'^2 / ((1 + c_{2m-1})(xi_m + l)): every factor positive."""
    ell = co.ell
    lp2 = (1.0 - ell) * (1.0 + ell)
    gap = co.Mhat * (1.0 - ell)
    for m in range(co.r):
        c_odd = co.c[2 * m]
        xi = math.sqrt((ell * ell + c_odd) / (1.0 + c_odd))
        diff = c_odd * lp2 / ((1.0 + c_odd) * (xi + ell))
        gap *= diff * diff / (ell * ell + c_odd)
    return gap


def next_ell(ell: float, r: int) -> float:
    """Algorithm 1 step (c): l := Zhat(l; l) (the value Eq. (8) takes at x = l)."""
    return 1.0 - one_minus_zhat_at_ell(zolotarev_coeffs(ell, r))


def ell_schedule(ell0: float, r: int, tol: float = TABLE1_TOL, max_iter: int = 50):
    """l_0, l_1, ..., l_K with K the first k such that 1 - l_k <= tol (Table 1)."""
    ells = [float(ell0)]
    gap = 1.0 - float(ell0)
    while gap > tol and len(ells) <= max_iter:
        gap = one_minus_zhat_at_ell(zolotarev_coeffs(ells[-1], r))
        ells.append(1.0 - gap)
    return ells


def iterations_needed(kappa: float, r: int) -> int:
    """One entry of Table 1: iterations for l_0 = 1/kappa."""
    return len(ell_schedule(1.0 / kappa, r)) - 1


def choose_r(ell0: float, max_r: int = 8) -> int:
    """Smallest r <= 8 needing at most two iterations (Section 2.2, after Table 1)."""
    for r in range(1, max_r + 1):
        if len(ell_schedule(ell0, r)) - 1 <= 2:
            return r
    return max_r


def uses_qr(co: Coeffs, ell: float, limit: float = 100.0) -> bool:
    """QR form unless the bound kappa(Z_1) <= (1 + c_1)/(l^2 + c_1) is at most `limit`."""
    c1 = co.c[0]
    return (1.0 + c1) / (ell * ell + c1) > limit


def dwh_closed_form(ell: float):
    """QDWH weights (a, b, c) of the dynamically weighted Halley step, Eq. (2),
    in the closed form of Nakatsukasa, Bai and Gygi (SIMAX 2010)."""
    g = (4.0 * (1.0 - ell * ell) / ell ** 4) ** (1.0 / 3.0)
    a = math.sqrt(1.0 + g) + 0.5 * math.sqrt(
        8.0 - 4.0 * g + 8.0 * (2.0 - ell * ell) / (ell * ell * math.sqrt(1.0 + g)))
    b = (a - 1.0) ** 2 / 4.0
    c = a + b - 1.0
    return a, b, c


# ---------------------------------------------------------------------------
# Dense Householder QR, Cholesky, triangular solves (unblocked textbook forms)
# ---------------------------------------------------------------------------

def householder_vector(x: np.ndarray):
    """v (v[0] = 1), tau, beta with (I - tau v v^T) x = beta e_1."""
    alpha = x[0]
    xnorm = np.linalg.norm(x[1:])
    v = x.copy()
    v[0] = 1.0
    if xnorm == 0.0:
        v[1:] = 0.0
        return v, 0.0, alpha
    beta = -math.copysign(math.hypot(alpha, xnorm), alpha)
    tau = (beta - alpha) / beta
    v[1:] = x[1:] / (alpha - beta)
    return v, tau, beta


def householder_qr(W: np.ndarray):
    """Unblocked Householder QR of a dense p x n matrix W (p >= n).

    Returns the reflectors (list of (v, tau) acting on rows k..p-1) and R."""
    W = np.array(W, dtype=np.float64, copy=True)
    p, n = W.shape
    refl = []
    for k in range(n):
        v, tau, beta = householder_vector(W[k:, k])
        if tau != 0.0:
            w = v @ W[k:, k:]
            W[k:, k:] -= tau * np.outer(v, w)
        W[k, k] = beta
        W[k + 1:, k] = 0.0
        refl.append((v, tau))
    return refl, np.triu(W[:n, :])


def thin_q(refl, p: int, n: int) -> np.ndarray:
    """Explicit thin Q = H_0 H_1 ... H_{n-1} [I_n; 0] (p x n)."""
    Q = np.zeros((p, n))
    Q[:n, :n] = np.eye(n)
    for k in range(n - 1, -1, -1):
        v, tau = refl[k]
        if tau != 0.0:
            w = v @ Q[k:, k:]
            Q[k:, k:] -= tau * np.outer(v, w)
    return Q


def alpha_bound(A: np.ndarray) -> float:
    """An upper bound of sigma_max(A) when none is given (Algorithm 1 step 1 takes
    alpha >= ||A||_2 as known): the smaller of ||A||_F and sqrt(||A||_1 ||A||_inf),
    both >= ||A||_2 (the second since ||A||_2^2 = ||A^T A||_2 <= ||A^T||_1 ||A||_1)."""
    A = np.asarray(A, dtype=np.float64)
    fro = math.sqrt(float(np.sum(A * A)))
    one = float(np.max(np.sum(np.abs(A), axis=0)))
    inf = float(np.max(np.sum(np.abs(A), axis=1)))
    return min(fro, math.sqrt(one) * math.sqrt(inf))


def beta_estimate(A: np.ndarray, alpha: float) -> float:
    """A lower bound of sigma_min(A) from the triangular factor of X0 = A / alpha.

    Not in the paper (its Section 3.2 takes alpha and beta as known).  With
    X0 = Q R, sigma_min(X0) = 1 / ||R^{-1}||_2 >= 1 / ||R^{-1}||_F, so
    beta = alpha / ||R^{-1}||_F <= sigma_min(A), loose by at most sqrt(n)."""
    _, R = householder_qr(np.asarray(A, dtype=np.float64) / alpha)
    Rinv = solve_right_upper(np.eye(R.shape[0]), R)
    return float(alpha / np.linalg.norm(Rinv))


def cholesky_upper(Z: np.ndarray) -> np.ndarray:
    """Upper R with Z = R^T R (unblocked); raises on a non-positive pivot."""
    n = Z.shape[0]
    R = np.zeros_like(Z)
    for j in range(n):
        s = Z[j, j] - R[:j, j] @ R[:j, j]
        if not s > 0.0:
            raise np.linalg.LinAlgError(f"Cholesky breakdown at column {j}")
        R[j, j] = math.sqrt(s)
        R[j, j + 1:] = (Z[j, j + 1:] - R[:j, j] @ R[:j, j + 1:]) / R[j, j]
    return R


def solve_right_upper(X: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Y = X R^{-1} for upper-triangular R, column by column (Y R = X)."""
    n = R.shape[0]
    Y = np.zeros_like(X)
    for j in range(n):
        Y[:, j] = (X[:, j] - Y[:, :j] @ R[:j, j]) / R[j, j]
    return Y


def solve_right_upper_transpose(Y: np.ndarray, R: np.ndarray) -> np.ndarray:
    """W = Y R^{-T} for upper-triangular R (W R^T = Y), last column first."""
    n = R.shape[0]
    W = np.zeros_like(Y)
    for j in range(n - 1, -1, -1):
        W[:, j] = (Y[:, j] - W[:, j + 1:] @ R[j, j + 1:]) / R[j, j]
    return W


# ---------------------------------------------------------------------------
# One Zolo-PD iteration: Eq. (12) (QR form) and Algorithm 1 step (d) (Cholesky)
# ---------------------------------------------------------------------------

def zolo_step_qr(X: np.ndarray, co: Coeffs) -> np.ndarray:
    """X_new = M_hat (X + sum_j a_j / sqrt(c_{2j-1}) Q_{j1} Q_{j2}^T), Eq. (12).

    Each [X; sqrt(c_{2j-1}) I] is factored densely (deliberately not structured)."""
    m, n = X.shape
    S = np.zeros_like(X)
    for j in range(co.r):
        c_odd = co.c[2 * j]
        W = np.vstack([X, math.sqrt(c_odd) * np.eye(n)])
        refl, _ = householder_qr(W)
        Q = thin_q(refl, m + n, n)
        Q1, Q2 = Q[:m], Q[m:]
        S += (co.a[j] / math.sqrt(c_odd)) * (Q1 @ Q2.T)
    return co.Mhat * (X + S)


def zolo_step_chol(X: np.ndarray, co: Coeffs) -> np.ndarray:
    """X_new = M_hat (X + sum_j a_j (X R_j^{-1}) R_j^{-T}), Z_j = X^T X + c_{2j-1} I = R_j^T R_j."""
    n = X.shape[1]
    G = X.T @ X
    S = np.zeros_like(X)
    for j in range(co.r):
        Z = G + co.c[2 * j] * np.eye(n)
        R = cholesky_upper(Z)
        Y = solve_right_upper(X, R)
        S += co.a[j] * solve_right_upper_transpose(Y, R)
    return co.Mhat * (X + S)


def group_terms(X: np.ndarray, co: Coeffs, shifts, qr: bool) -> np.ndarray:
    """Algorithm 3 step 4(c): the process groups j in `shifts` each factor their
    own shifted problem and form T_j (Eq. 12 in the QR form, Algorithm 1 step
    (d) in the Cholesky form); returns the sum of those T_j, which step 4(d)
    (DGSUM2D) adds across all groups before X_{k+1} = M_hat (X + sum_j T_j)."""
    m, n = X.shape
    S = np.zeros_like(X)
    G = None if qr else X.T @ X
    for j in shifts:
        c_odd = co.c[2 * j]
        if qr:
            W = np.vstack([X, math.sqrt(c_odd) * np.eye(n)])
            refl, _ = householder_qr(W)
            Q = thin_q(refl, m + n, n)
            S += (co.a[j] / math.sqrt(c_odd)) * (Q[:m] @ Q[m:].T)
        else:
            R = cholesky_upper(G + c_odd * np.eye(n))
            S += co.a[j] * solve_right_upper_transpose(solve_right_upper(X, R), R)
    return S


def newton_schulz_step(X: np.ndarray) -> np.ndarray:
    """X <- 1.5 X - 0.5 X (X^T X): one Newton-Schulz polar refinement step."""
    return 1.5 * X - 0.5 * (X @ (X.T @ X))


@dataclasses.dataclass
class PDInfo:
    r: int
    iters: int
    ells: list
    used_qr: list
    delta: list
    extra_iters: int


def zolo_pd(A: np.ndarray, alpha: float, beta: float, r: int = 0, max_iter: int = 6,
            ns_steps: int = 0, posteriori: bool = False):
    """Algorithm 1: Q_p, H with A = Q_p H.  alpha >= sigma_max(A), beta <= sigma_min(A).

    The iteration count is the a-priori one of Table 1 (1 - l_K <= 1e-15).  With
    `posteriori`, the test of Algorithm 1 step (d) is applied literally after it:
    while the last relative change exceeds eps^(1/(2r+1)), one more (Cholesky)
    iteration runs, up to max_iter in total.  Returns (Qp, H, PDInfo)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    assert m >= n and alpha > 0.0 and 0.0 < beta <= alpha
    X = A / alpha                                     # step 1
    ell = beta / alpha                                # step 2 (l_0 from bounds on A)
    if r == 0:
        r = choose_r(ell)                             # step 3
    ells = ell_schedule(ell, r)
    K = min(len(ells) - 1, max_iter)
    used_qr, delta = [], []
    for k in range(K):                                # step 4, one pass per l_k
        co = zolotarev_coeffs(ells[k], r)
        qr = uses_qr(co, ells[k])
        Xn = zolo_step_qr(X, co) if qr else zolo_step_chol(X, co)
        delta.append(float(np.linalg.norm(Xn - X) / np.linalg.norm(Xn)))
        used_qr.append(qr)
        X = Xn
    extra = 0
    ell_k = ells[K] if K < len(ells) else ells[-1]
    # Algorithm 1 step (d): verify ||X_2 - X_1||_F / ||X_2||_F <= eps^(1/(2r+1)).
    while posteriori and delta and delta[-1] > EPS ** (1.0 / (2 * r + 1)) and len(delta) < max_iter:
        co = zolotarev_coeffs(ell_k, r)
        Xn = zolo_step_chol(X, co)
        delta.append(float(np.linalg.norm(Xn - X) / np.linalg.norm(Xn)))
        used_qr.append(False)
        ell_k = 1.0 - one_minus_zhat_at_ell(co)
        ells.append(ell_k)
        X = Xn
        extra += 1
    for _ in range(ns_steps):
        X = newton_schulz_step(X)
    Qp = X
    M = Qp.T @ A                                      # step 5
    H = 0.5 * (M + M.T)
    info = PDInfo(r=r, iters=len(delta), ells=ells[:len(delta) + 1], used_qr=used_qr,
                  delta=delta, extra_iters=extra)
    return Qp, H, info


# ---------------------------------------------------------------------------
# Eigendecomposition of H and Zolo-SVD (Algorithm 2)
# ---------------------------------------------------------------------------

def _round_robin_pairs(n: int):
    """Rounds of the round-robin (tournament) ordering over indices 0..n-1 (n even)."""
    idx = list(range(n))
    rounds = []
    for _ in range(n - 1):
        rounds.append([(idx[i], idx[n - 1 - i]) for i in range(n // 2)])
        idx = [idx[0]] + [idx[-1]] + idx[1:-1]
    return rounds


def hestenes_columns(X: np.ndarray, max_sweeps: int = 40):
    """One-sided (Hestenes) Jacobi: right rotations X <- X J until the columns are
    mutually orthogonal, |x_p . x_q| <= eps ||x_p|| ||x_q|| for every pair.

    Rotations follow the round-robin ordering; each round applies n/2 disjoint
    rotations at once.  Returns (X with orthogonal columns, sweeps used)."""
    X = np.array(X, dtype=np.float64, copy=True)
    n0 = X.shape[1]
    n = n0 + (n0 % 2)
    if n != n0:                                       # a zero column never rotates
        X = np.hstack([X, np.zeros((X.shape[0], 1))])
    rounds = _round_robin_pairs(n)
    sweeps = 0
    for sweeps in range(1, max_sweeps + 1):
        rotated = False
        for pairs in rounds:
            P = np.array([p for p, q in pairs])
            Q = np.array([q for p, q in pairs])
            al = np.einsum("ij,ij->j", X[:, P], X[:, P])
            be = np.einsum("ij,ij->j", X[:, Q], X[:, Q])
            ga = np.einsum("ij,ij->j", X[:, P], X[:, Q])
            rot = np.abs(ga) > EPS * np.sqrt(al * be)
            if not rot.any():
                continue
            rotated = True
            zeta = np.where(rot, (be - al) / np.where(rot, 2.0 * ga, 1.0), 0.0)
            t = np.where(rot, np.where(zeta >= 0, 1.0, -1.0)
                         / (np.abs(zeta) + np.sqrt(1.0 + zeta * zeta)), 0.0)
            cs = 1.0 / np.sqrt(1.0 + t * t)
            sn = cs * t
            XP, XQ = X[:, P].copy(), X[:, Q].copy()
            X[:, P] = cs * XP - sn * XQ
            X[:, Q] = sn * XP + cs * XQ
        if not rotated:
            break
    return X[:, :n0], sweeps


def jacobi_eigh(H: np.ndarray, max_sweeps: int = 40):
    """Eigendecomposition of a symmetric positive (semi)definite H.

    H = R^T R (Cholesky, upper R); one-sided Jacobi on R^T gives R^T Z = W diag(s)
    with orthonormal W, so H = R^T R = W diag(s^2) W^T: the eigenvectors are the
    normalised columns.  The eigenvalues are taken as the Rayleigh quotients
    lam_i = w_i^T H w_i of those columns (the squared column norms carry the
    rounding of every rotation the column went through).  (Two-sided
    Jacobi on H itself converges only linearly in the absolute off-diagonal norm
    when the spectrum is geometric over many decades; the Cholesky factor is the
    preconditioner that restores quadratic convergence.)  If the factorisation
    breaks down (eigenvalues at rounding level), H + s I with s = 10 n eps ||H||_F is
    factored instead; it has the same eigenvectors.
    Returns (eigenvalues, V) unsorted, with H ~= V diag(lam) V^T."""
    H = 0.5 * (np.asarray(H, dtype=np.float64) + np.asarray(H, dtype=np.float64).T)
    n = H.shape[0]
    shift = 0.0
    try:
        R = cholesky_upper(H)
    except np.linalg.LinAlgError:
        shift = 10.0 * n * EPS * np.linalg.norm(H)
        R = cholesky_upper(H + shift * np.eye(n))
    X, _ = hestenes_columns(R.T, max_sweeps)
    s = np.linalg.norm(X, axis=0)
    V = X / np.where(s > 0, s, 1.0)
    lam = np.einsum("ij,ij->j", V, H @ V)
    return lam, V


def zolo_svd(A: np.ndarray, alpha: float, beta: float, r: int = 0, max_iter: int = 6,
             ns_steps: int = 0, posteriori: bool = False):
    """Algorithm 2: A = U diag(S) V^T via Zolo-PD and an eigendecomposition of H.

    Singular values descending; a negative eigenvalue (rounding) gives sigma = |lam|
    with the sign of the matching column of U flipped."""
    Qp, H, info = zolo_pd(A, alpha, beta, r=r, max_iter=max_iter, ns_steps=ns_steps,
                          posteriori=posteriori)
    lam, V = jacobi_eigh(H)
    order = np.argsort(-lam)
    lam, V = lam[order], V[:, order]
    U = Qp @ V
    neg = lam < 0.0
    U[:, neg] *= -1.0
    S = np.abs(lam)
    order = np.argsort(-S, kind="stable")
    return U[:, order], S[order], V[:, order], info


def one_sided_jacobi_svd(A: np.ndarray, max_sweeps: int = 60):
    """Brute-force SVD of a small matrix by one-sided (Hestenes) Jacobi rotations.

    Returns (U, S, V) with S descending."""
    Uw = np.array(A, dtype=np.float64, copy=True)
    m, n = Uw.shape
    V = np.eye(n)
    for _ in range(max_sweeps):
        rotated = False
        for p in range(n - 1):
            for q in range(p + 1, n):
                al = Uw[:, p] @ Uw[:, p]
                be = Uw[:, q] @ Uw[:, q]
                ga = Uw[:, p] @ Uw[:, q]
                if abs(ga) <= EPS * math.sqrt(al * be) or ga == 0.0:
                    continue
                rotated = True
                zeta = (be - al) / (2.0 * ga)
                t = math.copysign(1.0, zeta) / (abs(zeta) + math.sqrt(1.0 + zeta * zeta))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = c * t
                up, uq = Uw[:, p].copy(), Uw[:, q].copy()
                Uw[:, p], Uw[:, q] = c * up - s * uq, s * up + c * uq
                vp, vq = V[:, p].copy(), V[:, q].copy()
                V[:, p], V[:, q] = c * vp - s * vq, s * vp + c * vq
        if not rotated:
            break
    S = np.linalg.norm(Uw, axis=0)
    order = np.argsort(-S)
    S, Uw, V = S[order], Uw[:, order], V[:, order]
    U = Uw / np.where(S > 0, S, 1.0)
    return U, S, V


# ---------------------------------------------------------------------------
# Accuracy measures (Section 4.4, Eq. (13)) and the contract's normalisations
# ---------------------------------------------------------------------------

def backward_error_pd(A, Qp, H) -> float:
    """||A - Qp H||_F / ||A||_F."""
    return float(np.linalg.norm(A - Qp @ H) / np.linalg.norm(A))


def orthogonality(Q) -> float:
    """||Q^T Q - I||_F / sqrt(n)."""
    n = Q.shape[1]
    return float(np.linalg.norm(Q.T @ Q - np.eye(n)) / math.sqrt(n))


def svd_residual(A, U, S, V) -> float:
    """Res of Eq. (13): ||A - U Sigma V^T||_F / ||A||_2."""
    return float(np.linalg.norm(A - (U * S) @ V.T) / np.linalg.norm(A, 2))


def orth_paper(Q) -> float:
    """OrthL / OrthR of Section 4.4: ||I - Q Q^T||_F / n, for square Q."""
    n = Q.shape[1]
    return float(np.linalg.norm(np.eye(Q.shape[0]) - Q @ Q.T) / n)
