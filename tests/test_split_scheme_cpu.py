"""A numpy model of the split-precision product's arithmetic (no GPU).

The tensor-core path writes every FP64 row of op(A) / column of op(B), scaled by
its power of two 2^e into (-1/2, 1/2), as the integer N = round(x 2^(6S - e)) in
S balanced base-64 digits (|d_s| <= 32), and sums the digit-pair products of
levels s + t <= S + 2.  This model does the same in exact integer arithmetic and
checks the claims the design rests on: the error bound, a small multiple of
sqrt(K) 2^-6S max|A_i| max|B_j| (the rounding of N, relative to a row maximum in
[1/4, 1/2), dominates it), FP64 grade at S = 9, the gain from keeping level S + 2, the bias that
truncated digits put on a Gram diagonal and balanced ones do not, and that a
level's partial sums over a 2048-long chunk stay exact in FP32.
"""
import math

import numpy as np
import pytest

BETA = 6


def exponents(X, axis):
    """e with max |x| 2^-e in [1/4, 1/2) along the given axis (0 for zero rows)."""
    mx = np.max(np.abs(X), axis=axis)
    e = np.zeros(mx.shape, dtype=np.int64)
    nz = mx > 0
    e[nz] = np.frexp(mx[nz])[1] + 1          # mx = f 2^E, f in [1/2, 1): mx 2^-(E+1) in [1/4, 1/2)
    return e


def digits(X, e, S, balanced=True):
    """Integer digits d[s] (s = 0..S-1, most significant first) of X 2^-e on S base-64 places."""
    N = np.vectorize(int, otypes=[object])(np.rint(np.ldexp(X, (BETA * S - e))))  # exact ints
    out = []
    for _ in range(S - 1):
        d = np.vectorize(lambda v: ((v + 32) % 64) - 32 if balanced else v % 64, otypes=[object])(N)
        out.append(d)
        N = (N - d) // 64
    out.append(N)
    return out[::-1]


def split_product(A, B, S, max_level, balanced=True):
    ea = exponents(A, axis=1)                 # rows of A
    eb = exponents(B, axis=0)                 # columns of B
    da = digits(A, ea[:, None], S, balanced)
    db = digits(B, eb[None, :], S, balanced)
    acc = np.zeros((A.shape[0], B.shape[1]), dtype=object)
    for s in range(S):
        for t in range(S):
            if (s + 1) + (t + 1) > max_level:
                continue
            acc += (da[s].dot(db[t])) * (2 ** (BETA * (2 * S - (s + 1) - (t + 1))))
    # value = acc 2^-(12S) 2^(ea + eb)
    C = np.empty(acc.shape)
    for i in range(acc.shape[0]):
        for j in range(acc.shape[1]):
            C[i, j] = math.ldexp(float(acc[i, j]), int(ea[i] + eb[j]) - 2 * BETA * S)
    return C


def exact_product(A, B):
    return (A.astype(np.longdouble) @ B.astype(np.longdouble)).astype(np.float64)


@pytest.fixture(scope="module")
def operands():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((12, 300)) * np.exp(rng.uniform(-8, 8, (12, 1)))
    B = rng.standard_normal((300, 10)) * np.exp(rng.uniform(-8, 8, (1, 10)))
    return A, B


def test_nine_slices_are_fp64_grade(operands):
    A, B = operands
    S, K = 9, A.shape[1]
    C = split_product(A, B, S, S + 2)
    ref = exact_product(A, B)
    scale = np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(B), axis=0)[None, :]
    err = np.max(np.abs(C - ref) / scale)
    assert err <= 8 * math.sqrt(K) * 2.0 ** (-BETA * S)
    assert err <= 2e-16 * math.sqrt(K)


def test_keeping_level_s_plus_2_cuts_the_error(operands):
    A, B = operands
    S = 9
    ref = exact_product(A, B)
    scale = np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(B), axis=0)[None, :]
    e_keep = np.max(np.abs(split_product(A, B, S, S + 2) - ref) / scale)
    e_drop = np.max(np.abs(split_product(A, B, S, S + 1) - ref) / scale)
    assert e_drop > 4 * e_keep


def test_balanced_digits_leave_no_bias_on_a_gram_diagonal():
    # the dropped pairs of a truncated (non-negative) digit expansion all push
    # x^T x the same way; balanced digits make them zero-mean
    rng = np.random.default_rng(12)
    x = rng.uniform(0.25, 0.5, (1, 4000))
    S, lvl = 4, 4 + 1           # coarse enough that the dropped pairs, not the rounding, dominate
    ref = float(exact_product(x, x.T)[0, 0])
    bal = split_product(x, x.T, S, lvl, balanced=True)[0, 0]
    tru = split_product(x, x.T, S, lvl, balanced=False)[0, 0]
    assert abs(tru - ref) > 5 * abs(bal - ref)


def test_level_sums_are_exact_in_fp32_over_a_chunk():
    # a level of p pairs (p <= 7 for levels 2..8, each in its own TMEM accumulator)
    # of |d_s d_t| <= 2^10 over 2048 terms stays within FP32's 24-bit integer range
    for level in range(2, 9):
        p = level - 1
        assert p * 2048 * 2 ** 10 <= 2 ** 24
    # and the digits' bound itself: |d| <= 32 for every digit of the model
    rng = np.random.default_rng(13)
    X = rng.standard_normal((5, 64)) * 10.0 ** rng.uniform(-20, 20, (5, 1))
    for d in digits(X, exponents(X, axis=1)[:, None], 9):
        assert max(abs(int(v)) for v in d.ravel()) <= 32


# ---- the FP16 form: FP16's exponent range (down to 2^-24) cannot hold a digit
# pre-scaled by 2^-7s, so its slices are the raw base-128 digits (|d| <= 64,
# exact in FP16), every level L = s + t keeps its own accumulator, and the
# scale 2^-7L is applied when the levels are joined: levels 2..7 as an int64 in
# units of 2^-49, levels 8 and 9 into one FP32 in units of 2^-56.  S = 8 slices
# (56 bits), levels <= S + 1 (36 slice pairs), K-chunks of 512.

def digits_base(X, e, S, beta):
    N = np.vectorize(int, otypes=[object])(np.rint(np.ldexp(X, (beta * S - e))))
    half, full = 2 ** (beta - 1), 2 ** beta
    out = []
    for _ in range(S - 1):
        d = np.vectorize(lambda v: ((v + half) % full) - half, otypes=[object])(N)
        out.append(d)
        N = (N - d) // full
    out.append(N)
    return out[::-1]


def split_product_fp16(A, B, S=8, max_level=9, chunk=512):
    """The FP16 form's arithmetic: per-chunk exact level sums, joined as the kernel
    joins them (levels 2..7 in an int64 of 2^-49 units, 8 and 9 in one FP32 of
    2^-56 units, accumulated over the chunks in FP32)."""
    beta = 7
    ea = exponents(A, axis=1)
    eb = exponents(B, axis=0)
    da = digits_base(A, ea[:, None], S, beta)
    db = digits_base(B, eb[None, :], S, beta)
    M, N, K = A.shape[0], B.shape[1], A.shape[1]
    iacc = np.zeros((M, N), dtype=object)
    fm = np.zeros((M, N), dtype=np.float32)
    for k0 in range(0, K, chunk):
        ks = slice(k0, min(K, k0 + chunk))
        for L in range(2, max_level + 1):
            lv = np.zeros((M, N), dtype=object)
            for s in range(1, S + 1):
                t = L - s
                if 1 <= t <= S:
                    lv = lv + da[s - 1][:, ks].dot(db[t - 1][ks, :])
            # the accumulator holds an integer: exact in FP32 while |lv| <= 2^24
            assert max(abs(int(v)) for v in lv.ravel()) <= 2 ** 24
            if L <= 7:
                iacc = iacc + lv * (2 ** (49 - 7 * L))
            else:   # the accumulator's FP32 integer, times 2^-7 for level 9, added in FP32
                v = np.vectorize(float)(lv).astype(np.float32)
                fm = (fm + (v if L == 8 else v * np.float32(2.0 ** -7))).astype(np.float32)
    assert max(abs(int(v)) for v in iacc.ravel()) < 2 ** 63
    C = np.empty((M, N))
    for i in range(M):
        for j in range(N):
            v = float(iacc[i, j]) + float(fm[i, j]) * 2.0 ** -7
            C[i, j] = math.ldexp(v, int(ea[i] + eb[j]) - 49)
    return C


def test_fp16_form_is_fp64_grade(operands):
    A, B = operands
    K = A.shape[1]
    C = split_product_fp16(A, B)
    ref = exact_product(A, B)
    scale = np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(B), axis=0)[None, :]
    err = np.max(np.abs(C - ref) / scale)
    # same grade as the BF16 form's bound (8 sqrt(K) 2^-54)
    assert err <= 8 * math.sqrt(K) * 2.0 ** -54
    assert err <= 2e-16 * math.sqrt(K)


def test_fp16_form_level_sums_exact_over_a_512_chunk():
    # |d| <= 64: a level of p <= 8 pairs over 512 terms stays within 2^24
    for level in range(2, 10):
        p = min(level - 1, 8, 17 - level)
        assert p * 512 * 64 * 64 <= 2 ** 24
    rng = np.random.default_rng(14)
    X = rng.standard_normal((5, 64)) * 10.0 ** rng.uniform(-20, 20, (5, 1))
    for d in digits_base(X, exponents(X, axis=1)[:, None], 8, 7):
        assert max(abs(int(v)) for v in d.ravel()) <= 64
    # the worst case of the model's own accumulators (checked inside) with operands
    # at the digit bound over a whole chunk
    A = np.full((2, 512), 0.4999)
    B = np.full((512, 2), -0.4999)
    C = split_product_fp16(A, B)
    assert abs(C[0, 0] - exact_product(A, B)[0, 0]) <= 512 * 2.0 ** -52


def test_fp16_form_without_level_9_is_worse(operands):
    A, B = operands
    ref = exact_product(A, B)
    scale = np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(B), axis=0)[None, :]
    keep = np.max(np.abs(split_product_fp16(A, B, max_level=9) - ref) / scale)
    drop = np.max(np.abs(split_product_fp16(A, B, max_level=8) - ref) / scale)
    assert drop > 4 * keep


# ---- the FP8 (E4M3) form: E4M3 holds every integer |d| <= 16 exactly but nothing
# pre-scaled below 2^-9, so its slices are raw balanced base-32 digits
# (|d| <= 16), S = 11 slices (55 bits), levels L = s + t <= S + 2 = 13 (76 slice
# pairs), one accumulator per level, K-chunks of 4096; the epilogue adds levels
# 2..9 to an int64 of 2^-48 units and levels 10..13 to one FP32 of 2^-65 units,
# joined as iacc + f 2^-17.

def split_product_fp8(A, B, S=11, max_level=13, chunk=4096):
    """The FP8 form's arithmetic, joined as the kernel joins it."""
    beta = 5
    ea = exponents(A, axis=1)
    eb = exponents(B, axis=0)
    da = digits_base(A, ea[:, None], S, beta)
    db = digits_base(B, eb[None, :], S, beta)
    M, N, K = A.shape[0], B.shape[1], A.shape[1]
    iacc = np.zeros((M, N), dtype=object)
    fm = np.zeros((M, N), dtype=np.float32)
    for k0 in range(0, K, chunk):
        ks = slice(k0, min(K, k0 + chunk))
        for L in range(2, max_level + 1):
            lv = np.zeros((M, N), dtype=object)
            for s in range(1, S + 1):
                t = L - s
                if 1 <= t <= S:
                    lv = lv + da[s - 1][:, ks].dot(db[t - 1][ks, :])
            assert max(abs(int(v)) for v in lv.ravel()) <= 2 ** 24
            if L <= 9:
                iacc = iacc + lv * (2 ** (48 - 5 * L))
            else:   # the FP32 integer times 2^(65 - 5L), exact, added in FP32
                v = np.vectorize(float)(lv).astype(np.float32)
                fm = (fm + v * np.float32(2.0 ** (65 - 5 * L))).astype(np.float32)
        assert max(abs(int(v)) for v in iacc.ravel()) < 2 ** 63
    C = np.empty((M, N))
    for i in range(M):
        for j in range(N):
            v = float(iacc[i, j]) + float(fm[i, j]) * 2.0 ** -17
            C[i, j] = math.ldexp(v, int(ea[i] + eb[j]) - 48)
    return C


def test_fp8_form_is_fp64_grade(operands):
    A, B = operands
    K = A.shape[1]
    C = split_product_fp8(A, B)
    ref = exact_product(A, B)
    scale = np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(B), axis=0)[None, :]
    err = np.max(np.abs(C - ref) / scale)
    assert err <= 8 * math.sqrt(K) * 2.0 ** -54
    assert err <= 2e-16 * math.sqrt(K)


def test_fp8_form_keeps_level_13():
    # with levels <= S + 1 only, the dropped level-13 pairs dominate the error
    rng = np.random.default_rng(15)
    A = rng.standard_normal((6, 200))
    B = rng.standard_normal((200, 5))
    ref = exact_product(A, B)
    scale = np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(B), axis=0)[None, :]
    e_keep = np.max(np.abs(split_product_fp8(A, B) - ref) / scale)
    e_drop = np.max(np.abs(split_product_fp8(A, B, max_level=12) - ref) / scale)
    assert e_drop > 2 * e_keep
    assert sum(1 for s in range(1, 12) for t in range(1, 12) if s + t <= 13) == 76


def test_fp8_digits_are_exact_in_e4m3():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no E4M3 dtype in this torch")
    d = torch.arange(-16, 17, dtype=torch.float32)
    assert torch.equal(d.to(torch.float8_e4m3fn).to(torch.float32), d)
    assert torch.float8_e4m3fn is not None and float(torch.tensor(17.0).to(torch.float8_e4m3fn)) != 17.0
    rng = np.random.default_rng(16)
    X = rng.standard_normal((5, 64)) * 10.0 ** rng.uniform(-20, 20, (5, 1))
    for dg in digits_base(X, exponents(X, axis=1)[:, None], 11, 5):
        assert max(abs(int(v)) for v in dg.ravel()) <= 16


def test_fp8_form_level_sums_exact_over_a_4096_chunk():
    # |d| <= 16: a level of p <= 11 pairs over 4096 terms stays within 2^24
    for level in range(2, 14):
        p = min(level - 1, 11, 23 - level)
        assert p * 4096 * 16 * 16 <= 2 ** 24
    # the int64 of 2^-48 units: levels 2..9 of one chunk at the digit bound stay
    # below 2^58.1, so about 29 chunks (K ~ 110000) fit
    per_chunk = sum(min(L - 1, 11) * 4096 * 256 * 2 ** (48 - 5 * L) for L in range(2, 10))
    assert 29 * per_chunk < 2 ** 63
    # the model's own accumulators (checked inside) at the digit bound over two chunks
    A = np.full((1, 8192), 0.4999)
    B = np.full((8192, 1), -0.4999)
    C = split_product_fp8(A, B)
    assert abs(C[0, 0] - exact_product(A, B)[0, 0]) <= 8192 * 2.0 ** -52


def test_long_k_pieces_keep_the_int64_exact():
    # gemm_split cuts K into products of at most 56 x 2048 (BF16), 120 x 512
    # (FP16) and 28 x 4096 (FP8) terms: at the digit bounds the int64 of 2^-48
    # (FP16: 2^-49) units, summed over those chunks, stays below 2^63
    def per_chunk(bits, chunk, top_int_level, unit, pairs_cap):
        return sum(min(L - 1, pairs_cap) * chunk * 2 ** (2 * (bits - 1)) * 2 ** (unit - bits * L)
                   for L in range(2, top_int_level + 1))
    bf16 = per_chunk(6, 2048, 8, 48, 9)
    fp16 = per_chunk(7, 512, 7, 49, 8)
    fp8 = per_chunk(5, 4096, 9, 48, 11)
    assert 56 * bf16 < 2 ** 63 and 120 * fp16 < 2 ** 63 and 28 * fp8 < 2 ** 63
    # and the pieces are not needlessly short: twice as many chunks would not fit
    assert 2 * 56 * bf16 > 2 ** 63 and 2 * 120 * fp16 > 2 ** 63 and 2 * 28 * fp8 > 2 ** 63
