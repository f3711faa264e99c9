"""CPU model of the FP64 GEMM's split-K index arithmetic (no GPU).

With ksplit > 1 a CTA of output tile column n0 and K slice s runs the 16-deep
steps k0 = max(kbeg, s kc), ..., < min(K, (s + 1) kc) with kc = ceil(ceil(K /
ksplit) / 16) 16, kbeg = 0, or floor(n0 / 16) 16 when op(B) is lower triangular;
every step must fall in exactly one slice, so the slices' raw sums add up to the
one-pass kernel's sum over the same steps.
"""
import pytest

BK = 16


def steps(K, ksplit, s, kbeg0):
    kc = -(-(-(-K // ksplit)) // BK) * BK
    lo, hi = max(kbeg0, s * kc), min(K, (s + 1) * kc)
    return list(range(lo, hi, BK)) if ksplit > 1 else list(range(kbeg0, K, BK))


@pytest.mark.parametrize("K", [1, 15, 16, 17, 100, 257, 1000, 1024, 4096, 4099])
@pytest.mark.parametrize("ksplit", [2, 4, 8])
@pytest.mark.parametrize("n0", [0, 64, 128, 960])
def test_split_k_slices_partition_the_steps(K, ksplit, n0):
    for b_lower in (False, True):
        kbeg0 = (n0 // BK) * BK if b_lower else 0
        one_pass = steps(K, 1, 0, kbeg0)
        split = [k for s in range(ksplit) for k in steps(K, ksplit, s, kbeg0)]
        assert sorted(split) == one_pass
        assert len(split) == len(set(split))
