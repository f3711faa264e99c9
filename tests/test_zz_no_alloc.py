"""The allocation-free GEMM entry point (zolo_dgemm_noalloc).

It serves callers that cannot allocate device memory where they call the
library: its scratch is a fixed device array, not cudaMalloc.  It must give the
same result as zolo_dgemm on the split tensor-core path, call after call (the
shared array keeps the previous call's contents, so the second call checks that
nothing stale leaks in).  This file is collected last on purpose; it also has to
pass on its own in a fresh process."""
import numpy as np
import pytest

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


def dev(a):
    import torch
    return torch.from_numpy(np.asfortranarray(a)).cuda()


# the last case is a tall product with more than 8192 rows: its slices fit the
# scratch and so must its exponents (one per padded row and column)
@pytest.mark.parametrize("m,n,k,ta,tb,S", [(256, 192, 300, 0, 0, 8), (100, 257, 129, 1, 1, 9),
                                           (9000, 8, 8, 0, 0, 8)])
def test_noalloc_matches_allocating_entry_point_twice(zb, m, n, k, ta, tb, S):
    h = zb.Handle(0)
    try:
        for call in range(2):
            rng = np.random.default_rng(10 * call + m)
            A = rng.standard_normal((k, m) if ta else (m, k))
            B = rng.standard_normal((n, k) if tb else (k, n))
            C0 = rng.standard_normal((m, n))
            C_ref, C_na = dev(C0), dev(C0)
            zb.zolo_dgemm(h, dev(A), dev(B), C_ref, alpha=0.5, beta=2.0, transA=bool(ta),
                          transB=bool(tb), prec=zb.ZOLO_SPLIT_BF16, slices=S)
            zb.zolo_dgemm_noalloc(dev(A), dev(B), C_na, alpha=0.5, beta=2.0, transA=bool(ta),
                                  transB=bool(tb), slices=S)
            ref, got = C_ref.cpu().numpy(), C_na.cpu().numpy()
            # same kernels and inputs: agreement to rounding (in practice bit for bit)
            assert np.allclose(got, ref, rtol=1e-14, atol=1e-14 * np.abs(ref).max())
            exact = 0.5 * (A.T if ta else A) @ (B.T if tb else B) + 2.0 * C0
            assert np.max(np.abs(got - exact)) < 1e-11 * np.abs(exact).max()
    finally:
        h.close()


def test_noalloc_refuses_sizes_beyond_its_scratch(zb):
    import torch
    A = torch.zeros((2048, 2048), dtype=torch.float64, device="cuda").t()
    C = torch.zeros((2048, 2048), dtype=torch.float64, device="cuda").t()
    assert zb.zolo_dgemm_noalloc(A, A, C, check=False) == 5   # ZOLO_ENOMEM, nothing touched
