"""The bounded waits' error exit on the GPU, made to run on purpose.

zolo_debug_stall makes a kernel's first wait one that nothing completes (an
mbarrier no thread or copy arrives at in the split-precision product; a flag
no thread sets in the FP32 Jacobi sweep and before the first column pair of the
FP64 sweep, whose other blocks wait for that pair's columns), bounded by a few
milliseconds.  The
kernel must give up, let what it has in flight finish, release its tensor
memory and return; the call must report ZOLO_ETIMEOUT; and the next call on the
same handle, with the hook off, must compute the right result.  Nothing here
faults or hangs the GPU: every wait involved is bounded."""
import numpy as np
import pytest

from oracle import zolo_oracle as zo

pytestmark = pytest.mark.gpu

ZOLO_ETIMEOUT = 7
STALL_NS = 5_000_000   # 5 ms


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


def test_split_product_wait_expires_then_recovers(zb):
    h = zb.Handle(0)
    try:
        rng = np.random.default_rng(3)
        A, B = rng.standard_normal((300, 200)), rng.standard_normal((200, 260))
        zb.debug_stall(h, zb.ZOLO_STALL_SPLIT_GEMM, STALL_NS)
        C = zb.empty_colmajor(300, 260)
        for _ in range(2):   # the flag is cleared at the start of every call
            with pytest.raises(zb.ZoloError) as ex:
                zb.zolo_dgemm(h, dev(A), dev(B), C, prec=zb.ZOLO_SPLIT_BF16, slices=9)
            assert ex.value.code == ZOLO_ETIMEOUT
        zb.debug_stall(h, 0, 0)
        C = zb.zolo_dgemm(h, dev(A), dev(B), prec=zb.ZOLO_SPLIT_BF16, slices=9).cpu().numpy()
        ref = A @ B
        assert np.max(np.abs(C - ref)) <= 1e-13 * np.max(np.abs(A) @ np.abs(B))
    finally:
        h.close()


def test_split_polar_decomposition_reports_timeout_then_matches_oracle(zb):
    from paper_1806_06204_gb300 import synth
    sm = synth.square_geometric(160, 1e6, seed=1010)
    A = dev(sm.A)
    h = zb.Handle(0)
    try:
        o = zb.opts(beta=float(sm.sigma[-1]), alpha=1.0, r=4, prec=zb.ZOLO_SPLIT_BF16, ns_steps=1)
        zb.debug_stall(h, zb.ZOLO_STALL_SPLIT_GEMM, STALL_NS)
        _, _, info = zb.zolo_pd(h, A, o, check=False)
        assert info.status == ZOLO_ETIMEOUT
        zb.debug_stall(h, 0, 0)
        Qp, H, info = zb.zolo_pd(h, A, o)
        assert info.status == 0
        Qo, Ho, io = zo.zolo_pd(sm.A, 1.0, float(sm.sigma[-1]), r=4, ns_steps=1)
        Qp, H = Qp.cpu().numpy(), H.cpu().numpy()
        assert zo.backward_error_pd(sm.A, Qp, H) < 1e-13 and zo.orthogonality(Qp) < 1e-13
        assert np.linalg.norm(H - Ho) / np.linalg.norm(Ho) < 1e-12
    finally:
        h.close()


@pytest.mark.parametrize("n", [200, 600])
def test_jacobi_grid_barrier_wait_expires_then_recovers(zb, n):
    # 600: two blocks per block pair, which also meet at a barrier between the
    # Gram partials and the rotations
    from paper_1806_06204_gb300 import synth
    sm = synth.square_geometric(n, 1e6, seed=1011)
    A = dev(sm.A)
    h = zb.Handle(0)
    try:
        o = zb.opts(beta=float(sm.sigma[-1]), alpha=1.0, r=4)
        zb.debug_stall(h, zb.ZOLO_STALL_JACOBI32, STALL_NS)
        _, _, _, info = zb.zolo_svd(h, A, o, check=False)
        assert info.status == ZOLO_ETIMEOUT
        zb.debug_stall(h, 0, 0)
        U, S, V, info = zb.zolo_svd(h, A, o)
        assert info.status == 0
        assert np.max(np.abs(S.cpu().numpy() - sm.sigma)) <= 1e-12 * sm.sigma[0]
    finally:
        h.close()


def test_jacobi_fp64_sweep_wait_expires_then_recovers(zb):
    # the first FP64 sweep's block 0 stalls before its first column pair: the
    # blocks whose pairs need those columns give up on the error flag
    from paper_1806_06204_gb300 import synth
    sm = synth.square_geometric(300, 1e6, seed=1012)
    A = dev(sm.A)
    h = zb.Handle(0)
    try:
        o = zb.opts(beta=float(sm.sigma[-1]), alpha=1.0, r=4)
        zb.debug_stall(h, zb.ZOLO_STALL_JACOBI64, STALL_NS)
        for _ in range(2):
            _, _, _, info = zb.zolo_svd(h, A, o, check=False)
            assert info.status == ZOLO_ETIMEOUT
        zb.debug_stall(h, 0, 0)
        U, S, V, info = zb.zolo_svd(h, A, o)
        assert info.status == 0
        assert np.max(np.abs(S.cpu().numpy() - sm.sigma)) <= 1e-12 * sm.sigma[0]
        U, V = U.cpu().numpy(), V.cpu().numpy()
        assert zo.orthogonality(U) <= 1e-13 and zo.orthogonality(V) <= 1e-13
    finally:
        h.close()
