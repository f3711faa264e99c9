"""zolo_pd_sharded on one GPU: the shifts of every iteration shared out over
ranks (Section 3.2, Algorithm 3), each rank a host thread with its own handle
and stream.  The sum over ranks runs on the host side of the exchange: a rank
waits for its own stream, publishes its partial sum, and every rank adds the
partial sums in rank order once all are in (so all ranks keep identical bits).
No kernel of one rank waits on another rank's: the ranks meet only on the host,
between kernels.  The results must equal zolo_pd's on the same matrix."""
import threading

import numpy as np
import pytest

from oracle import zolo_oracle as zo

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


class HostSum:
    """A sum over `n` thread-ranks: the all-reduce of the exchange, in rank order."""

    def __init__(self, n):
        self.parts = [None] * n
        self.bar = threading.Barrier(n, timeout=120)

    def for_rank(self, rank):
        import torch

        def f(t):
            s = torch.cuda.current_stream()
            self.parts[rank] = t.clone()
            s.synchronize()
            self.bar.wait()
            tot = self.parts[0].clone()
            for p in self.parts[1:]:
                tot += p
            t.copy_(tot)
            s.synchronize()
            self.bar.wait()       # nobody overwrites a part before all have read it
        return f


def run_ranks(zb, A, o, nranks):
    import torch
    ex = HostSum(nranks)
    res = [None] * nranks
    errs = []

    def work(rank):
        try:
            torch.cuda.set_device(0)
            h = zb.Handle(0)
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                Qp, H, info = zb.zolo_pd_sharded(h, A, o, rank, nranks, ex.for_rank(rank))
            s.synchronize()
            res[rank] = (Qp.cpu().numpy(), H.cpu().numpy(), info)
            h.close()
        except Exception as e:   # surfaced below
            errs.append(e)
            ex.bar.abort()

    ts = [threading.Thread(target=work, args=(k,)) for k in range(nranks)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errs, errs
    return res


@pytest.mark.parametrize("n,kappa,r,nranks,split", [(192, 1e8, 6, 2, False), (160, 1e6, 5, 3, False),
                                                   (192, 1e8, 6, 2, True), (96, 1e4, 3, 4, False)])
def test_sharded_equals_single_rank(zb, n, kappa, r, nranks, split):
    import torch
    from paper_1806_06204_gb300 import synth
    sm = synth.square_geometric(n, kappa, seed=1020 + n)
    A = torch.from_numpy(sm.A).cuda()
    prec = zb.ZOLO_SPLIT_BF16 if split else zb.ZOLO_FP64
    o = zb.opts(beta=float(sm.sigma[-1]), alpha=1.0, r=r, prec=prec, ns_steps=1 if split else 0)
    h = zb.Handle(0)
    Q1, H1, i1 = zb.zolo_pd(h, A, o)
    Q1, H1 = Q1.cpu().numpy(), H1.cpu().numpy()
    h.close()
    res = run_ranks(zb, A, o, nranks)
    for Qp, H, info in res:
        assert np.array_equal(Qp, res[0][0]) and np.array_equal(H, res[0][1])
        assert info.iters == i1.iters and info.used_qr == i1.used_qr and info.r == r
        assert np.allclose(info.delta, i1.delta, rtol=1e-10, atol=1e-15)
    Qp, H, _ = res[0]
    assert zo.orthogonality(Qp) < 1e-13 and zo.backward_error_pd(sm.A, Qp, H) < 1e-13
    # H is well conditioned; Q_p's smallest singular directions move by ~eps kappa
    # under a different rounding order of the shifts' sum
    assert np.linalg.norm(H - H1) / np.linalg.norm(H1) < 1e-13
    assert np.linalg.norm(Qp - Q1) / np.linalg.norm(Q1) < 1e-13 + 1e-15 * kappa


def test_breakdown_on_one_rank_makes_every_rank_redo_in_qr_form(zb):
    # the Cholesky form forced on kappa 1e12: the small shifts (rank 0's block)
    # break down; the summed flag makes both ranks redo the iteration in the QR form
    import torch
    from paper_1806_06204_gb300 import synth
    sm = synth.square_geometric(128, 1e12, seed=9)
    A = torch.from_numpy(sm.A).cuda()
    o = zb.opts(beta=1e-12, r=8, force_qr=0)
    res = run_ranks(zb, A, o, 2)
    for Qp, H, info in res:
        assert info.chol_fallbacks >= 1 and info.used_qr[0]
        assert np.array_equal(Qp, res[0][0])
    Qp, H, _ = res[0]
    assert zo.orthogonality(Qp) < 1e-13 and zo.backward_error_pd(sm.A, Qp, H) < 1e-13
