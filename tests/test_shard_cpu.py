"""The shift-sharded path (Section 3.2, Algorithm 3) on CPU ranks.

Algorithm 3 gives each of r process groups one shifted factorisation and sums
their terms T_j with DGSUM2D.  zolo_pd_sharded does the same over ranks: the
library's zolo_shift_range hands each rank a block of the shifts and a sum
over ranks (torch_allreduce: torch.distributed's all-reduce) joins the
partial sums.  Here two gloo ranks run that exchange with the oracle's
per-group terms in place of the GPU kernels, and the result must equal the
single-process oracle's; the partition itself must cover every shift once."""
import socket
import sys

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def zb():
    from paper_1806_06204_gb300 import build
    build.build()
    from paper_1806_06204_gb300 import binding
    return binding


def test_shift_ranges_cover_every_shift_once_and_balance(zb):
    for r in range(1, 9):
        for nranks in range(1, 11):
            got = [zb.shift_range(r, k, nranks) for k in range(nranks)]
            assert got[0][0] == 0 and got[-1][1] == r
            for (a0, a1), (b0, b1) in zip(got, got[1:]):
                assert a1 == b0                                  # contiguous, no overlap
            sizes = [j1 - j0 for j0, j1 in got]
            assert max(sizes) - min(sizes) <= 1 and sum(sizes) == r
    with pytest.raises(zb.ZoloError):
        zb.shift_range(8, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle import zolo_oracle as zo
    from paper_1806_06204_gb300 import binding as zb, synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        res = {}
        for m, n, kappa, r in ((40, 24, 1e8, 6), (32, 32, 1e3, 3)):
            sm = synth.tall_uniform(m, n, 1.0 / kappa, seed=17) if m > n else \
                synth.square_geometric(n, kappa, seed=18)
            ell0 = float(sm.sigma[-1])
            ells, used_qr, _ = zb.schedule(ell0, r)
            j0, j1 = zb.shift_range(r, rank, world)
            total = zb.torch_allreduce()
            X = sm.A.copy()
            for k, qr in enumerate(used_qr):
                co = zo.zolotarev_coeffs(ells[k], r)
                S = torch.from_numpy(zo.group_terms(X, co, range(j0, j1), qr))
                total(S)                                  # DGSUM2D over the ranks
                X = co.Mhat * (X + S.numpy())
            res[(m, n)] = X
        out[rank] = res
    finally:
        dist.destroy_process_group()


def test_two_ranks_sum_their_shifts_to_the_single_process_result():
    import torch.multiprocessing as mp
    from oracle import zolo_oracle as zo
    from paper_1806_06204_gb300 import synth
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for (m, n, kappa, r) in ((40, 24, 1e8, 6), (32, 32, 1e3, 3)):
        sm = synth.tall_uniform(m, n, 1.0 / kappa, seed=17) if m > n else \
            synth.square_geometric(n, kappa, seed=18)
        Qp, _, info = zo.zolo_pd(sm.A, 1.0, float(sm.sigma[-1]), r=r)
        X0, X1 = res[0][(m, n)], res[1][(m, n)]
        assert np.array_equal(X0, X1)                     # every rank holds the same X
        assert np.linalg.norm(X0 - Qp) / np.linalg.norm(Qp) < 1e-14
