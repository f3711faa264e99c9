"""The benchmark's own batch at its full size: the 512 square matrices (n from 64
to 1024, kappa log-uniform in [1e2, 1e12], r from Table 1's rule) in one
zolo_pd_batched call, FP64 and the three split forms.  Every result meets the
invariants the contract fixes (backward error and orthogonality <= 1e-13, H
exactly symmetric); the members the CPU oracle decomposes in seconds (n = 64)
are compared with it entry by entry: H to 1e-13 of its norm, Qp within the
polar factor's conditioning (its sensitivity is about 1/(sigma_{n-1}+sigma_n))."""
import math

import numpy as np
import pytest

from oracle import zolo_oracle as zo
from paper_1806_06204_gb300 import synth

pytestmark = pytest.mark.gpu

ORACLE = {}   # the oracle's results, shared by the precisions


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
def batch():
    import torch
    mats = synth.batch(512, seed=4000)
    return mats, [torch.from_numpy(sm.A).cuda() for sm in mats]


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_full_batch_meets_the_bar_and_matches_the_oracle(zb, batch, prec):
    import torch
    mats, As = batch
    h = zb.Handle(0)
    try:
        os_ = [zb.opts(beta=float(sm.sigma[-1]), alpha=1.0, r=0, prec=prec,
                       ns_steps=1 if prec else 0) for sm in mats]
        Qps, Hs, infos, st = zb.zolo_pd_batched(h, As, os_)
        assert st == 0
        worst_b, worst_o = 0.0, 0.0
        checked = 0
        for sm, a, q, hh, inf in zip(mats, As, Qps, Hs, infos):
            n = a.shape[1]
            I = torch.eye(n, dtype=torch.float64, device="cuda")
            b = float(torch.linalg.norm(a - q @ hh) / torch.linalg.norm(a))
            o = float(torch.linalg.norm(q.T @ q - I) / math.sqrt(n))
            worst_b, worst_o = max(worst_b, b), max(worst_o, o)
            assert torch.equal(hh, hh.T)
            assert inf.r == zo.choose_r(float(sm.sigma[-1]))
            if n <= 64:
                key = (sm.seed, 1 if prec else 0)
                if key not in ORACLE:
                    ORACLE[key] = zo.zolo_pd(sm.A, 1.0, float(sm.sigma[-1]), ns_steps=key[1])
                Qo, Ho, io = ORACLE[key]
                assert inf.iters == io.iters and inf.used_qr == io.used_qr
                Hh, Qh = hh.cpu().numpy(), q.cpu().numpy()
                assert np.linalg.norm(Hh - Ho) <= 1e-13 * np.linalg.norm(Ho)
                s = np.sort(sm.sigma)
                assert np.max(np.abs(Qh - Qo)) <= 200 * zo.EPS / ((s[0] + s[1]) / s[-1])
                checked += 1
        assert worst_b <= 1e-13 and worst_o <= 1e-13, (worst_b, worst_o)
        assert checked >= 20
    finally:
        h.close()
