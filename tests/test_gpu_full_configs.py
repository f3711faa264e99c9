"""The single-matrix configurations at their full sizes, with the generators and
seeds bench.py uses: the 4096^2 Zolo-SVD (sigma geometric 1..1e-12, r = 8, FP64,
kernels kept by the autotuner in a warm-up call, as the bench's timed steps use
them) and the 16384 x 4096 Zolo-PD (sigma uniform in [1e-6, 1], r = 6) in FP64
and in the BF16 and FP16 split forms.  The CPU oracle cannot decompose these
sizes in a test's time, so the results are checked by what holds at any size:
the backward error and orthogonality bar (1e-13), the singular values the
matrix was built from (1e-12 sigma_1), and the factors of A = U diag(sigma) V^T,
which fix the exact answer: Qp = U V^T, H = V diag(sigma) V^T, and the singular
vectors of well separated singular values up to sign.  The checks run on the
device with torch (test infrastructure, not the product path)."""
import math

import numpy as np
import pytest

from paper_1806_06204_gb300 import synth

pytestmark = pytest.mark.gpu

EPS = 2.220446049250313e-16


@pytest.fixture(scope="module")
def zb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06204_gb300 import build
    build.build()
    from paper_1806_06204_gb300 import binding
    return binding


def test_svd_4096_kappa_1e12_r8(zb):
    import torch
    n = 4096
    sm = synth.make_matrix(n, n, synth.geometric_sigma(n, 1e12), 2000)
    A = torch.from_numpy(sm.A).cuda()
    o = zb.opts(beta=float(sm.sigma[-1]), alpha=1.0, r=8)
    h = zb.Handle(0)
    try:
        zb.autotune(h, True)
        zb.zolo_svd(h, A, o)
        zb.autotune(h, False)
        U, S, V, info = zb.zolo_svd(h, A, o)
        assert info.status == 0 and info.r == 8 and info.used_qr[:2] == [True, False]
        sig = torch.from_numpy(sm.sigma).cuda()
        I = torch.eye(n, dtype=torch.float64, device="cuda")
        assert float(torch.max(torch.abs(S - sig))) <= 1e-12 * sm.sigma[0]
        assert float(torch.linalg.norm(A - (U * S) @ V.T) / torch.linalg.norm(A)) <= 1e-13
        assert float(torch.linalg.norm(U.T @ U - I)) / math.sqrt(n) <= 1e-13
        assert float(torch.linalg.norm(V.T @ V - I)) / math.sqrt(n) <= 1e-13
        # singular vectors of singular values 1e-3 sigma_1 apart: error about
        # eps ||A|| / gap, far below the tolerance
        s = sm.sigma
        gap = np.minimum(np.abs(np.diff(np.r_[np.inf, s])), np.abs(np.diff(np.r_[s, -np.inf])))
        sep = torch.from_numpy(gap > 1e-3 * s[0]).cuda()
        assert int(sep.sum()) >= 100
        Ug, Vg = torch.from_numpy(sm.U).cuda(), torch.from_numpy(sm.V).cuda()
        cu = torch.abs(torch.sum(U * Ug, dim=0))[sep]
        cv = torch.abs(torch.sum(V * Vg, dim=0))[sep]
        assert float(torch.max(torch.abs(cu - 1))) <= 1e-9
        assert float(torch.max(torch.abs(cv - 1))) <= 1e-9
    finally:
        h.close()


@pytest.fixture(scope="module")
def tall():
    import torch
    sm = synth.tall_uniform(16384, 4096, lo=1e-6, seed=2000)
    A = torch.from_numpy(sm.A).cuda()
    Ug, Vg = torch.from_numpy(sm.U).cuda(), torch.from_numpy(sm.V).cuda()
    sig = torch.from_numpy(sm.sigma).cuda()
    Qx = Ug @ Vg.T                       # the exact polar factor
    Hx = (Vg * sig) @ Vg.T               # the exact symmetric factor
    return sm, A, Qx, Hx


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_pd_16384x4096_uniform_sigma_r6(zb, tall, prec):
    import torch
    sm, A, Qx, Hx = tall
    m, n = A.shape
    o = zb.opts(beta=float(sm.sigma[-1]), alpha=1.0, r=6, prec=prec, ns_steps=1 if prec else 0)
    h = zb.Handle(0)
    try:
        Qp, H, info = zb.zolo_pd(h, A, o)
        assert info.status == 0 and info.r == 6
        I = torch.eye(n, dtype=torch.float64, device="cuda")
        nA = torch.linalg.norm(A)
        assert float(torch.linalg.norm(A - Qp @ H) / nA) <= 1e-13
        assert float(torch.linalg.norm(Qp.T @ Qp - I)) / math.sqrt(n) <= 1e-13
        assert torch.equal(H, H.T)
        # H is as well conditioned as A's perturbation allows (||dH|| <= sqrt 2 ||dA||)
        assert float(torch.linalg.norm(H - Hx) / torch.linalg.norm(Hx)) <= 1e-13
        # Qp moves by at most about ||dA|| / sigma_n: a backward error of 1e-12
        # bounds it by 1e-12 ||A||_F / sigma_n
        assert float(torch.linalg.norm(Qp - Qx)) <= 1e-12 * float(nA) / sm.sigma[-1]
    finally:
        h.close()
