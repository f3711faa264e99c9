"""Guard zones around the workspace's buffers (zolo_debug_guards).

With them on, every buffer carved from the handle's workspace is followed by a
4 KB zone of 0xFF bytes and the regions that normally share memory are laid out
apart; after the call a kernel checks every zone.  The decompositions below
(ragged shapes, both iteration forms, the three precisions, the SVD's
eigensolver) must leave every zone intact, and give the same bits as without
the zones: no kernel writes outside the buffers the workspace gives it."""
import numpy as np
import pytest

from paper_1806_06204_gb300 import synth

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


@pytest.mark.parametrize("m,n,kappa,r,prec,form", [(300, 129, 1e9, 5, 0, 0), (257, 257, 1e6, 4, 1, 1),
                                                   (700, 150, 1e8, 6, 2, 2), (96, 33, 30.0, 2, 0, 1)])
def test_pd_leaves_every_guard_zone_intact(zb, m, n, kappa, r, prec, form):
    sm = synth.make_matrix(m, n, synth.geometric_sigma(n, kappa), seed=1080 + m)
    A = dev(sm.A)
    o = zb.opts(beta=float(sm.sigma[-1]), r=r, prec=prec, ns_steps=1 if prec else 0, chol_form=form)
    h = zb.Handle(0)
    try:
        Q0, H0, i0 = zb.zolo_pd(h, A, o)
        zb.debug_guards(h, True)
        Q1, H1, i1 = zb.zolo_pd(h, A, o)        # raises ZoloError(ZOLO_EGUARD) on a breach
        assert i1.status == 0 and i1.iters == i0.iters
        assert np.array_equal(Q0.cpu().numpy(), Q1.cpu().numpy())
        assert np.array_equal(H0.cpu().numpy(), H1.cpu().numpy())
    finally:
        h.close()


def test_svd_eigensolver_leaves_every_guard_zone_intact(zb):
    sm = synth.square_geometric(200, 1e7, seed=1090)
    A = dev(sm.A)
    o = zb.opts(beta=1e-7, r=5)
    h = zb.Handle(0)
    try:
        U0, S0, V0, _ = zb.zolo_svd(h, A, o)
        zb.debug_guards(h, True)
        U1, S1, V1, info = zb.zolo_svd(h, A, o)
        assert info.status == 0
        assert np.array_equal(S0.cpu().numpy(), S1.cpu().numpy())
        assert np.array_equal(U0.cpu().numpy(), U1.cpu().numpy())
    finally:
        h.close()
