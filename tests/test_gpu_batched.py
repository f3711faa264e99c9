"""GPU parity of the grouped launch (zolo_pd_batched) through the C ABI.

Each matrix of a batch of mixed sizes, condition numbers and precisions must
meet the same invariants as a single zolo_pd call and agree with the oracle's
polar factor within the conditioning-scaled tolerance (the polar factor's
sensitivity is ~1/(sigma_{n-1} + sigma_n)).  A second call with the same
pointers replays the recorded CUDA graph and must give the same bits."""
import math

import numpy as np
import pytest

from oracle import zolo_oracle as zo
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


@pytest.fixture(scope="module")
def handle(zb):
    h = zb.Handle(0)
    yield h
    h.close()


def dev(a):
    import torch
    return torch.from_numpy(np.asfortranarray(a)).cuda()


def _case(shapes, kappas, seed):
    mats = []
    for i, ((m, n), kap) in enumerate(zip(shapes, kappas)):
        mats.append(synth.make_matrix(m, n, synth.geometric_sigma(n, kap), seed=seed + i))
    return mats


def _check(zb, sm, Qp, H, beta):
    A = sm.A
    Qh, Hh = Qp.cpu().numpy(), H.cpu().numpy()
    assert zo.orthogonality(Qh) <= 1e-13
    assert zo.backward_error_pd(A, Qh, Hh) <= 1e-13
    assert np.array_equal(Hh, Hh.T)
    Qo, Ho, _ = zo.zolo_pd(A, alpha=sm.sigma.max(), beta=beta)
    s = np.sort(sm.sigma)
    tol = 200 * zo.EPS / ((s[0] + s[1]) / s[-1])
    assert np.max(np.abs(Qh - Qo)) <= tol
    assert np.max(np.abs(Hh - Ho)) <= 1e-12 * s[-1]


def test_batched_mixed_sizes_fp64_matches_oracle_and_replays(zb, handle):
    shapes = [(96, 96), (130, 70), (64, 64), (200, 129), (33, 33), (257, 100)]
    kappas = [1e6, 1e3, 1e12, 20.0, 1e8, 1e15]
    mats = _case(shapes, kappas, 100)
    As = [dev(sm.A) for sm in mats]
    os = [zb.opts(beta=0.9 * sm.sigma.min() / sm.sigma.max(), alpha=sm.sigma.max())
          for sm in mats]
    Qps, Hs, infos, st = zb.zolo_pd_batched(handle, As, os)
    assert st == 0
    for sm, q, hh, inf, o in zip(mats, Qps, Hs, infos, os):
        assert inf.status == 0
        _check(zb, sm, q, hh, o.beta)
    first = [(q.cpu().numpy().copy(), hh.cpu().numpy().copy()) for q, hh in zip(Qps, Hs)]
    # same pointers and options: the recorded graph is replayed
    _, _, infos2, st2 = zb.zolo_pd_batched(handle, As, os, Qps=Qps, Hs=Hs)
    assert st2 == 0
    for (q0, h0), q, hh in zip(first, Qps, Hs):
        assert np.array_equal(q0, q.cpu().numpy())
        assert np.array_equal(h0, hh.cpu().numpy())


def test_batched_equals_single_calls_bit_for_bit(zb, handle):
    shapes = [(150, 120), (64, 48), (300, 300)]
    mats = _case(shapes, [1e10, 1e4, 1e7], 200)
    os = [zb.opts(beta=0.5 / 1e10, alpha=0.0), zb.opts(beta=0.5 / 1e4, alpha=0.0, r=3),
          zb.opts(beta=0.5 / 1e7, alpha=0.0)]
    As = [dev(sm.A) for sm in mats]
    Qps, Hs, infos, st = zb.zolo_pd_batched(handle, As, os)
    assert st == 0
    for a, o, q, hh, inf in zip(As, os, Qps, Hs, infos):
        q1, h1, inf1 = zb.zolo_pd(handle, a, o)
        assert inf.iters == inf1.iters and inf.r == inf1.r
        assert np.array_equal(q.cpu().numpy(), q1.cpu().numpy())
        assert np.array_equal(hh.cpu().numpy(), h1.cpu().numpy())


def test_batched_inverse_cholesky_form_equals_single_calls(zb, handle):
    # m >= 512: the batched call factors each QR panel on fewer CTAs than a single
    # call (many problems are in flight), which sums a column's norm and dot
    # products in another order, so the results agree to rounding; below 512
    # rows both use one CTA and agree bit for bit
    shapes = [(600, 150), (128, 128), (333, 97)]
    mats = _case(shapes, [1e6, 1e9, 1e3], 400)
    os = [zb.opts(beta=0.5 / 1e6, alpha=0.0, r=6), zb.opts(beta=0.5 / 1e9, r=8, chol_form=2),
          zb.opts(beta=0.5 / 1e3, r=4, chol_form=1)]
    As = [dev(sm.A) for sm in mats]
    Qps, Hs, infos, st = zb.zolo_pd_batched(handle, As, os)
    assert st == 0
    for sm, a, o, q, hh, inf in zip(mats, As, os, Qps, Hs, infos):
        _check(zb, sm, q, hh, o.beta / (o.alpha if o.alpha > 0 else 1.0))
        q1, h1, inf1 = zb.zolo_pd(handle, a, o)
        assert inf.iters == inf1.iters and inf.r == inf1.r
        if sm.A.shape[0] < 512:
            assert np.array_equal(q.cpu().numpy(), q1.cpu().numpy())
            assert np.array_equal(hh.cpu().numpy(), h1.cpu().numpy())
        else:
            s = np.sort(sm.sigma)
            assert np.max(np.abs(q.cpu().numpy() - q1.cpu().numpy())) <= 200 * zo.EPS / ((s[0] + s[1]) / s[-1])
            assert np.max(np.abs(hh.cpu().numpy() - h1.cpu().numpy())) <= 1e-13 * s[-1]


def test_batched_estimates_beta_as_the_single_call_does(zb, handle):
    # beta <= 0 and alpha <= 0: both bounds computed on the device before the batch
    # starts; every matrix then runs the schedule the single call would run
    shapes = [(180, 120), (96, 96), (250, 70)]
    mats = _case(shapes, [1e9, 1e3, 1e6], 500)
    os = [zb.opts(beta=0.0, alpha=0.0), zb.opts(beta=-1.0, alpha=1.0, r=3),
          zb.opts(beta=0.0, alpha=0.0, prec=zb.ZOLO_SPLIT_BF16, ns_steps=1)]
    As = [dev(sm.A) for sm in mats]
    Qps, Hs, infos, st = zb.zolo_pd_batched(handle, As, os)
    assert st == 0
    for sm, a, o, q, hh, inf in zip(mats, As, os, Qps, Hs, infos):
        q1, h1, inf1 = zb.zolo_pd(handle, a, o)
        assert inf.ell[0] == inf1.ell[0] and inf.r == inf1.r and inf.iters == inf1.iters
        s = np.sort(sm.sigma)
        alpha = zo.alpha_bound(sm.A) if o.alpha <= 0 else o.alpha
        beta = inf.ell[0] * alpha
        assert s[0] / math.sqrt(len(s)) * (1 - 1e-6) <= beta <= s[0] * (1 + 1e-6)
        Qh, Hh = q.cpu().numpy(), hh.cpu().numpy()
        assert zo.orthogonality(Qh) <= 1e-13 and zo.backward_error_pd(sm.A, Qh, Hh) <= 1e-13
        if o.prec == zb.ZOLO_FP64:
            assert np.array_equal(Qh, q1.cpu().numpy()) and np.array_equal(Hh, h1.cpu().numpy())
        else:   # the lanes' slice buffers may chunk a batched product differently
            assert np.max(np.abs(Qh - q1.cpu().numpy())) <= 200 * zo.EPS / ((s[0] + s[1]) / s[-1])


def test_batched_split_precision_invariants(zb, handle):
    # BF16, FP16 and FP8 slices side by side in one batch
    shapes = [(256, 256), (192, 128), (128, 128), (600, 300), (320, 200)]
    mats = _case(shapes, [1e8, 1e3, 1e14, 1e10, 1e12], 300)
    precs = [zb.ZOLO_SPLIT_BF16, zb.ZOLO_SPLIT_FP16, zb.ZOLO_SPLIT_FP8, zb.ZOLO_SPLIT_FP16,
             zb.ZOLO_SPLIT_FP8]
    os = [zb.opts(beta=0.9 * sm.sigma.min() / sm.sigma.max(), alpha=sm.sigma.max(),
                  prec=p) for sm, p in zip(mats, precs)]
    As = [dev(sm.A) for sm in mats]
    Qps, Hs, infos, st = zb.zolo_pd_batched(handle, As, os)
    assert st == 0
    for sm, q, hh in zip(mats, Qps, Hs):
        Qh, Hh = q.cpu().numpy(), hh.cpu().numpy()
        assert zo.orthogonality(Qh) <= 1e-13
        assert zo.backward_error_pd(sm.A, Qh, Hh) <= 1e-13


def test_batched_empty_and_bad_arguments(zb, handle):
    _, _, infos, st = zb.zolo_pd_batched(handle, [], [])
    assert st == 0 and infos == []
    sm = synth.make_matrix(64, 64, synth.geometric_sigma(64, 10.0), seed=7)
    o = zb.opts(beta=0.05, alpha=sm.sigma.max(), posteriori=True)
    _, _, infos, st = zb.zolo_pd_batched(handle, [dev(sm.A)], [o], check=False)
    assert st == -10 and infos[0].status == -10


def test_batched_without_graph_equals_graph_replay(zb):
    # zolo_batch_graphs(h, 0): the lanes' work is queued directly (for profilers);
    # the same kernels give the same bits as the recorded graph's replay
    h = zb.Handle(0)
    try:
        mats = _case([(160, 160), (96, 64), (300, 200)], [1e7, 1e3, 1e11], 700)
        As = [dev(sm.A) for sm in mats]
        os = [zb.opts(beta=0.5 * sm.sigma.min(), alpha=sm.sigma.max(),
                      prec=p) for sm, p in zip(mats, (0, 1, 2))]
        Q1, H1, _, st = zb.zolo_pd_batched(h, As, os)
        Q1, H1 = zb.zolo_pd_batched(h, As, os, Qps=Q1, Hs=H1)[:2]   # replayed
        assert st == 0
        zb.batch_graphs(h, False)
        Q2, H2, _, st2 = zb.zolo_pd_batched(h, As, os)
        assert st2 == 0
        for a, b, c, d in zip(Q1, Q2, H1, H2):
            assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
            assert np.array_equal(c.cpu().numpy(), d.cpu().numpy())
    finally:
        h.close()
