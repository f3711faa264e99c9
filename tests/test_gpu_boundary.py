"""The boundary's reporting and queueing entry points on the GPU.

info.ms_phase (per-phase CUDA-event times), info.bwd_est / orth_est (opts.estimate:
the backward error and orthogonality computed on the device) and zolo_pd_async
(no host synchronisation; the status arrives by a host function at the end of
the stream's work) must agree with what the host measures and with zolo_pd."""
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


@pytest.mark.parametrize("prec", [0, 1])
def test_estimates_match_the_host_computation(zb, handle, prec):
    sm = synth.make_matrix(300, 200, synth.geometric_sigma(200, 1e9), seed=1030)
    o = zb.opts(beta=float(sm.sigma[-1]), r=7, prec=prec, ns_steps=prec, estimate=True)
    Qp, H, info = zb.zolo_pd(handle, dev(sm.A), o)
    Qh, Hh = Qp.cpu().numpy(), H.cpu().numpy()
    bwd, orth = zo.backward_error_pd(sm.A, Qh, Hh), zo.orthogonality(Qh)
    # both are rounding-level quantities: agreement to a few units of their own size
    assert 0 < info.bwd_est < 1e-13 and 0 < info.orth_est < 1e-13
    assert abs(info.bwd_est - bwd) <= 0.5 * bwd + 1e-16
    assert abs(info.orth_est - orth) <= 0.5 * orth + 1e-16
    # without the option both stay 0
    _, _, i0 = zb.zolo_pd(handle, dev(sm.A), zb.opts(beta=float(sm.sigma[-1]), r=7, prec=prec))
    assert i0.bwd_est == 0.0 and i0.orth_est == 0.0


def test_phase_times_cover_the_call(zb, handle):
    sm = synth.square_geometric(256, 1e8, seed=1031)
    o = zb.opts(beta=1e-8, r=3, estimate=True)
    _, _, info = zb.zolo_pd(handle, dev(sm.A), o)
    ph = info.ms_phase
    assert info.used_qr == [True, False, False]
    assert ph["qr"] > 0 and ph["chol"] > 0 and ph["H"] > 0 and ph["estimates"] > 0
    assert ph["eig"] == 0 and ph["U"] == 0 and ph["newton_schulz"] == 0
    total = sum(ph.values())
    assert 0.5 * info.ms <= total <= info.ms * 1.01 + 0.05
    U, S, V, si = zb.zolo_svd(handle, dev(sm.A), zb.opts(beta=1e-8, r=3))
    assert si.ms_phase["eig"] > 0 and si.ms_phase["U"] > 0
    assert sum(si.ms_phase.values()) <= si.ms * 1.01 + 0.05


@pytest.mark.parametrize("prec", [0, 1])
def test_async_equals_the_synchronous_call(zb, handle, prec):
    import torch
    mats = [synth.make_matrix(m, n, synth.geometric_sigma(n, k), seed=1040 + i)
            for i, (m, n, k) in enumerate([(200, 150, 1e6), (128, 128, 1e10), (90, 40, 30.0)])]
    s = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(s):
        for sm in mats:
            o = zb.opts(beta=float(sm.sigma[-1]), prec=prec, ns_steps=prec, estimate=True)
            A = dev(sm.A)
            Qp, H, pending = zb.zolo_pd_async(handle, A, o)
            outs.append((sm, A, o, Qp, H, pending))
    s.synchronize()
    for sm, A, o, Qp, H, pending in outs:
        inf = pending()
        assert inf.status == 0 and inf.bwd_est < 1e-13 and inf.orth_est < 1e-13
        Q1, H1, i1 = zb.zolo_pd(handle, A, o)
        assert inf.iters == i1.iters and inf.r == i1.r and inf.used_qr == i1.used_qr
        assert np.allclose(inf.delta, i1.delta, rtol=1e-12, atol=0)
        assert np.array_equal(Qp.cpu().numpy(), Q1.cpu().numpy())
        assert np.array_equal(H.cpu().numpy(), H1.cpu().numpy())


def test_async_refuses_what_needs_a_round_trip(zb, handle):
    sm = synth.square_geometric(64, 1e4, seed=1050)
    with pytest.raises(zb.ZoloError) as ex:
        zb.zolo_pd_async(handle, dev(sm.A), zb.opts(beta=0.0))          # beta estimated
    assert ex.value.code == -10
    with pytest.raises(zb.ZoloError):
        zb.zolo_pd_async(handle, dev(sm.A), zb.opts(beta=1e-4, alpha=0.0))


def test_async_reports_a_cholesky_breakdown(zb, handle):
    import torch
    sm = synth.square_geometric(128, 1e12, seed=9)
    _, _, pending = zb.zolo_pd_async(handle, dev(sm.A), zb.opts(beta=1e-12, r=8, force_qr=0))
    torch.cuda.synchronize()
    assert pending().status == 2   # ZOLO_ECHOL: no fallback without a round trip


def test_batched_estimates(zb, handle):
    mats = [synth.make_matrix(n, n, synth.geometric_sigma(n, k), seed=1060 + n)
            for n, k in ((96, 1e5), (160, 1e11))]
    os_ = [zb.opts(beta=float(sm.sigma[-1]), estimate=True) for sm in mats]
    Qps, Hs, infos, st = zb.zolo_pd_batched(handle, [dev(sm.A) for sm in mats], os_)
    assert st == 0
    for sm, q, h, inf in zip(mats, Qps, Hs, infos):
        bwd = zo.backward_error_pd(sm.A, q.cpu().numpy(), h.cpu().numpy())
        assert 0 < inf.bwd_est < 1e-13 and abs(inf.bwd_est - bwd) <= 0.5 * bwd + 1e-16
        assert 0 < inf.orth_est < 1e-13


def test_profile_reports_sm_time_within_device_time(zb, handle):
    # zolo_profile: per kernel class the summed device time and the SM-time (each
    # launch's time times the share of the GPU's block slots its blocks take): a
    # share is at most 1, so 0 < sm_ms <= ms; the QR panel of a 96-column matrix
    # runs on one CTA per shift, a small share
    sm = synth.square_geometric(96, 1e8, seed=1070)
    zb.profile(True)
    try:
        zb.zolo_pd(handle, dev(sm.A), zb.opts(beta=float(sm.sigma[-1]), r=3))
        st = zb.profile_read()
    finally:
        zb.profile(False)
    used = {k: v for k, v in st.items() if v["launches"]}
    assert "qr_panel" in used and "gemm_f64" in used
    for k, v in used.items():
        assert 0.0 < v["sm_ms"] <= v["ms"] * (1 + 1e-9), (k, v)
    assert used["qr_panel"]["sm_ms"] < 0.1 * used["qr_panel"]["ms"]
