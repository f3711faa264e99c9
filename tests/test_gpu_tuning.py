"""r chosen by measurement (opts.r = ZOLO_R_TUNED) and the handle's tuning cache.

On one GPU the r shifted problems share the chip instead of running on r
process groups, so the fastest r is measured, not read off Table 1.  The tuned
call must give a result meeting the same invariants as any fixed r, record the r
it ran with, reuse it on the next call, and survive a save / load of the cache
(rejected when the file names another device or is malformed)."""
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


def dev(a):
    import torch
    return torch.from_numpy(np.asfortranarray(a)).cuda()


def _check(A, Qp, H):
    Qp, H = Qp.cpu().numpy(), H.cpu().numpy()
    assert zo.orthogonality(Qp) <= 1e-13
    assert zo.backward_error_pd(A, Qp, H) <= 1e-13
    assert np.array_equal(H, H.T)
    return Qp, H


def test_tuned_r_runs_caches_and_matches_oracle(zb, tmp_path):
    h = zb.Handle(0)
    try:
        sm = synth.make_matrix(256, 192, synth.geometric_sigma(192, 1e8), seed=41)
        beta = float(sm.sigma.min())
        o = zb.opts(beta=beta, r=zb.ZOLO_R_TUNED)
        assert zb.tuned_r(h, 256, 192, zb.ZOLO_FP64, beta) == 0
        Qp, H, info = zb.zolo_pd(h, dev(sm.A), o)
        r = zb.tuned_r(h, 256, 192, zb.ZOLO_FP64, beta)
        assert 1 <= r <= 8 and info.r == r
        Qp, H = _check(sm.A, Qp, H)
        Qo, Ho, io = zo.zolo_pd(sm.A, 1.0, beta, r=r)
        assert info.iters == io.iters
        s = np.sort(sm.sigma)
        assert np.max(np.abs(Qp - Qo)) <= 200 * zo.EPS / (s[0] + s[1])
        # the same key again: the cached r, no new tuning
        _, _, info2 = zb.zolo_pd(h, dev(sm.A), o)
        assert info2.r == r
        # another precision is another key
        assert zb.tuned_r(h, 256, 192, zb.ZOLO_SPLIT_BF16, beta) == 0
        # the cache round-trips through a file
        path = str(tmp_path / "tune.txt")
        zb.tune_save(h, path)
        h2 = zb.Handle(0)
        try:
            assert zb.tune_load(h2, path) == 0
            assert zb.tuned_r(h2, 256, 192, zb.ZOLO_FP64, beta) == r
            # a file from a device of another name, or malformed, is refused whole
            lines = open(path).read().splitlines()
            other = str(tmp_path / "other.txt")
            with open(other, "w") as f:
                f.write("zolo-tune 2 Some_Other_GPU\nr 512 512 0 8 3\n")
            assert zb.tune_load(h2, other) == 9   # ZOLO_EINVAL
            assert zb.tuned_r(h2, 512, 512, zb.ZOLO_FP64, 1e-8) == 0
            bad = str(tmp_path / "bad.txt")
            with open(bad, "w") as f:
                f.write(lines[0] + "\nr 64 64 0 2 5\nr 64 128 0 2 5\n")   # m < n
            assert zb.tune_load(h2, bad) == 9
            assert zb.tuned_r(h2, 64, 64, zb.ZOLO_FP64, 1e-2) == 0
            assert zb.tune_load(h2, str(tmp_path / "missing.txt")) == 8   # ZOLO_EIO
        finally:
            h2.close()
    finally:
        h.close()


def test_batched_uses_the_cached_r_else_table1(zb):
    h = zb.Handle(0)
    try:
        a = synth.make_matrix(128, 128, synth.geometric_sigma(128, 1e6), seed=42)
        b = synth.make_matrix(96, 64, synth.geometric_sigma(64, 1e10), seed=43)
        oa = zb.opts(beta=float(a.sigma.min()), r=zb.ZOLO_R_TUNED)
        ob = zb.opts(beta=float(b.sigma.min()), r=zb.ZOLO_R_TUNED)
        _, _, ia = zb.zolo_pd(h, dev(a.A), oa)       # tunes a's key only
        Qps, Hs, infos, st = zb.zolo_pd_batched(h, [dev(a.A), dev(b.A)], [oa, ob])
        assert st == 0
        assert infos[0].r == ia.r == zb.tuned_r(h, 128, 128, zb.ZOLO_FP64, oa.beta)
        assert infos[1].r == zb.schedule(ob.beta, 0)[2]
        for sm, q, hh in zip([a, b], Qps, Hs):
            _check(sm.A, q, hh)
    finally:
        h.close()


def test_svd_with_tuned_r(zb):
    h = zb.Handle(0)
    try:
        sm = synth.make_matrix(160, 160, synth.geometric_sigma(160, 1e4), seed=44)
        U, S, V, info = zb.zolo_svd(h, dev(sm.A), zb.opts(beta=float(sm.sigma.min()),
                                                             r=zb.ZOLO_R_TUNED))
        assert info.status == 0 and 1 <= info.r <= 8
        S = S.cpu().numpy()
        assert np.max(np.abs(S - np.sort(sm.sigma)[::-1])) <= 1e-12 * sm.sigma.max()
        U, V = U.cpu().numpy(), V.cpu().numpy()
        assert np.linalg.norm(sm.A - (U * S) @ V.T) <= 1e-13 * np.linalg.norm(sm.A) * math.sqrt(160)
    finally:
        h.close()
