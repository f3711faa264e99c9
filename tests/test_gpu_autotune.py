"""Contraction kernels chosen by measurement (zolo_autotune) and each kernel variant.

Every variant the tuner may keep must compute the same product: each is forced in
turn through a tuning-cache file (a "g" line for one shape) and compared with the
CPU product, including split-K on the Gram matrix (upper tiles only) and on the
batch-reduced triangular product of the inverse Cholesky form.  A decomposition
with tuning on must meet the usual invariants and match the oracle."""
import math

import numpy as np
import pytest

from oracle import zolo_oracle as zo
from paper_1806_06204_gb300 import synth

pytestmark = pytest.mark.gpu

VARIANTS = [0, 1, 2, 3, 4, 5]   # 64x64, 32x128, 32x64, split-K 2, 4, 8


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


def header(zb, tmp_path):
    h = zb.Handle(0)
    try:
        p = str(tmp_path / "empty.txt")
        zb.tune_save(h, p)
        return open(p).read().splitlines()[0]
    finally:
        h.close()


def forced(zb, tmp_path, head, lines):
    p = str(tmp_path / "forced.txt")
    with open(p, "w") as f:
        f.write(head + "\n" + "".join(l + "\n" for l in lines))
    h = zb.Handle(0)
    assert zb.tune_load(h, p) == 0
    return h


@pytest.mark.parametrize("v", VARIANTS)
@pytest.mark.parametrize("m,n,k,ta,beta", [(70, 45, 1000, 0, 0.0), (200, 33, 515, 1, 0.5),
                                           (31, 300, 257, 0, -1.0)])
def test_each_fp64_variant_matches_numpy(zb, tmp_path, v, m, n, k, ta, beta):
    head = header(zb, tmp_path)
    flags = ta | (32 if beta != 0.0 else 0)
    h = forced(zb, tmp_path, head, [f"g {m} {n} {k} 1 {flags} 0 {v}"])
    try:
        rng = np.random.default_rng(m + n + k + v)
        A = rng.standard_normal((k, m) if ta else (m, k))
        B = rng.standard_normal((k, n))
        C0 = rng.standard_normal((m, n))
        C = dev(C0)
        zb.zolo_dgemm(h, dev(A), dev(B), C, alpha=1.5, beta=beta, transA=bool(ta))
        ref = 1.5 * ((A.T if ta else A) @ B) + beta * C0
        assert np.max(np.abs(C.cpu().numpy() - ref)) <= 1e-13 * k * np.max(np.abs(ref))
    finally:
        h.close()


@pytest.mark.parametrize("v", [3, 4, 5, 2])
def test_forced_split_k_in_the_cholesky_iteration(zb, tmp_path, v):
    # Gram (M = N = n, K = m, transA, upper tiles: flags 17) and the inverse form's
    # W = sum_j a_j R_j^{-1} R_j^{-T} (M = N = K = n, batch r, transB | reduce |
    # b_lower | c_upper: flags 30) forced onto variant v
    m, n, r = 400, 150, 4
    head = header(zb, tmp_path)
    lines = [f"g {n} {n} {m} 1 17 0 {v}", f"g {n} {n} {n} {r} 30 0 {v}"]
    if v != 2:
        # the Cholesky panel update Rinv_kk^T panel is computed in place (flag 128):
        # split-K may serve it, a 32-row tile may not
        lines.append(f"g 64 86 64 {r} 129 0 {v}")
    h = forced(zb, tmp_path, head, lines)
    try:
        sm = synth.make_matrix(m, n, synth.geometric_sigma(n, 30.0), seed=5)
        o = zb.opts(beta=1.0 / 30.0, r=r, max_iter=1, force_qr=0, chol_form=2)
        X1, _, info = zb.zolo_pd(h, dev(sm.A), o)
        ref = zo.zolo_step_chol(sm.A, zo.zolotarev_coeffs(1.0 / 30.0, r))
        assert info.iters == 1 and info.chol_form == 2
        assert np.linalg.norm(X1.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-13
    finally:
        h.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_pd_with_autotune_matches_oracle_and_saves(zb, tmp_path, prec):
    h = zb.Handle(0)
    try:
        zb.autotune(h, True)
        sm = synth.make_matrix(320, 200, synth.geometric_sigma(200, 1e8), seed=6)
        beta = float(sm.sigma[-1])
        o = zb.opts(beta=beta, r=4, prec=prec, ns_steps=1 if prec else 0)
        Qp, H, info = zb.zolo_pd(h, dev(sm.A), o)
        Qo, Ho, io = zo.zolo_pd(sm.A, 1.0, beta, r=4, ns_steps=1 if prec else 0)
        Qp, H = Qp.cpu().numpy(), H.cpu().numpy()
        assert info.iters == io.iters
        assert zo.orthogonality(Qp) <= 1e-13 and zo.backward_error_pd(sm.A, Qp, H) <= 1e-13
        assert np.array_equal(H, H.T)
        assert np.linalg.norm(H - Ho) <= 1e-12 * np.linalg.norm(Ho)
        s = np.sort(sm.sigma)
        assert np.max(np.abs(Qp - Qo)) <= 200 * zo.EPS / (s[0] + s[1])
        p = str(tmp_path / "tuned.txt")
        zb.tune_save(h, p)
        glines = [l for l in open(p).read().splitlines() if l.startswith("g ")]
        assert len(glines) >= 5
        kernels = {int(l.split()[-1]) for l in glines}
        assert kernels <= {0, 1, 2, 3, 4, 5, 8}
        if prec:
            assert any(int(l.split()[6]) == 9 for l in glines)   # shapes keyed with 9 slices
        # tuning off: the choices stay, a second call gives the same bits
        zb.autotune(h, False)
        Qp2, H2, _ = zb.zolo_pd(h, dev(sm.A), o)
        assert np.array_equal(Qp2.cpu().numpy(), Qp) and np.array_equal(H2.cpu().numpy(), H)
        # the file reloads into a new handle
        h2 = zb.Handle(0)
        try:
            assert zb.tune_load(h2, p) == 0
            Qp3, H3, _ = zb.zolo_pd(h2, dev(sm.A), o)
            assert np.array_equal(Qp3.cpu().numpy(), Qp)
        finally:
            h2.close()
    finally:
        h.close()


def test_autotune_argument_checks(zb, tmp_path):
    import ctypes
    assert zb.LIB.zolo_autotune(ctypes.c_void_p(), 1) == -1
    h = zb.Handle(0)
    try:
        assert zb.LIB.zolo_autotune(h.ptr, 2) == -2
        head = header(zb, tmp_path)
        bad = str(tmp_path / "bad.txt")
        for line in ["g 10 10 10 1 0 0 7", "g 10 10 10 17 0 0 0", "g 10 10 10 1 0 0 8",
                     "x 1 2 3", "g 10 10", "g 64 86 64 4 129 0 2"]:
            with open(bad, "w") as f:
                f.write(head + "\n" + line + "\n")
            assert zb.tune_load(h, bad) == 9, line
    finally:
        h.close()


def test_in_place_product_keeps_a_safe_kernel(zb):
    # C <- A C with C = B (M = K = 64, many column tiles): a 32-row tile would let one
    # CTA overwrite rows of B that the other row tile still reads; with tuning on only
    # the built-in 64-row tile and split-K are candidates
    import torch
    h = zb.Handle(0)
    try:
        zb.autotune(h, True)
        rng = np.random.default_rng(9)
        A = rng.standard_normal((64, 64))
        B0 = rng.standard_normal((64, 3000))
        for _ in range(2):   # the first call tunes, the second uses the kept kernel
            C = dev(B0)
            zb.zolo_dgemm(h, dev(A), C, C)
            assert np.max(np.abs(C.cpu().numpy() - A @ B0)) <= 1e-12
    finally:
        h.close()


def test_batched_call_with_tuning_equals_tuned_single_calls(zb):
    # zolo_autotune on: the batched call measures the shapes of one matrix per
    # configuration before its lanes start, and the lanes replay those choices,
    # each with its own split-K scratch; FP64 single calls on the same handle then
    # use the same kernels and agree bit for bit (m < 512: the same panel kernel)
    from paper_1806_06204_gb300 import synth
    h = zb.Handle(0)
    try:
        zb.autotune(h, True)
        specs = [(200, 150, 1e6), (96, 96, 1e10), (300, 120, 40.0), (200, 150, 3e5)]
        mats = [synth.make_matrix(m, n, synth.geometric_sigma(n, k), seed=1070 + i)
                for i, (m, n, k) in enumerate(specs)]
        As = [dev(sm.A) for sm in mats]
        os_ = [zb.opts(beta=float(sm.sigma[-1])) for sm in mats]
        Qps, Hs, infos, st = zb.zolo_pd_batched(h, As, os_)
        assert st == 0
        first = [(q.cpu().numpy().copy(), x.cpu().numpy().copy()) for q, x in zip(Qps, Hs)]
        for sm, a, o, (q, x) in zip(mats, As, os_, first):
            assert zo.orthogonality(q) < 1e-13 and zo.backward_error_pd(sm.A, q, x) < 1e-13
            q1, h1, _ = zb.zolo_pd(h, a, o)
            assert np.array_equal(q, q1.cpu().numpy()) and np.array_equal(x, h1.cpu().numpy())
        # the tuned graph is replayed with the same bits
        zb.autotune(h, False)
        _, _, _, st2 = zb.zolo_pd_batched(h, As, os_, Qps=Qps, Hs=Hs)
        assert st2 == 0
        for (q, x), q2, x2 in zip(first, Qps, Hs):
            assert np.array_equal(q, q2.cpu().numpy()) and np.array_equal(x, x2.cpu().numpy())
    finally:
        h.close()
