"""Seeded synthetic inputs for the Zolo-PD / Zolo-SVD workloads.

This module only draws inputs; it holds none of the method's arithmetic, so the
CPU oracle and the CUDA path can both be fed from it without sharing any of the
computation under test.

Every matrix is A = U diag(sigma) V^T with U (m x n, orthonormal columns) and
V (n x n, orthogonal) Haar-distributed: the Q factor of a seeded N(0,1) matrix
with its columns multiplied by sign(diag R).  The paper's own test matrices
(SuiteSparse collection and its dense random rand1/rand2, Section 4) are not
available here; these stand in for them, with the condition numbers and
singular-value spreads of the workloads below.

Matrices are returned column-major (Fortran order), the layout of the C ABI.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class SynthMatrix:
    A: np.ndarray          # m x n, Fortran order
    U: np.ndarray          # m x n, orthonormal columns
    sigma: np.ndarray      # n, descending
    V: np.ndarray          # n x n, orthogonal
    seed: int

    @property
    def kappa(self) -> float:
        return float(self.sigma[0] / self.sigma[-1])


def haar_columns(rng: np.random.Generator, m: int, n: int) -> np.ndarray:
    """m x n matrix with Haar-distributed orthonormal columns."""
    g = rng.standard_normal((m, n))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d


def make_matrix(m: int, n: int, sigma: np.ndarray, seed: int) -> SynthMatrix:
    """A = U diag(sigma) V^T with seeded Haar U, V; sigma sorted descending."""
    sigma = np.sort(np.asarray(sigma, dtype=np.float64))[::-1].copy()
    assert sigma.shape == (n,) and m >= n
    rng = np.random.default_rng(seed)
    U = haar_columns(rng, m, n)
    V = haar_columns(rng, n, n)
    A = np.asfortranarray((U * sigma) @ V.T)
    return SynthMatrix(A=A, U=U, sigma=sigma, V=V, seed=seed)


def geometric_sigma(n: int, kappa: float) -> np.ndarray:
    return np.geomspace(1.0, 1.0 / kappa, n)


# ---------------------------------------------------------------------------
# The named workloads.  Seed = 1000 * workload number + matrix index.
# ---------------------------------------------------------------------------

def square_geometric(n: int = 256, kappa: float = 1e8, seed: int = 1000) -> SynthMatrix:
    """n x n, sigma geometric from 1 to 1/kappa (256^2 at kappa 1e8; 4096^2 at 1e12)."""
    return make_matrix(n, n, geometric_sigma(n, kappa), seed)


def tall_uniform(m: int = 16384, n: int = 4096, lo: float = 1e-6, seed: int = 3000) -> SynthMatrix:
    """m x n, sigma drawn uniform in [lo, 1] with sigma_1 = 1 and sigma_n = lo pinned."""
    rng = np.random.default_rng(seed + 500)
    s = rng.uniform(lo, 1.0, n)
    s[0], s[-1] = 1.0, lo
    return make_matrix(m, n, s, seed)


def clustered_square(n: int = 16384, cluster: int = 64, seed: int = 5000) -> SynthMatrix:
    """n x n, sigma geometric 1 .. 1e-16 on n - cluster values plus `cluster` values at 1e-3."""
    s = np.concatenate([np.geomspace(1.0, 1e-16, n - cluster), np.full(cluster, 1e-3)])
    return make_matrix(n, n, s, seed)


def clustered_square_device(n: int = 16384, cluster: int = 64, seed: int = 5000) -> SynthMatrix:
    """The clustered n x n workload drawn on the GPU (torch, seeded generator):
    the Haar factors of a 16384^2 matrix take minutes in numpy on the host.  Same
    spectrum as clustered_square; U and V are not kept (A only)."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)

    def haar(k):
        q, r = torch.linalg.qr(torch.randn(k, k, dtype=torch.float64, device="cuda", generator=g))
        d = torch.sign(torch.diagonal(r))
        d[d == 0] = 1.0
        return q * d

    s = np.concatenate([np.geomspace(1.0, 1e-16, n - cluster), np.full(cluster, 1e-3)])
    s = np.sort(s)[::-1].copy()
    U = haar(n)
    V = haar(n)
    A = (U * torch.from_numpy(s).cuda()) @ V.T
    del U, V
    A_host = np.asfortranarray(A.cpu().numpy())
    del A
    torch.cuda.empty_cache()
    return SynthMatrix(A=A_host, U=None, sigma=s, V=None, seed=seed)


def batch_sizes_and_kappas(count: int = 512, seed: int = 4000,
                           sizes=tuple(range(64, 1025, 64)),
                           log10_kappa=(2.0, 12.0)):
    """Per-matrix n drawn uniformly from `sizes`, kappa log-uniform over the range."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=count)
    kap = 10.0 ** rng.uniform(log10_kappa[0], log10_kappa[1], size=count)
    return [int(x) for x in ns], [float(k) for k in kap]


def batch(count: int = 512, seed: int = 4000, sizes=tuple(range(64, 1025, 64)),
          log10_kappa=(2.0, 12.0)):
    """The uneven batch: square matrices, n ~ U(sizes), sigma geometric over kappa."""
    ns, kap = batch_sizes_and_kappas(count, seed, sizes, log10_kappa)
    return [make_matrix(n, n, geometric_sigma(n, k), seed + 1 + i)
            for i, (n, k) in enumerate(zip(ns, kap))]
