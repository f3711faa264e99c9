"""CPU models of the FP64 one-sided Jacobi rounds' index and update arithmetic (no GPU).

One launch is one round: CTA i pairs the columns elem(i) and elem(n_even-1-i) of
a round-robin ordering with column 0 fixed and the others rotated by `round`.
Columns are stored scaled, x_p = d_p y_p, with their squared norms tracked, so a
rotation touches each row with two FMAs: y_p -= t (d_q / d_p) y_q,
y_q += t (d_p / d_q) y_p (with the old y_p), d_p, d_q *= c, and the squared
norms move by -/+ t g.  These models check that the ordering meets every pair
exactly once per sweep and that the scaled update is the textbook rotation.
"""
import itertools

import numpy as np
import pytest


def pairs_of_round(n_even, rnd):
    def elem(pos):
        return 0 if pos == 0 else 1 + (pos - 1 + rnd) % (n_even - 1)
    out = []
    for i in range(n_even // 2):
        p, q = elem(i), elem(n_even - 1 - i)
        out.append((min(p, q), max(p, q)))
    return out


@pytest.mark.parametrize("n", [2, 3, 8, 17, 64, 255])
def test_round_robin_meets_every_pair_once_per_sweep(n):
    n_even = n + (n & 1)
    seen = []
    for rnd in range(n_even - 1):
        prs = pairs_of_round(n_even, rnd)
        cols = [c for pq in prs for c in pq]
        assert len(set(cols)) == n_even            # a round touches each column once
        seen += [pq for pq in prs if pq[1] < n]    # pairs with the padding column are skipped
    assert sorted(seen) == sorted(itertools.combinations(range(n), 2))


def test_scaled_rotation_is_the_textbook_rotation():
    rng = np.random.default_rng(4)
    m = 50
    xp, xq = rng.standard_normal(m), rng.standard_normal(m) + 0.3 * rng.standard_normal(m)
    dp, dq = 0.7, 1.9                              # current column scales
    yp, yq = xp / dp, xq / dq
    a, b, g = xp @ xp, xq @ xq, xp @ xq
    zeta = (b - a) / (2 * g)
    t = np.sign(zeta) / (abs(zeta) + np.sqrt(1 + zeta * zeta))
    c = 1 / np.sqrt(1 + t * t)
    # the kernel's update
    yp2 = yp - t * (dq / dp) * yq
    yq2 = yq + t * (dp / dq) * yp
    dp2, dq2 = c * dp, c * dq
    a2, b2 = a - t * g, b + t * g
    xp2, xq2 = dp2 * yp2, dq2 * yq2
    # the textbook rotation that zeroes the cross product
    rp = c * (xp - t * xq)
    rq = c * (xq + t * xp)
    assert np.allclose(xp2, rp, atol=1e-14) and np.allclose(xq2, rq, atol=1e-14)
    assert abs(xp2 @ xq2) <= 1e-13 * np.sqrt(a * b)
    assert a2 == pytest.approx(xp2 @ xp2, rel=1e-13) and b2 == pytest.approx(xq2 @ xq2, rel=1e-13)
