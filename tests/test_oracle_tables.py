"""Pins of the oracle's 1D tables: Gauss rule, GLL nodes, Lagrange basis.

These are fixed by mathematics, not by the oracle itself: an n-point Gauss
rule integrates every polynomial of degree <= 2n-1 exactly and no more; the
interior GLL nodes of degree 3 are the roots +-1/sqrt(5) of P_3'; a nodal
Lagrange basis is the Kronecker delta at the nodes and reproduces every
polynomial of degree <= k.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_gauss_exact_to_degree_2n_minus_1(n):
    g, w = O.gauss_rule(n)
    assert np.all(np.diff(g) > 0) and g[0] > 0 and g[-1] < 1
    for m in range(2 * n):
        assert abs(np.sum(w * g ** m) - 1.0 / (m + 1)) < 2e-16 * 4
    # and not beyond: degree 2n is integrated with a visible error
    assert abs(np.sum(w * g ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-6


def test_gll_closed_forms():
    assert np.allclose(O.gll_nodes(1), [0.0, 1.0], atol=0, rtol=0)
    assert np.allclose(O.gll_nodes(2), [0.0, 0.5, 1.0], atol=1e-16)
    s = 1.0 / math.sqrt(5.0)             # roots of P_3'(s) = (15 s^2 - 3) / 2
    want = [0.0, 0.5 - 0.5 * s, 0.5 + 0.5 * s, 1.0]
    assert np.allclose(O.gll_nodes(3), want, atol=2e-16, rtol=0)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_lagrange_delta_partition_reproduction(k):
    z = O.gll_nodes(k)
    for b, zb in enumerate(z):
        l, _ = O.lagrange(k, zb)
        e = np.zeros(k + 1)
        e[b] = 1.0
        assert np.allclose(l, e, atol=1e-15)
    rng = np.random.default_rng(0)
    for t in rng.random(7):
        l, dl = O.lagrange(k, t)
        assert abs(l.sum() - 1.0) < 1e-14
        assert abs(dl.sum()) < 1e-12
        for m in range(k + 1):
            assert abs(np.sum(l * z ** m) - t ** m) < 1e-14
            dm = m * t ** (m - 1) if m else 0.0
            assert abs(np.sum(dl * z ** m) - dm) < 1e-12
