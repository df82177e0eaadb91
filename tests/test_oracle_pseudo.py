"""Pins of the oracle's pseudo-data generator (CPU): the Philox4x32-10
known-answer vectors of the generator's reference implementation, the
inversion's exact boundary cases, and the empirical distribution of many
draws against the exact Poisson law."""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def kat_rows():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert list(oracle.philox4x32_10(ctr, key)) == expect


@pytest.mark.parametrize("mu", [0.3, 3.7, 42.0, 250.0])
def test_inversion_boundaries(mu):
    em = math.exp(-mu)
    F1 = em + em * mu
    assert oracle.poisson_inv(mu, 0.0) == 0
    assert oracle.poisson_inv(mu, em) == 0  # F(0) >= u
    assert oracle.poisson_inv(mu, np.nextafter(em, 2.0)) == 1
    assert oracle.poisson_inv(mu, F1) in (1, 2)  # rounding of F(1) as summed
    assert oracle.poisson_inv(0.0, 0.999999) == 0


def test_inversion_is_monotone_in_u():
    us = np.linspace(0.0, 0.999999, 2001)
    ks = [oracle.poisson_inv(17.5, u) for u in us]
    assert all(b >= a for a, b in zip(ks, ks[1:]))
    assert ks[0] == 0 and ks[-1] > 30


@pytest.mark.parametrize("mu", [3.7, 42.0, 1234.5])
def test_draws_follow_the_poisson_law(mu):
    # (1234.5 is drawn as the sum of three parts of mean 411.5)
    # 200000 draws of one bin; chi-square of the counts against the exact pmf
    # (computed here by the recurrence in log space), bins of expected count >= 50
    n = 200000
    x = oracle.pseudo_data([mu], n, seed=12345)[:, 0].astype(np.int64)
    assert abs(x.mean() - mu) < 5 * math.sqrt(mu / n)
    assert abs(x.var() - mu) < 6 * mu * math.sqrt(2.0 / n) + 0.02 * mu
    kmax = int(mu + 12 * math.sqrt(mu) + 12)
    logp = np.array([-mu + k * math.log(mu) - math.lgamma(k + 1) for k in range(kmax + 1)])
    expect = n * np.exp(logp)
    counts = np.bincount(np.minimum(x, kmax), minlength=kmax + 1)[: kmax + 1].astype(float)
    keep = expect >= 50
    chi2 = float((((counts - expect) ** 2) / expect)[keep].sum())
    dof = int(keep.sum()) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof), (chi2, dof)


def test_data_sets_are_independent_of_their_order():
    mu = np.linspace(0.0, 300.0, 37)
    a = oracle.pseudo_data(mu, 10, seed=7)
    b = oracle.pseudo_data(mu, 4, seed=7, j0=6)
    assert np.array_equal(a[6:], b)
    assert np.all(a[:, 0] == 0) and np.all(a == np.round(a))
    assert not np.array_equal(a, oracle.pseudo_data(mu, 10, seed=8))
