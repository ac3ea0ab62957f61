"""Pins for the oracle's Philox generator and Gaussian compression matrix.

Philox4x32-10 is pinned to its published known-answer vectors; the Gaussian
matrix is pinned to the moments the paper states for GIID sampling (Sec. 3:
E ||Omega a||^2 = l ||a||^2 and V ||Omega a||^2 = 2 l ||a||^4) and to the
layout contract (prefix stability in l, independence of the stream id).
"""
import os

import numpy as np
import pytest

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(t, 16) for t in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    got = philox.philox4x32_10(np.array(ctr), np.array(key))
    assert [int(v) for v in got] == out


def test_unit_interval_open():
    lo = np.array([0, 0xFFFFFFFF], dtype=np.uint64)
    hi = np.array([0, 0xFFFFFFFF], dtype=np.uint64)
    u = philox.words_to_unit(lo, hi)
    assert u[0] == 2.0 ** -53
    assert u[1] < 1.0 and u[1] == 1.0 - 2.0 ** -53


def test_gaussian_moments():
    x = philox.gaussian_block(7, 64, 4096).ravel()
    n = x.size
    assert abs(x.mean()) < 5 / np.sqrt(n)
    assert abs(x.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    # fourth moment of N(0,1) is 3
    assert abs(np.mean(x ** 4) - 3.0) < 5 * np.sqrt(96.0 / n)


def test_prefix_stable_in_l():
    a = philox.gaussian_omega(3, 9, 50)
    b = philox.gaussian_omega(3, 16, 50)
    np.testing.assert_array_equal(a, b[:9])


def test_streams_and_seeds_differ():
    a = philox.gaussian_block(3, 4, 100, stream=1)
    b = philox.gaussian_block(3, 4, 100, stream=2)
    c = philox.gaussian_block(4, 4, 100, stream=1)
    assert np.abs(a - b).max() > 0.1 and np.abs(a - c).max() > 0.1


def test_sample_norm_chi_squared_law():
    """Sec. 3 / Sec. 3.1: for a fixed a, ||Omega a||^2 = x ||a||^2 with
    x ~ chi^2_l: mean l, variance 2 l."""
    ell, m, trials = 8, 40, 3000
    a = np.linspace(-1.0, 2.0, m)
    na2 = a @ a
    x = np.array([np.sum((philox.gaussian_omega(s, ell, m) @ a) ** 2) / na2
                  for s in range(trials)])
    assert abs(x.mean() - ell) < 5 * np.sqrt(2 * ell / trials)
    # variance of the sample variance of chi^2_l: (2 * (2l)^2/(n-1) + kappa4/n)
    assert abs(x.var() - 2 * ell) < 0.15 * 2 * ell
