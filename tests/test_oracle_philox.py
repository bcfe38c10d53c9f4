"""Pins for the oracle's counter-based Gaussian generator (Alg. 1 Omega).

P11: Philox4x32-10 against the published known-answer vectors; Box-Muller
against the N(0, 1) distribution (moments, Kolmogorov-Smirnov); stream and
element-index layout.
"""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox


def _kat(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[1:5], v[5:7], v[7:11]))
    return rows


def test_philox_known_answers(golden_dir):
    rows = _kat(golden_dir)
    assert len(rows) == 3
    for ctr, key, out in rows:
        got = philox.philox4x32_10(np.array([ctr], dtype=np.uint64),
                                   np.array(key, dtype=np.uint64))[0]
        assert [int(x) for x in got] == out


def test_philox_planted_mistake_is_caught(golden_dir):
    """A wrong multiplier constant must break the known-answer test."""
    ctr, key, out = _kat(golden_dir)[2]
    saved = philox.M1
    try:
        philox.M1 = np.uint64(0xCD9E8D59)
        got = philox.philox4x32_10(np.array([ctr], dtype=np.uint64),
                                   np.array(key, dtype=np.uint64))[0]
        assert [int(x) for x in got] != out
    finally:
        philox.M1 = saved


def test_gaussian_distribution():
    z = philox.gaussian_matrix(1234, 0, 500, 400).ravel()
    assert abs(z.mean()) < 5 * 1 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / z.size)
    assert abs(stats.skew(z)) < 0.02
    assert abs(stats.kurtosis(z)) < 0.04
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_layout_and_streams():
    # element e of a matrix is z_{e mod 4} of block e // 4, independent of
    # the matrix shape; streams 0 and 1 differ.
    a = philox.gaussian_matrix(99, 0, 7, 5).ravel()
    b = philox.gaussian_matrix(99, 0, 5, 7).ravel()
    assert np.array_equal(a, b)
    c = philox.gaussian_matrix(99, 1, 7, 5).ravel()
    assert not np.allclose(a, c)
    # block 3 of stream 0 drives elements 12..15
    w = philox.raw_words(99, 0, 1, first_block=3)[0].astype(np.float64)
    u = (w + 0.5) * 2.0 ** -32
    z0 = np.sqrt(-2 * np.log(u[0])) * np.cos(2 * np.pi * u[1])
    z3 = np.sqrt(-2 * np.log(u[2])) * np.sin(2 * np.pi * u[3])
    assert a[12] == pytest.approx(z0, rel=1e-15)
    assert a[15] == pytest.approx(z3, rel=1e-15)
    # seeds above 2^32 use the high key word
    hi = philox.gaussian_matrix((1 << 32) + 99, 0, 7, 5).ravel()
    assert not np.allclose(a, hi)
