"""Pins of the oracle's ABC flow u(x) = (A sin z + C cos y, B sin x + A cos z,
C sin y + B cos x) against properties fixed by mathematics, not by retyping it:
exact values at special points, the Beltrami property curl u = u, zero divergence and
2pi periodicity.  A swapped coordinate, a wrong sign or a dropped term fails one of
these."""
import math

import numpy as np
import pytest

import oracle

A, B, C = 0.7, 1.3, 2.1
rng = np.random.default_rng(5)


def u(x, y, z, a=A, b=B, c=C):
    return np.array(oracle.flow(a, b, c, np.atleast_1d(x), np.atleast_1d(y), np.atleast_1d(z)))


def test_origin_exact():
    # sin 0 = 0, cos 0 = 1: u(0) = (C, A, B) exactly.
    for a, b, c in [(1.0, 1.0, 1.0), (0.7, 1.3, 2.1), (-2.0, 0.5, 3.25)]:
        got = u(0.0, 0.0, 0.0, a, b, c)[:, 0]
        assert got.tolist() == [c, a, b]


@pytest.mark.parametrize("pt,expect", [
    # (x, y, z) -> u, using sin(pi/2) = 1, cos(pi/2) = 0, sin(pi) = 0, cos(pi) = -1
    ((math.pi / 2, 0.0, 0.0), (C, B + A, 0.0)),
    ((0.0, math.pi / 2, 0.0), (0.0, A, C + B)),
    ((0.0, 0.0, math.pi / 2), (A + C, 0.0, B)),
    ((math.pi, math.pi, math.pi), (-C, -A, -B)),
])
def test_special_points(pt, expect):
    got = u(*pt)[:, 0]
    assert np.allclose(got, expect, atol=1e-15, rtol=0)


def _jac_fd(x, h=1e-5):
    J = np.zeros((3, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (u(*(x + e))[:, 0] - u(*(x - e))[:, 0]) / (2 * h)
    return J


def test_beltrami_curl_equals_u():
    for _ in range(20):
        x = rng.uniform(0, 2 * math.pi, 3)
        J = _jac_fd(x)  # J[i, k] = d u_i / d x_k
        curl = np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])
        assert np.allclose(curl, u(*x)[:, 0], atol=1e-9)


def test_divergence_free():
    for _ in range(20):
        x = rng.uniform(0, 2 * math.pi, 3)
        assert abs(np.trace(_jac_fd(x))) < 1e-9


def test_periodic():
    x = rng.uniform(0, 2 * math.pi, (3, 100))
    base = u(*x)
    for k in range(3):
        xs = x.copy()
        xs[k] += 2 * math.pi
        assert np.allclose(u(*xs), base, atol=1e-14, rtol=0)
