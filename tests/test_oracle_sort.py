"""Pins of the oracle's cell keys, stable argsort and permute: exact rational floor
division away from cell boundaries and correctly rounded rational arithmetic at them,
brute-force O(N^2) stable selection, numpy's stable sort, and the sort
invariants (keys nondecreasing, perm a bijection, equal keys keep their order, every
field permuted alike)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import soax_inputs

TWO_PI = soax_inputs.TWO_PI


def test_keys_in_range():
    d = soax_inputs.basic_set(20000, 3)
    for G in (1, 2, 7, 32, 64):
        k = oracle.cell_keys(*d["pos"], G)
        assert k.max() < G ** 3
        if G == 1:
            assert np.all(k == 0)


def test_keys_exact_floor_away_from_boundaries():
    rng = np.random.default_rng(4)
    G = 32
    pts = rng.uniform(0, TWO_PI, (3, 3000))
    two_pi = Fraction(TWO_PI)
    keep = []
    exp = []
    for i in range(pts.shape[1]):
        idx, ok = [], True
        for c in range(3):
            q = Fraction(float(pts[c, i])) * G / two_pi
            fl = q.numerator // q.denominator
            if not (Fraction(1, 100) < q - fl < Fraction(99, 100)):
                ok = False
            idx.append(min(fl, G - 1))
        if ok:
            keep.append(i)
            exp.append((idx[2] * G + idx[1]) * G + idx[0])
    p = pts[:, keep]
    k = oracle.cell_keys(np.ascontiguousarray(p[0]), np.ascontiguousarray(p[1]), np.ascontiguousarray(p[2]), G)
    assert len(keep) > 2500
    assert k.tolist() == exp


def test_keys_boundaries():
    G = 64
    below = np.nextafter(TWO_PI, 0.0)
    x = np.array([0.0, below, 0.0, 0.0])
    y = np.array([0.0, 0.0, below, 0.0])
    z = np.array([0.0, 0.0, 0.0, below])
    k = oracle.cell_keys(x, y, z, G)
    assert k.tolist() == [0, G - 1, (G - 1) * G, (G - 1) * G * G]


def test_keys_at_cell_boundaries_exact_rounding():
    """Within a few ulps of cell boundaries the key is floor(RN(x RN(G / 2pi))): two
    binary64 roundings, taken here with exact rational arithmetic (Python's Fraction
    converts to the correctly rounded double), independently of the oracle's code.  A
    key that skipped either rounding (x c in extended precision, or c = G / 2pi kept
    exact) differs from this at some of these points."""
    for G in (32, 64, 7):
        c = float(Fraction(G) / Fraction(TWO_PI))           # RN(G / 2pi)
        xs = []
        for k in range(1, G):
            x0 = float(Fraction(k) / Fraction(c))            # nearest double to the boundary k / c
            x = x0
            for _ in range(4):
                x = np.nextafter(x, 0.0)
            for _ in range(9):                               # x0 - 4 ulp .. x0 + 4 ulp
                xs.append(x)
                x = np.nextafter(x, 8.0)
        xs = np.array(xs)
        exp = [min(int(float(Fraction(float(x)) * Fraction(c))), G - 1) for x in xs]  # floor(RN(x c))
        zeros = np.zeros_like(xs)
        assert oracle.cell_keys(xs, zeros, zeros, G).tolist() == exp
        assert oracle.cell_keys(zeros, xs, zeros, G).tolist() == [e * G for e in exp]
        assert oracle.cell_keys(zeros, zeros, xs, G).tolist() == [e * G * G for e in exp]
        # Both sides of every boundary occur, so the points do test the rounding.
        assert len(set(exp)) == G


def _selection_stable(keys):
    n = len(keys)
    used = [False] * n
    out = []
    for _ in range(n):
        best = None
        for i in range(n):  # first (lowest index) among the minimal keys
            if not used[i] and (best is None or keys[i] < keys[best]):
                best = i
        used[best] = True
        out.append(best)
    return out


@pytest.mark.parametrize("n", [0, 1, 2, 17, 64])
def test_argsort_brute_force(n):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 5, n).astype(np.uint32)
    perm, sk = oracle.stable_argsort(keys)
    assert perm.tolist() == _selection_stable(keys.tolist())
    assert sk.tolist() == sorted(keys.tolist())


def test_argsort_large_invariants():
    rng = np.random.default_rng(9)
    keys = rng.integers(0, 2 ** 15, 200000).astype(np.uint32)
    perm, sk = oracle.stable_argsort(keys)
    assert np.array_equal(perm, np.argsort(keys, kind="stable").astype(np.uint32))
    assert np.all(np.diff(sk.astype(np.int64)) >= 0)
    assert np.array_equal(np.sort(perm), np.arange(200000, dtype=np.uint32))
    same = sk[1:] == sk[:-1]
    assert np.all(perm[1:][same] > perm[:-1][same])  # stability


def test_permute_all_fields():
    d = soax_inputs.wide_set(5000, 2)
    planes = d["id"] + d["pos"] + d["vel"] + d["acc"] + d["mass"] + d["tag"]
    keys = oracle.cell_keys(*d["pos"], 64)
    perm, _ = oracle.stable_argsort(keys)
    out = oracle.permute(planes, perm)
    for a, b in zip(planes, out):
        assert np.array_equal(a[perm.astype(np.int64)], b)
    assert np.array_equal(np.sort(out[0]), d["id"][0])  # id multiset preserved
    k2 = oracle.cell_keys(out[1], out[2], out[3], 64)
    assert np.all(np.diff(k2.astype(np.int64)) >= 0)
    same = k2[1:] == k2[:-1]
    assert np.all(out[0][1:][same] > out[0][:-1][same])  # ids increase inside a key run
