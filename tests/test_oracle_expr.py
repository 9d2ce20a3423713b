"""Pins of the oracle's whole-array expressions (orc_expr: the expression templates of
Sec. 4.2 as postfix programs) against an evaluator written here from the operations'
IEEE definitions: numpy scalar arithmetic of the compute type for + - * / and sqrt
(each correctly rounded), exact rational arithmetic rounded once for fma, C casts for the
loads.  Random programs over sources of every type, Listing 5's expression, and the
special values."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

F32, F64 = np.float32, np.float64


def _round_f32(q):
    """The binary32 nearest the rational q (ties to even), from exact comparisons."""
    f = F32(float(q))
    best = None
    for c in (f, np.nextafter(f, F32(np.inf)), np.nextafter(f, F32(-np.inf))):
        if not np.isfinite(c):
            continue
        d = abs(Fraction(float(c)) - q)
        key = (d, int(np.array(c, F32).view(np.uint32)) & 1)
        if best is None or key < best[0]:
            best = (key, c)
    return best[1]


def _fma(a, b, c, T):
    if not (np.isfinite(a) and np.isfinite(b) and np.isfinite(c)):
        return T(T(a) * T(b) + T(c)) if T is F64 else F32(F64(a) * F64(b) + F64(c))
    q = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    if q == 0:
        # The sign of an exact zero: +0 unless both a*b and c are -0 or negative zero sums.
        return T(T(a) * T(b) + T(c))
    return F64(float(q)) if T is F64 else _round_f32(q)


def _load(a, i, T):
    v = a[i]
    if T is F64:
        return F64(v) if a.dtype != np.int64 else F64(float(int(v)))
    return F32(v)


def reference(program, compute, out_dtype):
    """Element-by-element evaluation with numpy scalars of the compute type."""
    T = F32 if compute == "f32" else F64
    n = next(item[1].size for item in program if not isinstance(item, str) and item[0] == "load")
    out = np.empty(n, out_dtype)
    with np.errstate(all="ignore"):
        for i in range(n):
            st = []
            for item in program:
                name, arg = (item, None) if isinstance(item, str) else item
                if name == "load":
                    st.append(_load(arg, i, T))
                elif name == "const":
                    st.append(T(arg))
                elif name in ("neg", "abs", "sqrt"):
                    a = st.pop()
                    st.append({"neg": lambda x: -x, "abs": abs, "sqrt": np.sqrt}[name](a))
                elif name == "fma":
                    c, b, a = st.pop(), st.pop(), st.pop()
                    st.append(T(_fma(a, b, c, T)))
                else:
                    b, a = st.pop(), st.pop()
                    if name == "add":
                        st.append(a + b)
                    elif name == "sub":
                        st.append(a - b)
                    elif name == "mul":
                        st.append(a * b)
                    elif name == "div":
                        st.append(a / b)
                    elif name == "min":
                        st.append(a if a < b else b)
                    else:
                        st.append(a if a > b else b)
            assert len(st) == 1
            out[i] = st[0]
    return out


def same(x, y):
    """Bit-equal, except that every NaN equals every NaN (IEEE fixes no NaN payload)."""
    x, y = np.asarray(x), np.asarray(y)
    nan = np.isnan(x) & np.isnan(y)
    return bool(np.all((x.view(np.uint64 if x.dtype == np.float64 else np.uint32) ==
                        y.view(np.uint64 if y.dtype == np.float64 else np.uint32)) | nan))


def _sources(n, rng):
    return [rng.integers(-2 ** 31, 2 ** 31 - 1, n, dtype=np.int32),
            rng.integers(-2 ** 62, 2 ** 62, n, dtype=np.int64),
            rng.integers(0, 256, n, dtype=np.uint8),
            (rng.standard_normal(n) * 3).astype(np.float32),
            rng.standard_normal(n) * 1e3,
            np.abs(rng.standard_normal(n)) + 0.5]


def _random_program(rng, srcs, length):
    prog, depth = [], 0
    while len(prog) < length or depth != 1:
        choices = []
        if depth < 6:
            choices += ["load", "load", "const"]
        if depth >= 1:
            choices += ["neg", "abs", "sqrt"]
        if depth >= 2:
            choices += ["add", "sub", "mul", "div", "min", "max"]
        if depth >= 3:
            choices += ["fma"]
        if len(prog) >= length and depth > 1:
            choices = [c for c in choices if c not in ("load", "const", "neg", "abs", "sqrt")]
        op = choices[rng.integers(len(choices))]
        if op == "load":
            prog.append(("load", srcs[rng.integers(len(srcs))]))
            depth += 1
        elif op == "const":
            prog.append(("const", float(rng.choice([0.5, -2.0, 3.25, 1e-3, 7.0, 0.1]))))
            depth += 1
        elif op in ("neg", "abs", "sqrt"):
            prog.append(op)
        elif op == "fma":
            prog.append(op)
            depth -= 2
        else:
            prog.append(op)
            depth -= 1
    return prog


@pytest.mark.parametrize("compute,out", [("f64", np.float64), ("f32", np.float32), ("f64", np.float32),
                                         ("f32", np.float64)])
def test_random_programs_match_the_ieee_definition(compute, out):
    rng = np.random.default_rng(5)
    n = 64
    srcs = _sources(n, rng)
    for _ in range(12):
        prog = _random_program(rng, srcs, int(rng.integers(3, 14)))
        got = oracle.expr(prog, compute, out)
        want = reference(prog, compute, out)
        assert same(got, want), prog


def test_listing5_expression():
    """posArr(0) = velArr(1) - velArr(2) (Listing 5) with f32 velocities into an f64
    position: each f32 converts exactly, one binary64 subtraction."""
    rng = np.random.default_rng(1)
    v1, v2 = (rng.standard_normal(1000).astype(np.float32) for _ in range(2))
    got = oracle.expr([("load", v1), ("load", v2), "sub"], "f64", np.float64)
    assert same(got, v1.astype(np.float64) - v2.astype(np.float64))


def test_loads_round_to_the_compute_type():
    """A binary64 source in a binary32 program is rounded on load; an i64 source beyond
    2^53 in a binary64 program too (a skipped conversion would keep more bits)."""
    x = np.array([1.0 + 2.0 ** -40, math.pi, -1e-40], np.float64)
    got = oracle.expr([("load", x), ("const", 0.0), "add"], "f32", np.float64)
    assert same(got, x.astype(np.float32).astype(np.float64))
    k = np.array([2 ** 62 + 1, -(2 ** 60) - 3, 12345], np.int64)
    got = oracle.expr([("load", k)], "f64", np.float64)
    assert same(got, np.array([float(int(v)) for v in k]))


def test_fma_is_one_rounding():
    """a*b + c with a*b's low bits cancelling: fma keeps them, mul then add does not."""
    a = np.array([1.0 + 2.0 ** -30], np.float64)
    c = np.array([-(1.0 + 2.0 ** -29)], np.float64)
    fused = oracle.expr([("load", a), ("load", a), ("load", c), "fma"], "f64")
    split = oracle.expr([("load", a), ("load", a), "mul", ("load", c), "add"], "f64")
    assert fused[0] == 2.0 ** -60 and split[0] == 0.0


def test_special_values():
    a = np.array([1.0, -1.0, 0.0, -0.0, np.inf, np.nan, 4.0], np.float64)
    b = np.array([0.0, 0.0, 0.0, 1.0, np.inf, 1.0, -2.0], np.float64)
    for name in ("div", "min", "max", "sub"):
        prog = [("load", a), ("load", b), name]
        for compute, T in (("f64", np.float64), ("f32", np.float32)):
            assert same(oracle.expr(prog, compute, T), reference(prog, compute, T)), (name, compute)
    for name in ("sqrt", "abs", "neg"):
        prog = [("load", a), name]
        assert same(oracle.expr(prog, "f64"), reference(prog, "f64", np.float64)), name
    # min/max take the second operand when the comparison is false (NaN included)
    m = oracle.expr([("load", a), ("load", b), "min"], "f64")
    assert m[5] == 1.0 and m[0] == 0.0 and np.signbit(m[2]) == np.signbit(b[2])
