"""GPU whole-array expressions (soax_expr: the expression templates of Sec. 4.2 as
postfix programs run in one pass) bit-exact against the oracle's evaluator: random
programs over every field type of the wide record in binary32 and binary64 arithmetic,
into f32 and f64 planes, at ragged sizes that span several tiles; Listing 5's assignment;
a destination that is also a source; special values."""
import numpy as np
import pytest

import oracle
import paper_1710_03462_b300 as sx
import soax_inputs

pytestmark = pytest.mark.gpu

EXTRA = [("id", "i64", 1, "N"), ("pos", "f64", 3, "P"), ("vel", "f32", 3, "V"), ("acc", "f32", 3, "A"),
         ("mass", "f32", 1, "M"), ("tag", "u8", 1, "T"), ("k", "i32", 1, "K")]


def _set(n, seed):
    d = soax_inputs.wide_set(n, seed)
    rng = np.random.default_rng(seed + 99)
    d["acc"] = [rng.standard_normal(n).astype(np.float32) * 10 for _ in range(3)]
    d["id"] = [rng.integers(-2 ** 62, 2 ** 62, n, dtype=np.int64)]
    d["k"] = [rng.integers(-2 ** 31, 2 ** 31 - 1, n, dtype=np.int32)]
    return d


def _same(x, y):
    nan = np.isnan(x) & np.isnan(y)
    u = np.uint64 if x.dtype == np.float64 else np.uint32
    return bool(np.all((x.view(u) == y.view(u)) | nan))


def _random_program(rng, fields, length):
    prog, depth = [], 0
    while len(prog) < length or depth != 1:
        choices = []
        if depth < 8:
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
            name, nc = fields[rng.integers(len(fields))]
            prog.append(("load", name, int(rng.integers(nc))))
            depth += 1
        elif op == "const":
            prog.append(("const", float(rng.choice([0.5, -2.0, 3.25, 1e-3, 7.0, 0.1, 1e300]))))
            depth += 1
        elif op in ("neg", "abs", "sqrt"):
            prog.append(op)
        else:
            prog.append(op)
            depth -= 2 if op == "fma" else 1
    return prog


def _oracle_program(prog, d):
    return [("load", d[it[1]][it[2]]) if isinstance(it, tuple) and it[0] == "load" else it for it in prog]


@pytest.mark.parametrize("n", [1, 3, 4097, 100003])
@pytest.mark.parametrize("compute", ["f32", "f64"])
def test_random_programs(n, compute):
    d = _set(n, n % 1000)
    p = sx.Particles(EXTRA, n)
    p.load(d)
    rng = np.random.default_rng(n * 7 + (compute == "f32"))
    fields = [(name, nc) for name, _, nc, _ in EXTRA]
    for t in range(6):
        prog = _random_program(rng, fields, int(rng.integers(3, 20)))
        dst = ("pos", t % 3) if t % 2 == 0 else ("acc", t % 3)
        p.expr(dst, prog, compute)
        got = p.numpy()[dst[0]][dst[1]]
        want = oracle.expr(_oracle_program(prog, d), compute, got.dtype, n=n)
        assert _same(got, want), prog
        d[dst[0]][dst[1]] = got  # the next program may read it


def test_listing5_assign_and_aliasing():
    n = 70001
    d = _set(n, 3)
    p = sx.Particles(EXTRA, n)
    p.load(d)
    p.assign("pos[0] = vel[1] - vel[2]")  # Listing 5, f32 velocities into an f64 position
    g = p.numpy()
    assert _same(g["pos"][0], d["vel"][1].astype(np.float64) - d["vel"][2].astype(np.float64))
    p.assign("vel[0] = vel[0] * mass / (1 + tag) + sqrt(abs(acc[2]))", compute="f32")
    want = oracle.expr([("load", d["vel"][0]), ("load", d["mass"][0]), "mul", ("const", 1.0), ("load", d["tag"][0]),
                        "add", "div", ("load", d["acc"][2]), "abs", "sqrt", "add"], "f32", np.float32)
    assert _same(p.numpy()["vel"][0], want)
    p.assign("pos[2] = fma(pos[2], 0.5, id) - min(k, 3) + max(pos[1], -1)")
    want = oracle.expr([("load", d["pos"][2]), ("const", 0.5), ("load", d["id"][0]), "fma", ("load", d["k"][0]),
                        ("const", 3.0), "min", "sub", ("load", d["pos"][1]), ("const", -1.0), "max", "add"], "f64")
    assert _same(p.numpy()["pos"][2], want)


def test_special_values():
    n = 8
    a = np.array([1.0, -1.0, 0.0, -0.0, np.inf, np.nan, 4.0, 1e-310])
    b = np.array([0.0, 0.0, 0.0, 1.0, np.inf, 1.0, -2.0, 3.0])
    p = sx.Particles([("a", "f64", 1, "A"), ("b", "f64", 1, "B"), ("r", "f64", 1, "R"), ("s", "f32", 1, "S")], n)
    p.load({"a": [a], "b": [b]})
    for op in ("div", "min", "max", "sub", "mul"):
        for compute, dst in (("f64", "r"), ("f32", "s")):
            p.expr((dst, 0), [("load", "a", 0), ("load", "b", 0), op], compute)
            got = p.numpy()[dst][0]
            want = oracle.expr([("load", a), ("load", b), op], compute, got.dtype)
            assert _same(got, want), (op, compute)
    for op in ("sqrt", "abs", "neg"):
        p.expr(("r", 0), [("load", "a", 0), op], "f64")
        assert _same(p.numpy()["r"][0], oracle.expr([("load", a), op], "f64")), op


def test_invalid_programs_are_rejected_before_any_launch():
    p = sx.Particles(EXTRA, 100)
    for prog in ([("load", "pos", 0), "add"], [("const", 1.0), ("const", 2.0)], ["neg"], [],
                 [("const", 1.0)] * 17 + ["add"] * 16):
        with pytest.raises(sx.SoaxError):
            p.expr(("pos", 0), prog)
    with pytest.raises(sx.SoaxError):
        p.expr(("tag", 0), [("const", 1.0)])  # integer destination
    with pytest.raises(sx.SoaxError):
        p.expr(("pos", 3), [("const", 1.0)])
