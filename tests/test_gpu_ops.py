"""GPU whole-array operations (Sec. 4: SetToValue via apply, Listing 7; the expression
posArr(0) = velArr(1) - velArr(2), Listing 5): bit-exact against the oracle."""
import numpy as np
import pytest

import oracle
import paper_1710_03462_b300 as sx
import soax_inputs

pytestmark = pytest.mark.gpu

LISTING5 = [("id", "i32", 1, "N"), ("pos", "f64", 3, "P"), ("vel", "f64", 3, "V"), ("mass", "f32", 1, "M")]


@pytest.mark.parametrize("n", [1, 3, 17, 100003])
def test_fill_all_fields_and_one_field(n):
    d = soax_inputs.wide_set(n, 1)
    p = sx.Particles(sx.WIDE_SCHEMA, n)
    p.load(d)
    p.fill(42)  # soax.apply<SetToValue>(42) of Sec. 4.2.1
    g = p.numpy()
    for name, dt, nc, _ in sx.WIDE_SCHEMA:
        for a in g[name]:
            ref = oracle.fill(np.empty(n, a.dtype), 42)
            assert a.tobytes() == ref.tobytes(), name
    p.fill(0.1, field="vel")
    assert all(a.tobytes() == oracle.fill(np.empty(n, np.float32), 0.1).tobytes() for a in p.numpy()["vel"])
    assert np.all(p.numpy()["mass"][0] == 42)


def test_fill_rejects_unrepresentable_values():
    p = sx.Particles(sx.WIDE_SCHEMA, 10)
    for v in (0.5, 256.0, -1.0):  # not an integer / out of u8 range
        with pytest.raises(sx.SoaxError):
            p.fill(v)
    with pytest.raises(sx.SoaxError):
        p.fill(1e39, field="vel")


@pytest.mark.parametrize("n", [1, 5, 100003])
def test_listing5_expression_and_lincomb(n):
    rng = np.random.default_rng(n)
    d = {"id": [np.arange(n, dtype=np.int32)], "pos": [rng.standard_normal(n) for _ in range(3)],
         "vel": [rng.standard_normal(n) for _ in range(3)], "mass": [rng.random(n).astype(np.float32)]}
    p = sx.Particles(LISTING5, n)
    p.load(d)
    p.lincomb(("pos", 0), [(("vel", 1), 1.0), (("vel", 2), -1.0)])  # posArr(0) = velArr(1) - velArr(2)
    g = p.numpy()
    assert np.array_equal(g["pos"][0], d["vel"][1] - d["vel"][2])
    ref = oracle.lincomb(np.empty(n), [d["pos"][1], d["vel"][0], d["pos"][2]], [0.3, -1.7, 2.5], 0.125)
    p.lincomb(("pos", 1), [(("pos", 1), 0.3), (("vel", 0), -1.7), (("pos", 2), 2.5)], constant=0.125)
    assert p.numpy()["pos"][1].tobytes() == ref.tobytes()
    q = sx.Particles([("x", "f32", 3, "P"), ("v", "f32", 3, "V")], n)
    xs = [rng.standard_normal(n).astype(np.float32) for _ in range(3)]
    vs = [rng.standard_normal(n).astype(np.float32) for _ in range(3)]
    q.load({"x": xs, "v": vs})
    q.lincomb(("x", 2), [(("x", 2), 1.0), (("v", 2), 1e-2)])  # Eq. 1 as an expression
    ref = oracle.lincomb(np.empty(n, np.float32), [xs[2], vs[2]], [1.0, 1e-2])
    assert q.numpy()["x"][2].tobytes() == ref.tobytes()
    with pytest.raises(sx.SoaxError):
        p.lincomb(("pos", 0), [(("mass", 0), 1.0)])  # mixed types
