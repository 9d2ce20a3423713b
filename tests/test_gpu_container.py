"""GPU container operations (Listings 5-6, Sec. 2): one-element getElement / push_back,
resize within capacity, and removal by overwriting with the last particle -- bit-exact
against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_1710_03462_b300 as sx
import soax_inputs

pytestmark = pytest.mark.gpu

ES = {"i32": 4, "i64": 8, "u8": 1, "f32": 4, "f64": 8}


def _planes(d, schema):
    return [a for name, _, _, _ in schema for a in d[name]]


def test_get_and_set_element():
    n = 1000
    d = soax_inputs.wide_set(n, 3)
    p = sx.Particles(sx.WIDE_SCHEMA, n)
    p.load(d)
    eb = [ES[t] for _, t, _, _ in sx.WIDE_SCHEMA]
    nc = [c for _, _, c, _ in sx.WIDE_SCHEMA]
    ref = oracle.soa_to_aos(_planes(d, sx.WIDE_SCHEMA), eb, nc).reshape(n, 64)
    for i in (0, 1, 517, n - 1):
        assert p.get_element(i).cpu().numpy().tobytes() == ref[i].tobytes()
    p.set_element(5, p.get_element(900))
    g = p.numpy()
    for name in g:
        for a, b in zip(g[name], d[name]):
            exp = b.copy()
            exp[5] = b[900]
            assert np.array_equal(a, exp)
    with pytest.raises(sx.SoaxError):
        p.get_element(n)


def test_push_back_and_resize():
    cap = 64
    d = soax_inputs.basic_set(cap, 4)
    p = sx.Particles(sx.BASIC_SCHEMA, cap)
    p.load(d)
    p.set_size(10)
    q = sx.Particles(sx.BASIC_SCHEMA, 1)
    q.load({k: [a[40:41] for a in v] for k, v in d.items()})
    p.push_back(q.get_element(0))
    assert p.size == 11
    g = p.numpy()
    assert g["id"][0][10] == 40 and g["pos"][0][10] == d["pos"][0][40]
    with pytest.raises(sx.SoaxError):
        p.set_size(cap + 1)


@pytest.mark.parametrize("n,k", [(10, 1), (10, 10), (1000, 0), (1000, 37), (100003, 5000), (100003, 99000)])
def test_remove_by_overwrite_with_last(n, k):
    rng = np.random.default_rng(n + k)
    d = soax_inputs.wide_set(n, 5)
    idx = np.sort(rng.choice(n, k, replace=False)).astype(np.uint32)
    p = sx.Particles(sx.WIDE_SCHEMA, n)
    p.load(d)
    p.remove(torch.from_numpy(idx.view(np.int32)).cuda())
    sx.sync()
    assert p.size == n - k
    ref = oracle.remove(_planes(d, sx.WIDE_SCHEMA), idx)
    got = _planes(p.numpy(), sx.WIDE_SCHEMA)
    assert all(a.tobytes() == b.tobytes() for a, b in zip(got, ref))


def test_remove_rejects_unsorted_indices_without_moving():
    n = 100
    d = soax_inputs.basic_set(n, 6)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    p.load(d)
    p.remove(torch.tensor([5, 3], dtype=torch.int32, device="cuda"))
    with pytest.raises(sx.SoaxError):
        sx.sync()
    assert np.array_equal(p.numpy()["id"][0], d["id"][0][: n - 2])
