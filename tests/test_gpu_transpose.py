"""GPU AoS <-> SoA transposes: byte-exact against the oracle, zero padding, round trip."""
import numpy as np
import pytest
import torch

import oracle
import paper_1710_03462_b300 as sx
import soax_inputs

pytestmark = pytest.mark.gpu

ES = {"i32": 4, "i64": 8, "u8": 1, "f32": 4, "f64": 8}
NP = {"i32": np.int32, "i64": np.int64, "u8": np.uint8, "f32": np.float32, "f64": np.float64}

ODD_SCHEMA = [("a", "u8", 1, "x"), ("b", "f64", 1, "y"), ("c", "u8", 3, "z"), ("d", "i32", 2, "w")]


def _odd_set(n, seed):
    rng = np.random.default_rng(seed)
    return {"a": [rng.integers(0, 256, n, dtype=np.uint8)], "b": [rng.standard_normal(n)],
            "c": [rng.integers(0, 256, n, dtype=np.uint8) for _ in range(3)],
            "d": [rng.integers(-2 ** 31, 2 ** 31 - 1, n).astype(np.int32) for _ in range(2)]}


CASES = [(sx.BASIC_SCHEMA, lambda n, s: soax_inputs.basic_set(n, s)),
         (sx.WIDE_SCHEMA, lambda n, s: soax_inputs.wide_set(n, s)),
         (ODD_SCHEMA, _odd_set)]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("n", [1, 127, 128, 129, 100003])
def test_transposes_vs_oracle(case, n):
    schema, gen = CASES[case]
    d = gen(n, n + case)
    eb = [ES[t] for _, t, _, _ in schema]
    nc = [c for _, _, c, _ in schema]
    planes = [a for name, _, _, _ in schema for a in d[name]]
    ref = oracle.soa_to_aos(planes, eb, nc)
    p = sx.Particles(schema, n)
    rb, offs = p.aos_layout()
    assert (rb, offs) == oracle.aos_layout(eb, nc)
    p.load(d)
    aos = torch.full((n * rb,), 0xAB, dtype=torch.uint8, device="cuda")  # garbage in the padding
    p.to_aos(aos)
    assert aos.cpu().numpy().tobytes() == ref.tobytes()
    # AoS -> SoA from records whose padding holds garbage.
    rec = ref.copy().reshape(n, rb)
    used = np.zeros(rb, bool)
    for (name, t, c, _), o in zip(schema, offs):
        used[o:o + ES[t] * c] = True
    rec[:, ~used] = 0x5C
    q = sx.Particles(schema, n)
    q.from_aos(torch.from_numpy(rec.reshape(-1)).cuda())
    back = oracle.aos_to_soa(rec.reshape(-1), eb, nc, [NP[t] for _, t, _, _ in schema])
    g = q.numpy()
    got = [a for name, _, _, _ in schema for a in g[name]]
    assert all(a.tobytes() == b.tobytes() for a, b in zip(got, back))
    assert all(a.tobytes() == b.tobytes() for a, b in zip(got, planes))


def test_full_size_sorted_n16M_round_trip():
    w = soax_inputs.WORKLOADS["sorted_n16M"]
    n = w["n"]
    d = soax_inputs.basic_set(n, w["seed"])
    p = sx.Particles(sx.BASIC_SCHEMA, n, shadow=False)
    p.load(d)
    aos = p.to_aos()
    idx = np.arange(0, n, 997)
    rec = aos.view(n, 48)[torch.from_numpy(idx).cuda()].cpu().numpy()
    sub = [np.ascontiguousarray(a[idx]) for name in ("id", "pos", "vel") for a in d[name]]
    assert rec.tobytes() == oracle.soa_to_aos(sub, [4, 8, 4], [1, 3, 3]).tobytes()
    before = [t.clone() for name in ("id", "pos", "vel") for t in p.field(name)]
    for name in ("id", "pos", "vel"):
        for t in p.field(name):
            t.zero_()
    p.from_aos(aos)
    after = [t for name in ("id", "pos", "vel") for t in p.field(name)]
    assert all(a.cpu().numpy().tobytes() == b.cpu().numpy().tobytes() for a, b in zip(before, after))
    del p, aos
    torch.cuda.empty_cache()
