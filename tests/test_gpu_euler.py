"""GPU Euler step (Eq. 1) on SoA planes (fused and per component) and on Listing 4's
AoS_SIZE records: bit-exact against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_1710_03462_b300 as sx

pytestmark = pytest.mark.gpu

SCHEMA = [("x", "f32", 3, "P"), ("v", "f32", 3, "V")]


@pytest.mark.parametrize("n", [1, 3, 4, 5, 1023, 100003])
@pytest.mark.parametrize("per_component", [False, True])
def test_euler_soa(n, per_component):
    rng = np.random.default_rng(n)
    x = [rng.standard_normal(n).astype(np.float32) for _ in range(3)]
    v = [rng.standard_normal(n).astype(np.float32) for _ in range(3)]
    p = sx.Particles(SCHEMA, n, shadow=False)
    p.load({"x": x, "v": v})
    for _ in range(3):
        p.euler(1e-2, per_component=per_component)
    ref = [a.copy() for a in x]
    for _ in range(3):
        for c in range(3):
            oracle.euler_f32(ref[c], v[c], 1e-2)
    g = p.numpy()
    for c in range(3):
        assert g["x"][c].tobytes() == ref[c].tobytes()
        assert g["v"][c].tobytes() == v[c].tobytes()


@pytest.mark.parametrize("size", [0, 1, 5, 32])
def test_euler_aos_listing4(size):
    n = 50001
    rng = np.random.default_rng(size)
    planes = [rng.standard_normal(n).astype(np.float32) for _ in range(6 + size)]
    ncomp = [3, 3] + ([size] if size else [])
    eb = [4] * len(ncomp)
    rec = oracle.soa_to_aos(planes, eb, ncomp)
    rb, offs = oracle.aos_layout(eb, ncomp)
    dev = torch.from_numpy(rec.copy()).cuda()
    sx.euler_aos(dev, n, rb, offs[0], offs[1], 1e-2)
    oracle.euler_aos_f32(rec, rb, offs[0], offs[1], 1e-2)
    assert dev.cpu().numpy().tobytes() == rec.tobytes()
