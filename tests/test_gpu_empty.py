"""Every call on an empty particle set (n = 0) succeeds and touches nothing, and the
batched step handles empty ensembles between non-empty ones."""
import numpy as np
import pytest
import torch

import paper_1710_03462_b300 as sx
import soax_inputs

pytestmark = pytest.mark.gpu


def test_every_call_on_an_empty_set():
    p = sx.Particles(sx.BASIC_SCHEMA, 0)
    f = sx.Flow()
    keys = p.cell_keys(32)
    assert keys.numel() == 0
    ws = p.sort_workspace(32)
    k1, p1 = p.sort_by_cell(32, ws)
    assert k1.numel() == 0 and p1.numel() == 0
    p.sort_by_keys(32, keys, ws)
    _, perm = p.sort_perm(32, keys, ws)
    p.permute(perm)
    p.step(f, 3)
    p.step_fused(f, 10, grid=32, keys=keys)
    p.step_fused(f, 10, grid=32, keys=keys, perm=perm)
    aos = p.to_aos()
    assert aos.numel() == 0
    p.from_aos(aos)
    p.step_aos(aos, f, 2)
    p.fill(2.0)              # every field (2.0 fits the i32 id too)
    p.fill(1.5, field="pos")
    p.lincomb(("vel", 0), [(("vel", 1), 1.0), (("vel", 2), -1.0)], 0.25)
    p.copy_plane("pos", 0, np.empty(0), True)
    p.copy_plane("vel", 2, np.empty(0, np.float32), False)
    sx.sync()
    q = sx.Particles([("x", "f32", 3, "P"), ("v", "f32", 3, "V")], 0, shadow=False)
    q.euler(1e-3)
    q.euler(1e-3, per_component=True)
    sx.sync()


def test_adjoint_on_an_empty_set():
    p = sx.Particles([("pos", "f64", 3, "P"), ("vel", "f32", 3, "V")], 0, shadow=False)
    f = sx.Flow()
    ws = p.adjoint_workspace(10, 4)
    p.step_checkpointed(f, 10, 4, ws)
    empty = [torch.empty(0, dtype=torch.float64, device="cuda") for _ in range(3)]
    xb0, vb0, g = p.step_adjoint(f, 10, 4, ws, empty)
    assert all(t.numel() == 0 for t in xb0 + vb0)
    assert np.all(g.cpu().numpy() == 0.0)
    sx.sync()


@pytest.mark.parametrize("fuse", [0, 1])
def test_batched_with_empty_ensembles(fuse):
    sizes = [0, 1000, 0, 77, 0]
    flows = [sx.Flow(A=1.1, tau=0.2), sx.Flow(), sx.Flow(B=0.8), sx.Flow(tau=0.05), sx.Flow()]
    parts, refs = [], []
    for e, ne in enumerate(sizes):
        d = soax_inputs.basic_set(ne, 40 + e)
        q = sx.Particles(sx.BASIC_SCHEMA, ne, shadow=False)
        q.load(d)
        parts.append(q)
        r = sx.Particles(sx.BASIC_SCHEMA, ne, shadow=False)
        r.load(d)
        (r.step_fused if fuse else r.step)(flows[e], 4)
        refs.append(r.numpy())
    sx.step_batched(parts, flows, 4, sx.Tune(2, 256, 128, fuse))
    sx.sync()
    for q, r in zip(parts, refs):
        g = q.numpy()
        for k in ("pos", "vel"):
            for a, b in zip(g[k], r[k]):
                assert a.tobytes() == b.tobytes()
