"""One handle beyond 2^28 particles (300,000,000): past the point where 32-bit byte
offsets of 8-byte elements would overflow.  The fused step with keys, the radix sort of
the keys and the fused step with the permute-gather, checked on sampled particles (the
last ones included) against the oracle, with the permutation checked as a bijection that
sorts the keys."""
import numpy as np
import pytest
import torch

import oracle
import paper_1710_03462_b300 as sx
from parity import assert_parity_fused

pytestmark = pytest.mark.gpu

N = 300_000_000
GRID, STEPS = 32, 10


def test_fused_sort_gather_beyond_2_28():
    torch.manual_seed(0)
    p = sx.Particles(sx.BASIC_SCHEMA, N)
    below = float(np.nextafter(sx.TWO_PI, 0.0))
    for t in p.field("pos"):
        t.uniform_(0.0, sx.TWO_PI).clamp_(max=below)
    for t in p.field("vel"):
        t.normal_(0.0, 0.1)
    p.field("id")[0].copy_(torch.arange(N, dtype=torch.int32, device="cuda"))
    rng = np.random.default_rng(1)
    idx = np.unique(np.concatenate([rng.integers(0, N, 200), np.arange(N - 100, N)]))
    it = torch.from_numpy(idx).cuda()
    x0 = [t[it].cpu().numpy() for t in p.field("pos")]
    v0 = [t[it].cpu().numpy() for t in p.field("vel")]
    f = sx.Flow()
    keys = p.step_fused(f, STEPS, grid=GRID)
    g = [t[it].cpu().numpy() for t in p.field("pos")], [t[it].cpu().numpy() for t in p.field("vel")]
    opos, ovel = [a.copy() for a in x0], [a.copy() for a in v0]
    oracle.step_soa(opos, ovel, 1.0, 1.0, 1.0, 0.1, 1e-3, STEPS)
    assert_parity_fused(g[0], g[1], opos, ovel, x0, v0, np.full(idx.size, 0.1), 1.0, 1.0, 1.0, 1e-3, STEPS)
    assert np.array_equal(keys[it].cpu().numpy().view(np.uint32), oracle.cell_keys(*g[0], GRID))
    # The radix sort of the keys: a bijection that puts them in nondecreasing order.
    ws = p.sort_workspace(GRID)
    _, perm = p.sort_perm(GRID, keys, ws)
    pl = perm.long()
    assert int(pl.min()) == 0 and int(pl.max()) == N - 1
    assert int(torch.bincount(pl, minlength=N).max()) == 1
    sk = keys[pl]
    assert bool((sk[1:] >= sk[:-1]).all())
    # The gather step: output i is input particle perm[i], advanced STEPS more steps.
    src = perm[it].long()
    y0 = [t[src].cpu().numpy() for t in p.field("pos")]
    w0 = [t[src].cpu().numpy() for t in p.field("vel")]
    ids = p.field("id")[0][src].cpu().numpy()
    p.step_fused(f, STEPS, grid=GRID, keys=keys, perm=perm)
    assert np.array_equal(p.field("id")[0][it].cpu().numpy(), ids)
    g2 = [t[it].cpu().numpy() for t in p.field("pos")], [t[it].cpu().numpy() for t in p.field("vel")]
    opos, ovel = [a.copy() for a in y0], [a.copy() for a in w0]
    oracle.step_soa(opos, ovel, 1.0, 1.0, 1.0, 0.1, 1e-3, STEPS)
    assert_parity_fused(g2[0], g2[1], opos, ovel, y0, w0, np.full(idx.size, 0.1), 1.0, 1.0, 1.0, 1e-3, STEPS)
    sx.sync()
    del p, ws, keys, perm, pl, sk
    torch.cuda.empty_cache()
