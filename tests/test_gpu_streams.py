"""Calls on a side stream with temporaries the binding allocates: the caching allocator
must not hand their memory to work on the current stream while the call still runs.

Each call is queued behind a long step on the side stream, its returned views are
dropped at once, and the current stream then allocates and overwrites blocks of the
same size many times; the results must still equal the oracle's."""
import numpy as np
import pytest
import torch

import oracle
import paper_1710_03462_b300 as sx
import soax_inputs

pytestmark = pytest.mark.gpu


def _scribble(nbytes, times=8):
    """Allocate and overwrite blocks of nbytes on the current stream (what another
    user of the allocator would do while a side-stream call is in flight)."""
    keep = []
    for k in range(times):
        t = torch.empty(max(nbytes, 16), dtype=torch.uint8, device="cuda")
        t.fill_(0xA5 ^ k)
        keep.append(t)
    return keep


def _busy(p, side, steps=400):
    """A long step on the side stream, so the call queued after it is still pending when
    the current stream reuses memory."""
    p.step(sx.Flow(), steps, stream=side)


def test_sort_by_cell_on_side_stream():
    n, grid = 200003, 32
    d = soax_inputs.basic_set(n, 21)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    p.load(d)
    busy = sx.Particles(sx.BASIC_SCHEMA, 1 << 20, shadow=False)
    busy.load(soax_inputs.basic_set(1 << 20, 22))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    _busy(busy, side)
    ws_bytes = p.sort_workspace(grid).numel()
    p.sort_by_cell(grid, stream=side)  # the returned views are dropped here
    junk = _scribble(ws_bytes)
    side.synchronize()
    torch.cuda.synchronize()
    g = p.numpy()
    perm, _ = oracle.stable_argsort(oracle.cell_keys(*d["pos"], grid))
    ref = oracle.permute(d["id"] + d["pos"] + d["vel"], perm)
    got = g["id"] + g["pos"] + g["vel"]
    for a, b in zip(got, ref):
        assert a.tobytes() == b.tobytes()
    del junk
    sx.sync(side)


def test_remove_and_get_element_on_side_stream():
    n = 50000
    d = soax_inputs.basic_set(n, 23)
    p = sx.Particles(sx.BASIC_SCHEMA, n, shadow=False)
    p.load(d)
    busy = sx.Particles(sx.BASIC_SCHEMA, 1 << 20, shadow=False)
    busy.load(soax_inputs.basic_set(1 << 20, 24))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    idx_np = np.arange(7, n, 977, dtype=np.uint32)
    idx = torch.from_numpy(idx_np.view(np.int32)).cuda()
    side.wait_stream(torch.cuda.current_stream())
    _busy(busy, side)
    idx.record_stream(side)
    p.remove(idx, stream=side)
    junk = _scribble(64 * idx_np.size)
    rec = p.get_element(3, stream=side)
    junk += _scribble(64)
    side.synchronize()
    torch.cuda.synchronize()
    ref = oracle.remove(d["id"] + d["pos"] + d["vel"], idx_np)
    g = p.numpy()
    for a, b in zip(g["id"] + g["pos"] + g["vel"], ref):
        assert a.tobytes() == b.tobytes()
    rb, _ = p.aos_layout()
    want = oracle.soa_to_aos([a[3:4] for a in ref], [4, 8, 4], [1, 3, 3])
    assert rec.cpu().numpy().tobytes() == want.tobytes()
    del junk
    sx.sync(side)
