"""soax_step_host: one sort interval of a set held in host memory, streamed through the
device in pieces.  Its result is bit-identical to the same interval on device-resident
planes (soax_step_fused_keys, soax_sort_perm, soax_permute), for every piece count,
ragged sizes, every field type, back-to-back calls with no synchronisation between them
(the piece count changing from one call to the next), pageable host memory, and work
queued before the call on its stream; and it agrees with the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_1710_03462_b300 as sx
import soax_inputs

pytestmark = pytest.mark.gpu

GRID = 32
FLOW = sx.Flow(tau=0.1, dt=1e-3)
WIDE_FLOW = sx.Flow(dt=5e-4, tau_field="mass", tau_scale=0.1, acc="acc")


def _host(d, pinned=True):
    out = {}
    for k, v in d.items():
        ts = [torch.from_numpy(np.ascontiguousarray(a).copy()) for a in v]
        out[k] = [t.pin_memory() for t in ts] if pinned else ts
    return out


def _device_interval(p, f, nsteps, grid):
    """The same interval on device-resident planes."""
    keys = p.step_fused(f, nsteps, grid=grid)
    _, perm = p.sort_perm(grid, keys)
    p.permute(perm)
    return perm


def _same(host, p):
    g = p.numpy()
    for k, v in host.items():
        for c, t in enumerate(v):
            assert t.numpy().tobytes() == g[k][c].tobytes(), (k, c)


@pytest.mark.parametrize("n", [1, 15, 17, 4099, 100003])
@pytest.mark.parametrize("nchunks", [0, 1, 3, 8, 1024])
def test_matches_the_device_interval(n, nchunks):
    d = soax_inputs.basic_set(n, 11)
    ref = sx.Particles(sx.BASIC_SCHEMA, n)
    ref.load(d)
    rperm = _device_interval(ref, FLOW, 10, GRID)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    host = _host(d)
    perm = p.step_host(host, FLOW, 10, GRID, nchunks=nchunks)
    torch.cuda.synchronize()
    sx.sync()
    assert torch.equal(perm, rperm)
    _same(host, ref)          # the host planes hold the result
    _same(host, p)            # and so does the device (the live set flipped)
    assert p.current == 1


def test_wide_schema_with_tau_field_and_acceleration():
    n = 50001
    d = soax_inputs.wide_set(n, 5)
    ref = sx.Particles(sx.WIDE_SCHEMA, n)
    ref.load(d)
    _device_interval(ref, WIDE_FLOW, 7, 64)
    p = sx.Particles(sx.WIDE_SCHEMA, n)
    host = _host(d)
    p.step_host(host, WIDE_FLOW, 7, 64, nchunks=5)
    torch.cuda.synchronize()
    _same(host, ref)


def test_back_to_back_calls_without_synchronising():
    # Three calls queued at once with 8, 3 and 13 pieces: each upload must wait for the
    # previous call's download of the same particles (host buffers and device ranges are
    # shared), whatever the pieces were.
    n = 200003
    d = soax_inputs.basic_set(n, 2)
    ref = sx.Particles(sx.BASIC_SCHEMA, n)
    ref.load(d)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    host = _host(d)
    s = torch.cuda.Stream()
    for nchunks in (8, 3, 13):
        p.step_host(host, FLOW, 10, GRID, nchunks=nchunks, stream=s)
        _device_interval(ref, FLOW, 10, GRID)
    s.synchronize()
    torch.cuda.synchronize()
    _same(host, ref)


def test_pageable_host_memory():
    n = 30011
    d = soax_inputs.basic_set(n, 4)
    ref = sx.Particles(sx.BASIC_SCHEMA, n)
    ref.load(d)
    _device_interval(ref, FLOW, 10, GRID)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    host = _host(d, pinned=False)
    p.step_host(host, FLOW, 10, GRID, nchunks=4)
    torch.cuda.synchronize()
    _same(host, ref)


def test_work_already_on_the_stream_comes_first():
    # A fill of the device planes queued on the stream before the call must not land
    # after the call's uploads (which run on another stream).
    n = 65536
    d = soax_inputs.basic_set(n, 8)
    ref = sx.Particles(sx.BASIC_SCHEMA, n)
    ref.load(d)
    _device_interval(ref, FLOW, 10, GRID)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        torch.cuda._sleep(20_000_000)       # keep the stream busy while the call is enqueued
        for t in p.field("pos") + p.field("vel"):
            t.fill_(3.0)
    host = _host(d)
    p.step_host(host, FLOW, 10, GRID, stream=s)
    torch.cuda.synchronize()
    _same(host, ref)


def test_zero_steps_sorts_only():
    n = 10007
    d = soax_inputs.basic_set(n, 6)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    host = _host(d)
    perm = p.step_host(host, FLOW, 0, GRID, nchunks=3)
    torch.cuda.synchronize()
    keys = oracle.cell_keys(*d["pos"], GRID)
    want, _ = oracle.stable_argsort(keys)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), want)
    for k, v in d.items():
        for c, a in enumerate(v):
            assert host[k][c].numpy().tobytes() == np.ascontiguousarray(a)[want].tobytes(), (k, c)


def test_agrees_with_the_oracle():
    n, steps = 4099, 10
    d = soax_inputs.basic_set(n, 12)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    host = _host(d)
    perm = p.step_host(host, FLOW, steps, GRID, nchunks=3)
    torch.cuda.synchronize()
    opos = [a.copy() for a in d["pos"]]
    ovel = [a.copy() for a in d["vel"]]
    oracle.step_soa(opos, ovel, FLOW.A, FLOW.B, FLOW.C, FLOW.tau, FLOW.dt, steps)
    perm = perm.cpu().numpy().view(np.uint32)
    # The permutation sorts the stepped particles' keys stably (keys taken from the
    # device's own positions: a position within rounding of a cell boundary may fall
    # either side of it on the two paths).
    gpos = [host["pos"][c].numpy() for c in range(3)]
    inv = np.empty(n, np.int64)
    inv[perm] = np.arange(n)
    stepped = [g[inv] for g in gpos]             # back to the input order
    keys = oracle.cell_keys(*stepped, GRID)
    assert np.array_equal(perm, oracle.stable_argsort(keys)[0])
    for c in range(3):
        dx = np.abs(stepped[c] - opos[c])
        assert np.all(np.minimum(dx, sx.TWO_PI - dx) <= 1e-11), c
        assert np.allclose(host["vel"][c].numpy()[inv], ovel[c], rtol=1e-5, atol=1e-9), c
    assert np.array_equal(host["id"][0].numpy(), d["id"][0][perm])


@pytest.mark.parametrize("pieces", [(16, 16, 16), (8, 3, 13), (5, 5, 1)])
def test_deferred_downloads_chain(pieces):
    # Each call leaves its downloads to the next (interleaved with its uploads when the
    # pieces match, all enqueued first when they do not); finish enqueues the last ones.
    n = 150001
    d = soax_inputs.basic_set(n, 21)
    ref = sx.Particles(sx.BASIC_SCHEMA, n)
    ref.load(d)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    host = _host(d)
    s = torch.cuda.Stream()
    for k in pieces:
        p.step_host(host, FLOW, 10, GRID, nchunks=k, stream=s, defer=True)
        _device_interval(ref, FLOW, 10, GRID)
    p.step_host_finish()
    torch.cuda.synchronize()
    _same(host, ref)
    _same(host, p)


def test_deferred_then_immediate_and_finish_twice():
    n = 40007
    d = soax_inputs.basic_set(n, 22)
    ref = sx.Particles(sx.BASIC_SCHEMA, n)
    ref.load(d)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    host = _host(d)
    p.step_host(host, FLOW, 10, GRID, nchunks=4, defer=True)
    p.step_host(host, FLOW, 10, GRID, nchunks=4)           # downloads the first, then its own
    _device_interval(ref, FLOW, 10, GRID)
    _device_interval(ref, FLOW, 10, GRID)
    p.step_host_finish()                                     # nothing pending: no work
    p.step_host_finish()
    torch.cuda.synchronize()
    _same(host, ref)


def test_deferred_into_other_host_buffers():
    # A deferred call's result goes to its own host planes even when the next call
    # streams from another set of host planes.
    n = 30000
    d = soax_inputs.basic_set(n, 23)
    ref = sx.Particles(sx.BASIC_SCHEMA, n)
    ref.load(d)
    _device_interval(ref, FLOW, 10, GRID)
    first = ref.numpy()
    _device_interval(ref, FLOW, 10, GRID)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    h1, h2 = _host(d), _host(d)
    p.step_host(h1, FLOW, 10, GRID, nchunks=6, defer=True)
    torch.cuda.synchronize()
    for k in h2:                                            # h2 holds the first result
        for c, t in enumerate(h2[k]):
            t.copy_(torch.from_numpy(first[k][c]))
    p.step_host(h2, FLOW, 10, GRID, nchunks=6, defer=True)
    p.step_host_finish()
    torch.cuda.synchronize()
    for k in h1:
        for c, t in enumerate(h1[k]):
            assert t.numpy().tobytes() == first[k][c].tobytes(), (k, c)
    _same(h2, ref)
