"""GPU batched persistent step: for every launch shape, bit-identical to the plain
per-ensemble step (one launch per step) or to the per-ensemble fused step (fuse_steps);
the autotuner; the 512-ensemble workload against the oracle."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1710_03462_b300 as sx
import soax_inputs

pytestmark = pytest.mark.gpu

SCHEMA = sx.BASIC_SCHEMA


def _ensembles(sizes, seed=0, dt=1e-3):
    rng = np.random.default_rng(seed)
    parts, flows = [], []
    for e, n in enumerate(sizes):
        p = sx.Particles(SCHEMA, int(n), shadow=False)
        p.load(soax_inputs.ensemble_set(e, n))
        parts.append(p)
        a, b, c = rng.uniform(0.5, 1.5, 3)
        flows.append(sx.Flow(A=a, B=b, C=c, tau=rng.uniform(0.01, 1.0), dt=dt))
    return parts, flows


def _bytes(parts):
    return [t.cpu().numpy().tobytes() for p in parts for name in ("pos", "vel") for t in p.field(name)]


SIZES = [1, 3, 4, 5, 1023, 4096, 70001, 2]


def _reference(sizes, seed, steps, fused, dt=1e-3):
    ref, flows = _ensembles(sizes, seed, dt=dt)
    for p, f in zip(ref, flows):
        (p.step_fused if fused else p.step)(f, steps)
    return _bytes(ref), flows


def test_batched_equals_plain_for_every_shape():
    steps = 6
    for fuse in (0, 1):
        want, flows = _reference(SIZES, 0, steps, fuse)
        for ppt in (1, 2, 4):
            for vb in (64, 128):
                for block in (128, 256, 512):
                    parts, _ = _ensembles(SIZES)
                    sx.step_batched(parts, flows, steps, sx.Tune(ppt, block, vb, fuse))
                    assert _bytes(parts) == want, (ppt, vb, block, fuse)


def test_batched_equals_plain_with_long_shifts():
    """dt = 0.05: groups mix the shift series and the table at the midpoint (and tau as
    short as 0.01 gives dt/tau up to 5); the per-coordinate choice keeps the bits equal."""
    steps = 4
    for fuse in (0, 1):
        want, flows = _reference(SIZES, 5, steps, fuse, dt=0.05)
        for ppt in (1, 2, 4):
            parts, _ = _ensembles(SIZES, 5, dt=0.05)
            sx.step_batched(parts, flows, steps, sx.Tune(ppt, 256, 128, fuse))
            assert _bytes(parts) == want, (ppt, fuse)


def test_batched_fused_mixed_field_forms():
    """Ensembles with and without a tau field and an acceleration field in one fused
    launch (the mixed kernel form) match their own fused steps."""
    rng = np.random.default_rng(9)
    parts, flows, solo = [], [], []
    for e, (n, wide) in enumerate([(3000, True), (4097, False), (65, True), (2000, False)]):
        schema = sx.WIDE_SCHEMA if wide else SCHEMA
        d = soax_inputs.wide_set(n, 40 + e) if wide else soax_inputs.ensemble_set(e, n)
        f = (sx.Flow(A=rng.uniform(0.5, 1.5), dt=5e-4, tau_field="mass", tau_scale=0.1, acc="acc") if wide
             else sx.Flow(B=rng.uniform(0.5, 1.5), tau=0.3, dt=5e-4))
        for lst in (parts, solo):
            p = sx.Particles(schema, n, shadow=False)
            p.load(d)
            lst.append(p)
        flows.append(f)
    sx.step_batched(parts, flows, 7, sx.Tune(1, 512, 128, 1))
    for p, f in zip(solo, flows):
        p.step_fused(f, 7)
    for a, b in zip(parts, solo):
        ga, gb = a.numpy(), b.numpy()
        for k in ga:
            for x, y in zip(ga[k], gb[k]):
                assert x.tobytes() == y.tobytes(), k


def test_batched_repeated_calls_and_graph_capture():
    ref, flows = _ensembles(SIZES, 1)
    parts, _ = _ensembles(SIZES, 1)
    for p, f in zip(ref, flows):
        p.step(f, 8)
    ws = sx.step_batched(parts, flows, 2)  # uploads the plan
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            sx.step_batched(parts, flows, 3, ws=ws, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert _bytes(parts) == _bytes(ref)


def test_autotune_returns_a_valid_shape_and_leaves_data():
    parts, flows = _ensembles([5000, 300, 123457], 2)
    before = _bytes(parts)
    t = sx.autotune(parts, flows, nsteps_probe=1, use_cache=False)
    assert t.parts_per_thread in (1, 2, 4) and t.block in (128, 256, 512) and t.vec_bits in (64, 128)
    assert t.fuse_steps == 0
    tf = sx.autotune(parts, flows, nsteps_probe=3, use_cache=False, fuse=True)
    assert tf.parts_per_thread in (1, 2, 4) and tf.block in (128, 256, 512) and tf.fuse_steps == 1
    assert _bytes(parts) == before


def test_batched_fused_graph_capture():
    """Two replays of a captured fused launch of 3 steps equal two soax_step_fused(3)
    calls per ensemble."""
    want, flows = _reference(SIZES, 1, 3, True)
    ref2, _ = _ensembles(SIZES, 1)
    for p, f in zip(ref2, flows):
        p.step_fused(f, 3)
        p.step_fused(f, 3)
    parts, _ = _ensembles(SIZES, 1)
    tune = sx.Tune(2, 512, 128, 1)
    ws = sx.step_batched(parts, flows, 3, tune)  # uploads the plan, advances 3 steps
    assert _bytes(parts) == want
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            sx.step_batched(parts, flows, 3, tune, ws=ws, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    assert _bytes(parts) == _bytes(ref2)


@pytest.mark.parametrize("fuse", [0, 1])
def test_stale_plan_is_reported_not_followed(fuse):
    """A workspace whose memory changed after its plan was uploaded (here: zeroed) while
    the library still records the plan: the kernels' header check finds it, nothing
    moves and soax_sync reports SOAX_EINVAL; after soax_batched_forget the plan is
    uploaded again and the step runs."""
    parts, flows = _ensembles([1000, 37, 5], 4)
    ref, _ = _ensembles([1000, 37, 5], 4)
    for p, f in zip(ref, flows):
        (p.step_fused if fuse else p.step)(f, 2)
        if fuse:
            p.step_fused(f, 1)
    tune = sx.Tune(2, 256, 128, fuse)
    ws = sx.step_batched(parts, flows, 2, tune)  # plan uploaded, 2 steps
    sx.sync()
    before = _bytes(parts)
    ws.zero_()
    sx.step_batched(parts, flows, 1, tune, ws=ws)  # the library still records the plan
    with pytest.raises(sx.SoaxError) as err:
        sx.sync()
    assert err.value.code == -1
    assert _bytes(parts) == before
    assert sx.lib().soax_batched_forget(ctypes.c_void_p(ws.data_ptr())) == 0
    sx.step_batched(parts, flows, 1, tune, ws=ws)
    sx.sync()
    if fuse:
        assert _bytes(parts) == _bytes(ref)
    else:
        for p, f in zip(ref, flows):
            p.step(f, 1)
        assert _bytes(parts) == _bytes(ref)


def test_mixed_flows_per_ensemble():
    # Ensembles with different amplitudes and tau must each follow their own flow.
    parts, flows = _ensembles([1000, 1000], 3)
    solo, _ = _ensembles([1000, 1000], 3)
    sx.step_batched(parts, flows, 4)
    for p, f in zip(solo, flows):
        p.step(f, 4)
    assert _bytes(parts) == _bytes(solo)
    assert _bytes(parts)[:6] != _bytes(parts)[6:]


def test_full_size_batched_512_sampled():
    """The 512-ensemble workload (3.0e8 particles) in both forms the bench times: 20 steps
    with one persistent launch per step, and the 200 steps of the workload in ONE fused
    persistent launch (on a device copy of the same initial state).  Every 64th ensemble
    is checked on sampled particles against the oracle with its own amplitudes and tau."""
    import oracle
    from parity import assert_parity, assert_parity_fused
    w = soax_inputs.WORKLOADS["batched_512"]
    sizes, taus, abc = soax_inputs.ensembles(w["nens"], w["nmin"], w["nmax"], w["seed"])
    parts, fparts, flows, data = [], [], [], {}
    for e, (ne, tau) in enumerate(zip(sizes, taus)):
        dset = soax_inputs.ensemble_set(e, ne)
        p = sx.Particles(SCHEMA, int(ne), shadow=False)
        p.load(dset)
        q = sx.Particles(SCHEMA, int(ne), shadow=False)
        for name in ("pos", "vel"):
            for a, b in zip(q.field(name), p.field(name)):
                a.copy_(b)
        parts.append(p)
        fparts.append(q)
        flows.append(sx.Flow(A=abc[e, 0], B=abc[e, 1], C=abc[e, 2], tau=float(tau), dt=w["dt"]))
        if e % 64 == 0:
            data[e] = dset
    sx.step_batched(parts, flows, 20)
    sx.step_batched(fparts, flows, w["steps"], sx.Tune(1, 512, 128, 1))
    for ps, steps, check in ((parts, 20, assert_parity), (fparts, w["steps"], assert_parity_fused)):
        for e, dset in data.items():
            n = int(sizes[e])
            idx = np.arange(0, n, max(1, n // 512))
            g = ps[e].numpy()
            x0 = [np.ascontiguousarray(a[idx]) for a in dset["pos"]]
            v0 = [np.ascontiguousarray(a[idx]) for a in dset["vel"]]
            opos, ovel = [a.copy() for a in x0], [a.copy() for a in v0]
            f = flows[e]
            oracle.step_soa(opos, ovel, f.A, f.B, f.C, f.tau, f.dt, steps)
            check([a[idx] for a in g["pos"]], [a[idx] for a in g["vel"]], opos, ovel, x0, v0,
                  np.full(idx.size, f.tau), f.A, f.B, f.C, f.dt, steps)
    del parts, fparts
    torch.cuda.empty_cache()
