"""GPU batched persistent step: bit-identical to the plain per-ensemble step for every
launch shape, fused or not, and the autotuner."""
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


def test_batched_equals_plain_for_every_shape():
    steps = 6
    ref, flows = _ensembles(SIZES)
    for p, f in zip(ref, flows):
        p.step(f, steps)
    want = _bytes(ref)
    for ppt in (1, 2, 4):
        for vb in (64, 128):
            for block in (128, 256, 512):
                for fuse in (0, 1):
                    parts, _ = _ensembles(SIZES)
                    sx.step_batched(parts, flows, steps, sx.Tune(ppt, block, vb, fuse))
                    assert _bytes(parts) == want, (ppt, vb, block, fuse)


def test_batched_equals_plain_with_long_shifts():
    """dt = 0.05: groups mix the shift series and the table at the midpoint (and tau as
    short as 0.01 gives dt/tau up to 5); the per-coordinate choice keeps the bits equal."""
    steps = 4
    ref, flows = _ensembles(SIZES, 5, dt=0.05)
    for p, f in zip(ref, flows):
        p.step(f, steps)
    want = _bytes(ref)
    for ppt in (1, 2, 4):
        for fuse in (0, 1):
            parts, _ = _ensembles(SIZES, 5, dt=0.05)
            sx.step_batched(parts, flows, steps, sx.Tune(ppt, 256, 128, fuse))
            assert _bytes(parts) == want, (ppt, fuse)


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
    assert _bytes(parts) == before


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
    """The 512-ensemble workload (3.0e8 particles), 20 steps in one persistent launch per
    step: every 64th ensemble checked on sampled particles against the oracle with its
    own amplitudes and tau."""
    import oracle
    from parity import assert_parity
    w = soax_inputs.WORKLOADS["batched_512"]
    sizes, taus, abc = soax_inputs.ensembles(w["nens"], w["nmin"], w["nmax"], w["seed"])
    parts, flows, data = [], [], {}
    for e, (ne, tau) in enumerate(zip(sizes, taus)):
        dset = soax_inputs.ensemble_set(e, ne)
        p = sx.Particles(SCHEMA, int(ne), shadow=False)
        p.load(dset)
        parts.append(p)
        flows.append(sx.Flow(A=abc[e, 0], B=abc[e, 1], C=abc[e, 2], tau=float(tau), dt=w["dt"]))
        if e % 64 == 0:
            data[e] = dset
    steps = 20
    sx.step_batched(parts, flows, steps)
    for e, dset in data.items():
        n = int(sizes[e])
        idx = np.arange(0, n, max(1, n // 512))
        g = parts[e].numpy()
        x0 = [np.ascontiguousarray(a[idx]) for a in dset["pos"]]
        v0 = [np.ascontiguousarray(a[idx]) for a in dset["vel"]]
        opos, ovel = [a.copy() for a in x0], [a.copy() for a in v0]
        f = flows[e]
        oracle.step_soa(opos, ovel, f.A, f.B, f.C, f.tau, f.dt, steps)
        assert_parity([a[idx] for a in g["pos"]], [a[idx] for a in g["vel"]], opos, ovel, x0, v0,
                      np.full(idx.size, f.tau), f.A, f.B, f.C, f.dt, steps)
    del parts
    torch.cuda.empty_cache()
