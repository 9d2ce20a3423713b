"""GPU parity of soax_step_fused (all steps of a call in one pass over the planes, the
position carried between steps as 64-bit fixed-point turns) against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_1710_03462_b300 as sx
import soax_inputs
from parity import assert_acc, assert_parity_fused

pytestmark = pytest.mark.gpu


def _run_both(n, steps, A=1.0, B=1.0, C=1.0, tau=0.1, dt=1e-3, seed=0):
    d = soax_inputs.basic_set(n, seed)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    p.load(d)
    p.step_fused(sx.Flow(A=A, B=B, C=C, tau=tau, dt=dt), steps)
    g = p.numpy()
    opos = [a.copy() for a in d["pos"]]
    ovel = [a.copy() for a in d["vel"]]
    oracle.step_soa(opos, ovel, A, B, C, tau, dt, steps)
    return d, g, opos, ovel


@pytest.mark.parametrize("n", [1, 2, 3, 5, 1023, 65537])
def test_fused_small_and_ragged(n):
    d, g, opos, ovel = _run_both(n, 20, seed=n)
    assert_parity_fused(g["pos"], g["vel"], opos, ovel, d["pos"], d["vel"], np.full(n, 0.1), 1.0, 1.0, 1.0, 1e-3, 20)
    assert np.array_equal(g["id"][0], d["id"][0])
    for c in range(3):
        assert np.all((g["pos"][c] >= 0.0) & (g["pos"][c] < sx.TWO_PI))


def test_fused_plain_n65536_100_steps_one_launch():
    """The 65,536-particle workload: all 100 steps in a single launch."""
    w = soax_inputs.WORKLOADS["plain_n65536"]
    d, g, opos, ovel = _run_both(w["n"], w["steps"], w["A"], w["B"], w["C"], w["tau"], w["dt"], w["seed"])
    nbad = assert_parity_fused(g["pos"], g["vel"], opos, ovel, d["pos"], d["vel"], np.full(w["n"], w["tau"]),
                               w["A"], w["B"], w["C"], w["dt"], w["steps"])
    assert nbad <= 5


def test_fused_agrees_with_per_step_launches():
    """soax_step_fused(10) against ten soax_step launches: velocities equal except for
    rare f32 midpoint flips, positions within a few ulps per step."""
    n, steps = 100003, 10
    d = soax_inputs.basic_set(n, 11)
    f = sx.Flow(tau=0.1, dt=1e-3)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    p.load(d)
    p.step_fused(f, steps)
    q = sx.Particles(sx.BASIC_SCHEMA, n)
    q.load(d)
    q.step(f, steps)
    a, b = p.numpy(), q.numpy()
    diff_v = np.zeros(n, bool)
    for c in range(3):
        diff_v |= a["vel"][c] != b["vel"][c]
    assert diff_v.sum() <= 2
    ok = ~diff_v
    for c in range(3):
        dx = np.abs(a["pos"][c] - b["pos"][c])
        dx = np.minimum(dx, sx.TWO_PI - dx)
        assert dx[ok].max() <= 1e-14


def test_fused_ragged_tail_bit_equal_to_full_group():
    """A particle handled by the scalar tail (odd n) gets the same bits as in a full
    vector group (even n)."""
    n = 4097
    d = soax_inputs.basic_set(n + 1, 5)
    f = sx.Flow(tau=0.3, dt=2e-3)
    outs = []
    for m in (n, n + 1):
        p = sx.Particles(sx.BASIC_SCHEMA, m)
        p.load({k: [a[:m] for a in v] for k, v in d.items()})
        p.step_fused(f, 9)
        outs.append(p.numpy())
    for k in ("pos", "vel"):
        for x, y in zip(outs[0][k], outs[1][k]):
            assert x.tobytes() == y[:n].tobytes()


def test_fused_zero_steps_and_empty():
    p = sx.Particles(sx.BASIC_SCHEMA, 0)
    p.step_fused(sx.Flow(), 5)
    d = soax_inputs.basic_set(100)
    q = sx.Particles(sx.BASIC_SCHEMA, 100)
    q.load(d)
    q.step_fused(sx.Flow(), 0)
    assert all(np.array_equal(a, b) for a, b in zip(q.numpy()["pos"], d["pos"]))


def test_fused_positions_at_the_box_edges():
    """Positions at 0, just below 2pi and at the binary64 2pi - ulp stay in [0, 2pi) and
    follow the oracle across the periodic boundary."""
    edge = np.array([0.0, 5e-324, 1e-300, 2 ** -9, np.nextafter(sx.TWO_PI, 0), sx.TWO_PI - 1e-12, 3.0, 1e-7])
    n = edge.size ** 2
    px = np.repeat(edge, edge.size)
    py = np.tile(edge, edge.size)
    pz = np.roll(px, 3)
    rng = np.random.default_rng(3)
    vel = [rng.choice([-0.5, 0.5, 0.0, -1e-3], n).astype(np.float32) for _ in range(3)]
    d = {"id": [np.arange(n, dtype=np.int32)], "pos": [px, py, pz], "vel": vel}
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    p.load(d)
    p.step_fused(sx.Flow(tau=0.1, dt=1e-3), 7)
    g = p.numpy()
    opos = [a.copy() for a in d["pos"]]
    ovel = [a.copy() for a in d["vel"]]
    oracle.step_soa(opos, ovel, 1.0, 1.0, 1.0, 0.1, 1e-3, 7)
    for c in range(3):
        assert np.all((g["pos"][c] >= 0.0) & (g["pos"][c] < sx.TWO_PI))
    assert_parity_fused(g["pos"], g["vel"], opos, ovel, d["pos"], d["vel"], np.full(n, 0.1), 1.0, 1.0, 1.0, 1e-3, 7)


def test_fused_wide_record_mass_tau_and_acc():
    n, steps = 30001, 12
    d = soax_inputs.wide_set(n, 4)
    p = sx.Particles(sx.WIDE_SCHEMA, n)
    p.load(d)
    p.step_fused(sx.Flow(dt=5e-4, tau_field="mass", tau_scale=0.1, acc="acc"), steps)
    g = p.numpy()
    opos = [a.copy() for a in d["pos"]]
    ovel = [a.copy() for a in d["vel"]]
    oacc = [a.copy() for a in d["acc"]]
    oracle.step_soa(opos, ovel, 1.0, 1.0, 1.0, 0.0, 5e-4, steps, acc=oacc, mass=d["mass"][0], tau_scale=0.1)
    taus = 0.1 * d["mass"][0].astype(np.float64)
    assert_parity_fused(g["pos"], g["vel"], opos, ovel, d["pos"], d["vel"], taus, 1.0, 1.0, 1.0, 5e-4, steps)
    assert assert_acc(g["acc"], oacc, g["pos"], g["vel"], opos, ovel) > n // 2
    for k in ("id", "mass", "tag"):
        assert np.array_equal(g[k][0], d[k][0])


@pytest.mark.parametrize("form", ["acc_only", "tau_only"])
def test_fused_wide_record_mixed_forms(form):
    """The two mixed field forms of the wide record, each its own kernel: a stored
    acceleration with a uniform tau (the check-free path applies) and tau from the mass
    field without an acceleration, against the oracle."""
    n, steps = 30001, 12
    d = soax_inputs.wide_set(n, 5)
    p = sx.Particles(sx.WIDE_SCHEMA, n)
    p.load(d)
    opos = [a.copy() for a in d["pos"]]
    ovel = [a.copy() for a in d["vel"]]
    if form == "acc_only":
        p.step_fused(sx.Flow(tau=0.1, dt=5e-4, acc="acc"), steps)
        oacc = [a.copy() for a in d["acc"]]
        oracle.step_soa(opos, ovel, 1.0, 1.0, 1.0, 0.1, 5e-4, steps, acc=oacc)
        taus = np.full(n, 0.1)
    else:
        p.step_fused(sx.Flow(dt=5e-4, tau_field="mass", tau_scale=0.1), steps)
        oracle.step_soa(opos, ovel, 1.0, 1.0, 1.0, 0.0, 5e-4, steps, mass=d["mass"][0], tau_scale=0.1)
        taus = 0.1 * d["mass"][0].astype(np.float64)
    g = p.numpy()
    assert_parity_fused(g["pos"], g["vel"], opos, ovel, d["pos"], d["vel"], taus, 1.0, 1.0, 1.0, 5e-4, steps)
    if form == "acc_only":
        assert assert_acc(g["acc"], oacc, g["pos"], g["vel"], opos, ovel) > n // 2
    else:
        for c in range(3):
            assert np.array_equal(g["acc"][c], d["acc"][c])  # not an output of this form
    for k in ("id", "mass", "tag"):
        assert np.array_equal(g[k][0], d[k][0])


@pytest.mark.parametrize("A,B,C,tau,dt", [(1.5, 0.5, 1.3, 0.01, 1e-3), (0.7, 1.4, 0.9, 0.05, 1e-3),
                                          (1.2, 1.1, 0.6, 0.2, 5e-4), (1.0, 1.0, 1.0, 0.002, 1e-3),
                                          (1.4, 0.6, 1.2, 0.004, 2e-3)])
def test_fused_amplitudes_and_stiff_tau(A, B, C, tau, dt):
    n, steps = 20001, 100
    d, g, opos, ovel = _run_both(n, steps, A, B, C, tau, dt, seed=int(tau * 1000))
    assert_parity_fused(g["pos"], g["vel"], opos, ovel, d["pos"], d["vel"], np.full(n, tau), A, B, C, dt, steps)


@pytest.mark.parametrize("A,B,C,tau,dt,steps", [(1.3, 0.8, 1.1, 0.2, 0.02, 30), (1.0, 1.0, 1.0, 5.0, 0.5, 8),
                                                (1.0, 1.0, 1.0, 0.3, 0.3, 6)])
def test_fused_long_shifts(A, B, C, tau, dt, steps):
    """Half-step shifts beyond the shift series (the midpoint from the table, in turns)
    and, at dt >= 0.3, displacements dt vm beyond the fast fixed-point conversion."""
    n = 20001
    d, g, opos, ovel = _run_both(n, steps, A, B, C, tau, dt, seed=77)
    assert_parity_fused(g["pos"], g["vel"], opos, ovel, d["pos"], d["vel"], np.full(n, tau), A, B, C, dt, steps)


def test_fused_full_size_sorted_n16M_sampled():
    """The 16.7M-particle workload in the launch the bench times (10 steps in one pass),
    checked on every 4096th particle against the oracle."""
    w = soax_inputs.WORKLOADS["sorted_n16M"]
    n, steps = w["n"], w["sort_every"]
    d = soax_inputs.basic_set(n, w["seed"])
    p = sx.Particles(sx.BASIC_SCHEMA, n, shadow=False)
    p.load(d)
    p.step_fused(sx.Flow(A=w["A"], B=w["B"], C=w["C"], tau=w["tau"], dt=w["dt"]), steps)
    idx = np.arange(0, n, 4096)
    gpos = [t[idx].cpu().numpy() for t in p.field("pos")]
    gvel = [t[idx].cpu().numpy() for t in p.field("vel")]
    x0 = [np.ascontiguousarray(a[idx]) for a in d["pos"]]
    v0 = [np.ascontiguousarray(a[idx]) for a in d["vel"]]
    opos = [a.copy() for a in x0]
    ovel = [a.copy() for a in v0]
    oracle.step_soa(opos, ovel, w["A"], w["B"], w["C"], w["tau"], w["dt"], steps)
    assert_parity_fused(gpos, gvel, opos, ovel, x0, v0, np.full(idx.size, w["tau"]), w["A"], w["B"], w["C"], w["dt"],
                        steps)
    del p
    torch.cuda.empty_cache()


@pytest.mark.parametrize("schema,grid,n", [("basic", 32, 100003), ("wide", 64, 30001), ("basic", 7, 4097)])
def test_fused_keys_equal_cell_keys(schema, grid, n):
    """The keys the fused step writes beside the final positions are soax_cell_keys of
    those positions, bit for bit, and the oracle's keys."""
    if schema == "basic":
        d, sch, f = soax_inputs.basic_set(n, 21), sx.BASIC_SCHEMA, sx.Flow(tau=0.1, dt=1e-3)
    else:
        d, sch = soax_inputs.wide_set(n, 22), sx.WIDE_SCHEMA
        f = sx.Flow(dt=5e-4, tau_field="mass", tau_scale=0.1, acc="acc")
    p = sx.Particles(sch, n)
    p.load(d)
    keys = p.step_fused(f, 10, grid=grid)
    again = p.cell_keys(grid)
    assert torch.equal(keys[:n], again)
    g = p.numpy()
    assert np.array_equal(keys[:n].cpu().numpy().view(np.uint32), oracle.cell_keys(*g["pos"], grid))
    # nsteps = 0: the keys of the current positions.
    k0 = p.step_fused(f, 0, grid=grid)
    assert torch.equal(k0[:n], again)


def test_sort_by_keys_equals_sort_by_cell():
    """step_fused with keys + sort_by_keys (the bench step) gives the same planes and
    permutation as step_fused + sort_by_cell."""
    n, grid = 200003, 32
    d = soax_inputs.basic_set(n, 23)
    f = sx.Flow(tau=0.1, dt=1e-3)
    a = sx.Particles(sx.BASIC_SCHEMA, n)
    b = sx.Particles(sx.BASIC_SCHEMA, n)
    a.load(d)
    b.load(d)
    wa, wb = a.sort_workspace(grid), b.sort_workspace(grid)
    for _ in range(3):
        a.step_fused(f, 10)
        ka, pa = a.sort_by_cell(grid, wa)
        keys = b.step_fused(f, 10, grid=grid)
        kb, pb = b.sort_by_keys(grid, keys, wb)
        assert torch.equal(ka, kb) and torch.equal(pa, pb)
    ga, gb = a.numpy(), b.numpy()
    for k in ga:
        for x, y in zip(ga[k], gb[k]):
            assert x.tobytes() == y.tobytes()
    sk = ka.cpu().numpy().view(np.uint32)
    assert np.all(np.diff(sk.astype(np.int64)) >= 0)


@pytest.mark.parametrize("schema,grid", [("basic", 32), ("wide", 64), ("basic", 0), ("wide_acc_only", 64),
                                         ("wide_tau_only", 0)])
def test_permute_step_fused_equals_permute_then_step(schema, grid):
    """soax_permute_step_fused gives the bits of soax_permute followed by the fused step
    (and its keys), for every field of the record and every field form of the step, and
    flips the live set."""
    n = 50003
    if schema == "basic":
        d, sch, f = soax_inputs.basic_set(n, 31), sx.BASIC_SCHEMA, sx.Flow(tau=0.2, dt=1e-3)
    else:
        d, sch = soax_inputs.wide_set(n, 32), sx.WIDE_SCHEMA
        f = {"wide": sx.Flow(dt=5e-4, tau_field="mass", tau_scale=0.1, acc="acc"),
             "wide_acc_only": sx.Flow(tau=0.1, dt=5e-4, acc="acc"),
             "wide_tau_only": sx.Flow(dt=5e-4, tau_field="mass", tau_scale=0.1)}[schema]
    rng = np.random.default_rng(5)
    perm = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
    a = sx.Particles(sch, n)
    b = sx.Particles(sch, n)
    a.load(d)
    b.load(d)
    a.permute(perm)
    ka = a.step_fused(f, 7, grid=grid) if grid else a.step_fused(f, 7)
    before = b.current
    kb = b.step_fused(f, 7, grid=grid if grid else None, perm=perm)
    assert b.current == 1 - before
    ga, gb = a.numpy(), b.numpy()
    for k in ga:
        for x, y in zip(ga[k], gb[k]):
            assert x.tobytes() == y.tobytes(), k
    if grid:
        assert torch.equal(ka[:n], kb[:n])
    sx.sync()


def test_permute_step_fused_reports_bad_index():
    """A perm entry >= n is not read: particle 0 is gathered instead and soax_sync
    reports SOAX_EINVAL."""
    n = 1000
    d = soax_inputs.basic_set(n, 33)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    p.load(d)
    perm = torch.arange(n, dtype=torch.int32, device="cuda")
    perm[17] = n + 5
    p.step_fused(sx.Flow(), 2, perm=perm)
    with pytest.raises(sx.SoaxError) as err:
        sx.sync()
    assert err.value.code == -1
    assert int(p.field("id")[0][17]) == 0


def test_deferred_permute_sequence_equals_sort_by_keys():
    """The bench's sequence -- each fused step gathers by the permutation the previous
    sort left, then sort_perm -- ends, after one last permute, in the state of fused steps
    with keys each followed by sort_by_keys."""
    n, grid = 120001, 32
    d = soax_inputs.basic_set(n, 34)
    f = sx.Flow(tau=0.1, dt=1e-3)
    a = sx.Particles(sx.BASIC_SCHEMA, n)
    b = sx.Particles(sx.BASIC_SCHEMA, n)
    a.load(d)
    b.load(d)
    wa, wb = a.sort_workspace(grid), b.sort_workspace(grid)
    ka = torch.empty(n, dtype=torch.int32, device="cuda")
    kb = torch.empty(n, dtype=torch.int32, device="cuda")
    perm = None
    for _ in range(4):
        a.step_fused(f, 10, grid=grid, keys=ka)
        a.sort_by_keys(grid, ka, wa)
        b.step_fused(f, 10, grid=grid, keys=kb, perm=perm)
        _, perm = b.sort_perm(grid, kb, wb)
    b.permute(perm)
    ga, gb = a.numpy(), b.numpy()
    for k in ga:
        for x, y in zip(ga[k], gb[k]):
            assert x.tobytes() == y.tobytes(), k


def test_fused_full_size_wide_n64M_sampled():
    """The 67,108,864-particle wide record in the fused form: one sort interval (20 steps,
    tau from mass, acc) in one launch with the keys on the 64^3 grid, then the gather of
    the next interval through the permutation of those keys; every 16384th particle
    against the oracle, the keys bit-exact on the sample."""
    w = soax_inputs.WORKLOADS["wide_n64M"]
    n, steps, grid = w["n"], w["sort_every"], w["grid"]
    d = soax_inputs.wide_set(n, w["seed"])
    p = sx.Particles(sx.WIDE_SCHEMA, n)
    p.load(d)
    f = sx.Flow(A=w["A"], B=w["B"], C=w["C"], dt=w["dt"], tau_field="mass", tau_scale=w["tau_scale"], acc="acc")
    keys = p.step_fused(f, steps, grid=grid)
    idx = np.arange(3, n, 16384)
    gpos = [t[idx].cpu().numpy() for t in p.field("pos")]
    gvel = [t[idx].cpu().numpy() for t in p.field("vel")]
    x0 = [np.ascontiguousarray(a[idx]) for a in d["pos"]]
    v0 = [np.ascontiguousarray(a[idx]) for a in d["vel"]]
    m = np.ascontiguousarray(d["mass"][0][idx])
    opos, ovel = [a.copy() for a in x0], [a.copy() for a in v0]
    oracle.step_soa(opos, ovel, w["A"], w["B"], w["C"], 0.0, w["dt"], steps, mass=m, tau_scale=w["tau_scale"])
    assert_parity_fused(gpos, gvel, opos, ovel, x0, v0, w["tau_scale"] * m.astype(np.float64), w["A"], w["B"],
                        w["C"], w["dt"], steps)
    assert np.array_equal(keys[idx].cpu().numpy().view(np.uint32), oracle.cell_keys(*gpos, grid))
    del d
    ws = p.sort_workspace(grid)
    _, perm = p.sort_perm(grid, keys, ws)
    ids_before = p.field("id")[0].clone()
    p.step_fused(f, 1, grid=grid, keys=keys, perm=perm)
    sx.sync()
    ids = p.field("id")[0]
    assert torch.equal(ids, ids_before[perm.long()])
    sk = keys.cpu().numpy().view(np.uint32)
    assert sk.min() >= 0 and sk.max() < grid ** 3
    del p, ws, keys, perm, ids_before, ids
    torch.cuda.empty_cache()


@pytest.mark.parametrize("G", [7, 32, 64, 1024])
def test_fused_keys_at_cell_boundaries(G):
    """The fused kernels take a particle's key from its turns except within 2^-40 of a cell
    boundary, where the stored position decides.  Positions within a few ulps of every
    boundary (and at 0 and just below 2pi), held still (zero flow and velocity), exercise
    that fallback in the plain fused step, its ragged tail and the gather step: the keys
    must be soax_cell_keys of the positions they store, bit for bit."""
    c = G / sx.TWO_PI
    base = np.arange(G + 1) / c
    xs = [base, np.array([0.0, np.nextafter(sx.TWO_PI, 0.0), 1e-300])]
    up, dn = base.copy(), base.copy()
    for _ in range(4):
        up = np.nextafter(up, np.inf)
        dn = np.nextafter(dn, -np.inf)
        xs += [up.copy(), dn.copy()]
    x = np.concatenate(xs)
    x = x[(x >= 0) & (x < sx.TWO_PI)]
    rng = np.random.default_rng(G)
    n = 3 * x.size + 5                      # a ragged tail
    pos = [rng.choice(x, n) for _ in range(3)]
    d = {"id": [np.arange(n, dtype=np.int32)], "pos": pos, "vel": [np.zeros(n, np.float32) for _ in range(3)]}
    still = sx.Flow(A=0.0, B=0.0, C=0.0, tau=0.1, dt=1e-3)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    p.load(d)
    keys = p.step_fused(still, 1, grid=G)
    assert torch.equal(keys[:n], p.cell_keys(G))
    assert np.array_equal(keys[:n].cpu().numpy().view(np.uint32), oracle.cell_keys(*p.numpy()["pos"], G))
    ident = torch.arange(n, dtype=torch.int32, device=p.device)
    keys = p.step_fused(still, 1, grid=G, perm=ident)
    assert torch.equal(keys[:n], p.cell_keys(G))
