"""GPU parity of the midpoint-RK2 step (soax_step, soax_step_aos) against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_1710_03462_b300 as sx
import soax_inputs
from parity import assert_acc, assert_parity

pytestmark = pytest.mark.gpu


def _run_both(n, steps, A=1.0, B=1.0, C=1.0, tau=0.1, dt=1e-3, seed=0):
    d = soax_inputs.basic_set(n, seed)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    p.load(d)
    p.step(sx.Flow(A=A, B=B, C=C, tau=tau, dt=dt), steps)
    g = p.numpy()
    opos = [a.copy() for a in d["pos"]]
    ovel = [a.copy() for a in d["vel"]]
    oracle.step_soa(opos, ovel, A, B, C, tau, dt, steps)
    return d, g, opos, ovel


@pytest.mark.parametrize("n", [1, 3, 4, 5, 1023, 65537])
def test_step_small_and_ragged(n):
    d, g, opos, ovel = _run_both(n, 20, seed=n)
    assert_parity(g["pos"], g["vel"], opos, ovel, d["pos"], d["vel"], np.full(n, 0.1), 1.0, 1.0, 1.0, 1e-3, 20)
    assert np.array_equal(g["id"][0], d["id"][0])  # untouched


def test_plain_n65536_100_steps():
    w = soax_inputs.WORKLOADS["plain_n65536"]
    d, g, opos, ovel = _run_both(w["n"], w["steps"], w["A"], w["B"], w["C"], w["tau"], w["dt"], w["seed"])
    nbad = assert_parity(g["pos"], g["vel"], opos, ovel, d["pos"], d["vel"], np.full(w["n"], w["tau"]), w["A"],
                         w["B"], w["C"], w["dt"], w["steps"])
    assert nbad <= 5


def test_zero_steps_and_empty():
    p = sx.Particles(sx.BASIC_SCHEMA, 0)
    p.step(sx.Flow(), 5)
    d = soax_inputs.basic_set(100)
    q = sx.Particles(sx.BASIC_SCHEMA, 100)
    q.load(d)
    q.step(sx.Flow(), 0)
    assert all(np.array_equal(a, b) for a, b in zip(q.numpy()["pos"], d["pos"]))


@pytest.mark.parametrize("dt", [1e-3, 0.02])
def test_aos_step_bit_equal_to_soa(dt):
    n = 50001
    d = soax_inputs.basic_set(n, 3)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    p.load(d)
    aos = p.to_aos()
    f = sx.Flow(tau=0.2, dt=dt)
    p.step(f, 7)
    p.step_aos(aos, f, 7)
    q = sx.Particles(sx.BASIC_SCHEMA, n)
    q.from_aos(aos)
    a, b = p.numpy(), q.numpy()
    for k in a:
        for x, y in zip(a[k], b[k]):
            assert x.tobytes() == y.tobytes()


def test_wide_record_mass_tau_and_acc():
    n = 30001
    d = soax_inputs.wide_set(n, 4)
    p = sx.Particles(sx.WIDE_SCHEMA, n)
    p.load(d)
    f = sx.Flow(dt=5e-4, tau_field="mass", tau_scale=0.1, acc="acc")
    p.step(f, 12)
    g = p.numpy()
    opos = [a.copy() for a in d["pos"]]
    ovel = [a.copy() for a in d["vel"]]
    oacc = [a.copy() for a in d["acc"]]
    oracle.step_soa(opos, ovel, 1.0, 1.0, 1.0, 0.0, 5e-4, 12, acc=oacc, mass=d["mass"][0], tau_scale=0.1)
    taus = 0.1 * d["mass"][0].astype(np.float64)
    assert_parity(g["pos"], g["vel"], opos, ovel, d["pos"], d["vel"], taus, 1.0, 1.0, 1.0, 5e-4, 12)
    assert assert_acc(g["acc"], oacc, g["pos"], g["vel"], opos, ovel) > n // 2
    for k in ("id", "mass", "tag"):
        assert np.array_equal(g[k][0], d[k][0])
    # AoS variant of the wide record is bit-equal.
    q = sx.Particles(sx.WIDE_SCHEMA, n)
    q.load(d)
    aos = q.to_aos()
    q.step_aos(aos, f, 12)
    q.from_aos(aos)
    h = q.numpy()
    for k in g:
        for x, y in zip(g[k], h[k]):
            assert x.tobytes() == y.tobytes()


def test_full_size_sorted_n16M_sampled():
    """The 16.7M-particle workload in the launch shape the bench times, 10 steps, checked
    on every 4096th particle against the oracle."""
    w = soax_inputs.WORKLOADS["sorted_n16M"]
    n, steps = w["n"], 10
    d = soax_inputs.basic_set(n, w["seed"])
    p = sx.Particles(sx.BASIC_SCHEMA, n, shadow=False)
    p.load(d)
    p.step(sx.Flow(A=w["A"], B=w["B"], C=w["C"], tau=w["tau"], dt=w["dt"]), steps)
    idx = np.arange(0, n, 4096)
    gpos = [t[idx].cpu().numpy() for t in p.field("pos")]
    gvel = [t[idx].cpu().numpy() for t in p.field("vel")]
    x0 = [np.ascontiguousarray(a[idx]) for a in d["pos"]]
    v0 = [np.ascontiguousarray(a[idx]) for a in d["vel"]]
    opos = [a.copy() for a in x0]
    ovel = [a.copy() for a in v0]
    oracle.step_soa(opos, ovel, w["A"], w["B"], w["C"], w["tau"], w["dt"], steps)
    assert_parity(gpos, gvel, opos, ovel, x0, v0, np.full(idx.size, w["tau"]), w["A"], w["B"], w["C"], w["dt"],
                  steps)


def test_full_size_wide_n64M_sampled():
    w = soax_inputs.WORKLOADS["wide_n64M"]
    n, steps = w["n"], 4
    d = soax_inputs.wide_set(n, w["seed"])
    p = sx.Particles(sx.WIDE_SCHEMA, n, shadow=False)
    p.load(d)
    p.step(sx.Flow(A=w["A"], B=w["B"], C=w["C"], dt=w["dt"], tau_field="mass", tau_scale=w["tau_scale"], acc="acc"),
           steps)
    idx = np.arange(7, n, 16384)
    gpos = [t[idx].cpu().numpy() for t in p.field("pos")]
    gvel = [t[idx].cpu().numpy() for t in p.field("vel")]
    x0 = [np.ascontiguousarray(a[idx]) for a in d["pos"]]
    v0 = [np.ascontiguousarray(a[idx]) for a in d["vel"]]
    m = np.ascontiguousarray(d["mass"][0][idx])
    opos = [a.copy() for a in x0]
    ovel = [a.copy() for a in v0]
    oracle.step_soa(opos, ovel, w["A"], w["B"], w["C"], 0.0, w["dt"], steps, mass=m, tau_scale=w["tau_scale"])
    assert_parity(gpos, gvel, opos, ovel, x0, v0, w["tau_scale"] * m.astype(np.float64), w["A"], w["B"], w["C"],
                  w["dt"], steps)
    del p
    torch.cuda.empty_cache()


@pytest.mark.parametrize("A,B,C,tau,dt", [(1.5, 0.5, 1.3, 0.01, 1e-3), (0.7, 1.4, 0.9, 0.05, 1e-3),
                                          (1.2, 1.1, 0.6, 0.2, 5e-4), (1.0, 1.0, 1.0, 0.002, 1e-3),
                                          (1.4, 0.6, 1.2, 0.004, 2e-3)])
def test_step_amplitudes_and_stiff_tau(A, B, C, tau, dt):
    """Non-unit amplitudes and dt/tau up to 0.1 (the range of the batched workload), and
    dt/tau = 0.5, beyond every workload (float-pair errors grow with dt/tau)."""
    n, steps = 20001, 100
    d, g, opos, ovel = _run_both(n, steps, A, B, C, tau, dt, seed=int(tau * 1000))
    assert_parity(g["pos"], g["vel"], opos, ovel, d["pos"], d["vel"], np.full(n, tau), A, B, C, dt, steps)


@pytest.mark.parametrize("A,B,C,tau,dt,steps", [(1.3, 0.8, 1.1, 0.2, 0.02, 30), (1.0, 1.0, 1.0, 5.0, 0.5, 8)])
def test_step_long_shifts(A, B, C, tau, dt, steps):
    """Steps long enough that the half-step shift (dt/2)|v| leaves the range of the shift
    series for some coordinates (and, at dt = 0.5, carries midpoints across the periodic
    boundary): those coordinates take the table at the midpoint itself."""
    n = 20001
    d, g, opos, ovel = _run_both(n, steps, A, B, C, tau, dt, seed=77)
    assert_parity(g["pos"], g["vel"], opos, ovel, d["pos"], d["vel"], np.full(n, tau), A, B, C, dt, steps)
