"""Pins of the oracle's midpoint-RK2 step (dx/dt = v, dv/dt = (u(x) - v)/tau, periodic
box), each fixed by mathematics rather than by the oracle's own formula:

  * zero flow: each step multiplies v by g = 1 - h + h^2/2 (h = dt/tau), and positions
    follow the closed form x_K = x0 + tau v0 (1 - g^K);
  * a flow constant along the trajectory (A = B = 0, v_y = 0): closed form for x_K;
  * second-order convergence of the FP64-state forward;
  * an independent 50-digit brute-force step on a few particles (mpmath);
  * the AoS and SoA variants are bit-equal;
  * per-particle tau from the mass field equals uniform tau when all masses are equal;
  * the Euler step of Eq. 1 equals numpy's float32 x + dt*v;
  * speeds grow by at most (1 + h^2)(1 + 2^-23) per step past max(|v|, max |u|), and a
    constructed particle reaches that factor (the bound the fused kernels rely on to skip
    their per-step check).
"""
import math

import mpmath
import numpy as np

import oracle
import soax_inputs

TWO_PI = soax_inputs.TWO_PI


def _set(n, seed=0):
    d = soax_inputs.basic_set(n, seed)
    return [p.copy() for p in d["pos"]], [v.copy() for v in d["vel"]]


def _minimg(d):
    return (d + math.pi) % (2 * math.pi) - math.pi


def test_zero_flow_velocity_factor():
    tau, dt, K = 0.1, 1e-3, 40
    h = dt / tau
    g = 1.0 - h + h * h / 2.0
    pos, vel = _set(4096, 1)
    v = [x.copy() for x in vel]
    for _ in range(K):
        v = [(x.astype(np.float64) * g).astype(np.float32) for x in v]
    oracle.step_soa(pos, vel, 0.0, 0.0, 0.0, tau, dt, K)
    # Bit-equal except where v*g lands within a few f64 ulps of an f32 rounding midpoint.
    mism = sum(int((a != b).sum()) for a, b in zip(vel, v))
    assert mism <= 2


def test_zero_flow_positions_closed_form():
    tau, dt, K = 0.1, 1e-3, 100
    h = dt / tau
    g = 1.0 - h + h * h / 2.0
    pos, vel = _set(2048, 2)
    x0 = [p.copy() for p in pos]
    v0 = [v.astype(np.float64) for v in vel]
    # FP64-state forward: exact closed form up to rounding.
    pd = [p.copy() for p in pos]
    vd = [v.copy() for v in v0]
    oracle.step_f64state(pd, vd, 0.0, 0.0, 0.0, tau, dt, K)
    for c in range(3):
        expect = x0[c] + tau * v0[c] * (1.0 - g ** K)
        assert np.max(np.abs(_minimg(pd[c] - expect))) < 1e-13
        assert np.allclose(vd[c], v0[c] * g ** K, rtol=1e-13, atol=0)
    # f32-stored forward: each stored v carries at most sum_k 2^-24 |v| g^k <= 2^-24 vmax/(1-g)
    # of rounding error, so positions are within K dt 2^-24 vmax / (1-g).
    oracle.step_soa(pos, vel, 0.0, 0.0, 0.0, tau, dt, K)
    for c in range(3):
        expect = x0[c] + tau * v0[c] * (1.0 - g ** K)
        bound = K * dt * 2.0 ** -24 * np.abs(v0[c]) / (1.0 - g) + 1e-13
        assert np.all(np.abs(_minimg(pos[c] - expect)) <= bound)


def test_constant_flow_closed_form():
    # A = B = 0: u_y = 0 and, with v_y = 0, y never changes, so
    # u = (C cos y0, 0, C sin y0) is constant along the path and
    # x_K = x0 + K dt u + tau (1 - g^K) (v0 - u).
    Cc, tau, dt, K = 1.7, 0.2, 1e-3, 300
    h = dt / tau
    g = 1.0 - h + h * h / 2.0
    pos, vel = _set(1024, 3)
    vel[1][:] = 0.0
    x0 = [p.copy() for p in pos]
    v0 = [v.astype(np.float64) for v in vel]
    uc = [Cc * np.cos(x0[1]), np.zeros_like(x0[1]), Cc * np.sin(x0[1])]
    pd = [p.copy() for p in pos]
    vd = [v.copy() for v in v0]
    oracle.step_f64state(pd, vd, 0.0, 0.0, Cc, tau, dt, K)
    assert np.array_equal(pd[1], x0[1])
    for c in (0, 2):
        expect = x0[c] + K * dt * uc[c] + tau * (1.0 - g ** K) * (v0[c] - uc[c])
        assert np.max(np.abs(_minimg(pd[c] - expect))) < 1e-12
        assert np.allclose(vd[c], uc[c] + (v0[c] - uc[c]) * g ** K, atol=1e-13)
    oracle.step_soa(pos, vel, 0.0, 0.0, Cc, tau, dt, K)
    assert np.array_equal(pos[1], x0[1])
    for c in (0, 2):
        expect = x0[c] + K * dt * uc[c] + tau * (1.0 - g ** K) * (v0[c] - uc[c])
        vmax = np.maximum(np.abs(v0[c]), np.abs(uc[c]))
        bound = K * dt * 2.0 ** -24 * vmax / (1.0 - g) + 1e-12
        assert np.all(np.abs(_minimg(pos[c] - expect)) <= bound)


def _run_f64(pos, vel, dt, K, A=1.0, B=0.9, C=1.1, tau=0.1):
    p = [x.copy() for x in pos]
    v = [x.astype(np.float64) for x in vel]
    oracle.step_f64state(p, v, A, B, C, tau, dt, K)
    return p, v


def test_second_order_convergence():
    pos, vel = _set(64, 4)
    T = 0.2
    ref, _ = _run_f64(pos, vel, T / 6400, 6400)
    errs = []
    for m in (50, 100, 200):
        p, _ = _run_f64(pos, vel, T / m, m)
        errs.append(max(np.max(np.abs(_minimg(p[c] - ref[c]))) for c in range(3)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, (errs, r1, r2)


def _mp_step(x, v, A, B, C, tau, dt):
    """50-digit midpoint step written from the ODE (independent of the C code)."""
    def uf(p):
        return [A * mpmath.sin(p[2]) + C * mpmath.cos(p[1]), B * mpmath.sin(p[0]) + A * mpmath.cos(p[2]),
                C * mpmath.sin(p[1]) + B * mpmath.cos(p[0])]
    f0 = uf(x)
    acc1 = [(f0[k] - v[k]) / tau for k in range(3)]
    xh = [x[k] + dt / 2 * v[k] for k in range(3)]
    vh = [v[k] + dt / 2 * acc1[k] for k in range(3)]
    f1 = uf(xh)
    acc2 = [(f1[k] - vh[k]) / tau for k in range(3)]
    xn = [x[k] + dt * vh[k] for k in range(3)]
    twopi = 2 * mpmath.pi
    xn = [q - twopi if q >= twopi else (q + twopi if q < 0 else q) for q in xn]
    return xn, [v[k] + dt * acc2[k] for k in range(3)]


def test_brute_force_mpmath():
    mpmath.mp.dps = 50
    A, B, C, tau, dt, K = 1.0, 0.8, 1.2, 0.1, 1e-3, 5
    pos, vel = _set(8, 6)
    p, v = _run_f64(pos, vel, dt, K, A, B, C, tau)
    for i in range(8):
        x = [mpmath.mpf(float(pos[c][i])) for c in range(3)]
        w = [mpmath.mpf(float(vel[c][i])) for c in range(3)]
        for _ in range(K):
            x, w = _mp_step(x, w, A, B, C, tau, dt)
        for c in range(3):
            assert abs(float(x[c]) - p[c][i]) < 1e-14
            assert abs(float(w[c]) - v[c][i]) < 1e-14


def test_aos_equals_soa_bitwise():
    d = soax_inputs.basic_set(3000, 7)
    planes = d["id"] + d["pos"] + d["vel"]
    rec = oracle.soa_to_aos(planes, [4, 8, 4], [1, 3, 3])
    rb, offs = oracle.aos_layout([4, 8, 4], [1, 3, 3])
    pos = [p.copy() for p in d["pos"]]
    vel = [v.copy() for v in d["vel"]]
    oracle.step_soa(pos, vel, 1.0, 1.0, 1.0, 0.1, 1e-3, 25)
    oracle.step_aos(rec, rb, offs[1], offs[2], 1.0, 1.0, 1.0, 0.1, 1e-3, 25)
    back = oracle.aos_to_soa(rec, [4, 8, 4], [1, 3, 3], [np.int32, np.float64, np.float32])
    for a, b in zip(back, d["id"] + pos + vel):
        assert a.tobytes() == b.tobytes()


def test_aos_equals_soa_wide_record():
    d = soax_inputs.wide_set(2000, 8)
    eb, nc = [8, 8, 4, 4, 4, 1], [1, 3, 3, 3, 1, 1]
    planes = d["id"] + d["pos"] + d["vel"] + d["acc"] + d["mass"] + d["tag"]
    rec = oracle.soa_to_aos(planes, eb, nc)
    rb, offs = oracle.aos_layout(eb, nc)
    pos = [p.copy() for p in d["pos"]]
    vel = [v.copy() for v in d["vel"]]
    acc = [a.copy() for a in d["acc"]]
    oracle.step_soa(pos, vel, 1.0, 1.0, 1.0, 0.0, 5e-4, 20, acc=acc, mass=d["mass"][0], tau_scale=0.1)
    oracle.step_aos(rec, rb, offs[1], offs[2], 1.0, 1.0, 1.0, 0.0, 5e-4, 20, acc_off=offs[3], mass_off=offs[4],
                    tau_scale=0.1)
    back = oracle.aos_to_soa(rec, eb, nc, [np.int64, np.float64, np.float32, np.float32, np.float32, np.uint8])
    for a, b in zip(back, d["id"] + pos + vel + acc + d["mass"] + d["tag"]):
        assert a.tobytes() == b.tobytes()


def test_mass_tau_matches_uniform_tau():
    pos, vel = _set(500, 9)
    p2, v2 = [p.copy() for p in pos], [v.copy() for v in vel]
    m = np.full(500, 0.5, np.float32)
    oracle.step_soa(pos, vel, 1.0, 1.0, 1.0, 0.05, 1e-3, 10, mass=m, tau_scale=0.1)
    oracle.step_soa(p2, v2, 1.0, 1.0, 1.0, 0.1 * 0.5, 1e-3, 10)
    for a, b in zip(pos + vel, p2 + v2):
        assert np.array_equal(a, b)


def test_acc_is_last_stage_acceleration():
    # With zero flow a2 = -vm/tau and vm = v(1 - h/2): a check of the stage value.
    tau, dt = 0.1, 1e-3
    pos, vel = _set(100, 10)
    v0 = [v.astype(np.float64) for v in vel]
    acc = [np.zeros(100, np.float32) for _ in range(3)]
    oracle.step_soa(pos, vel, 0.0, 0.0, 0.0, tau, dt, 1, acc=acc)
    for c in range(3):
        assert np.allclose(acc[c], -v0[c] * (1 - dt / tau / 2) / tau, rtol=1e-6)


def test_euler_eq1_f32():
    rng = np.random.default_rng(11)
    x = rng.standard_normal(1000).astype(np.float32)
    v = rng.standard_normal(1000).astype(np.float32)
    ref = x + np.float32(1e-2) * v
    oracle.euler_f32(x, v, 1e-2)
    assert np.array_equal(x, ref)


def test_euler_aos_equals_soa_listing4_records():
    # Particle<SIZE> of Listing 4: float x[3]; float v[3]; float temp[SIZE].
    rng = np.random.default_rng(12)
    n, dt = 999, np.float32(1e-2)
    x = [rng.standard_normal(n).astype(np.float32) for _ in range(3)]
    v = [rng.standard_normal(n).astype(np.float32) for _ in range(3)]
    for size in (0, 1, 32):
        planes = x + v + [rng.standard_normal(n).astype(np.float32) for _ in range(size)]
        ncomp = [3, 3] + ([size] if size else [])
        eb = [4] * len(ncomp)
        rec = oracle.soa_to_aos(planes, eb, ncomp)
        rb, offs = oracle.aos_layout(eb, ncomp)
        assert rb == 24 + 4 * size
        oracle.euler_aos_f32(rec, rb, offs[0], offs[1], dt)
        xs = [a.copy() for a in x]
        for c in range(3):
            oracle.euler_f32(xs[c], v[c], dt)
        back = oracle.aos_to_soa(rec, eb, ncomp, [np.float32] * len(ncomp))
        for c in range(3):
            assert back[c].tobytes() == xs[c].tobytes()
            assert np.array_equal(xs[c], x[c] + dt * v[c])


def test_fill_and_lincomb_pins():
    # SetToValue (Listing 7) on each type; the expression of Listing 5 against numpy.
    for dt, val in ((np.int32, -7), (np.int64, 2 ** 40), (np.uint8, 200), (np.float32, 0.1), (np.float64, 0.1)):
        a = oracle.fill(np.zeros(17, dt), val)
        assert np.all(a == np.array(val).astype(dt))
    rng = np.random.default_rng(3)
    for dt in (np.float32, np.float64):
        v1, v2 = rng.standard_normal(1000).astype(dt), rng.standard_normal(1000).astype(dt)
        out = oracle.lincomb(np.empty(1000, dt), [v1, v2], [1.0, -1.0])
        assert np.array_equal(out, v1 - v2)  # fma(1, a, 0) = a exactly, then fma(-1, b, a) = RN(a - b)
        w = oracle.lincomb(np.empty(1000, dt), [v1], [2.0], 0.5)
        assert np.array_equal(w, (dt(2.0) * v1 + dt(0.5)).astype(dt))  # 2 v1 is exact: one rounding


def test_remove_by_overwrite_with_last_pins():
    # Brute force on the definition: the survivors are the same multiset, the size drops by
    # k, and elements below the new size that were not removed stay in place.
    rng = np.random.default_rng(4)
    for n, k in ((10, 0), (10, 10), (10, 3), (1000, 37), (1000, 999)):
        ids = np.arange(n, dtype=np.int64)
        idx = np.sort(rng.choice(n, k, replace=False)).astype(np.uint32)
        out = oracle.remove([ids], idx)[0]
        assert out.size == n - k
        assert sorted(out.tolist()) == sorted(set(range(n)) - set(idx.tolist()))
        keep = [i for i in range(n - k) if i not in set(idx.tolist())]
        assert np.array_equal(out[keep], ids[keep])
    # Sec. 2: removing one particle overwrites it with the last one.
    for i in range(7):
        out = oracle.remove([np.arange(7, dtype=np.int32)], np.array([i], np.uint32))[0]
        exp = list(range(6))
        if i < 6:
            exp[i] = 6
        assert out.tolist() == exp
    # Holes below n - k take the surviving tail particles in ascending order.
    out = oracle.remove([np.arange(10, dtype=np.int32)], np.array([2, 4, 7], np.uint32))[0]
    assert out.tolist() == [0, 1, 8, 3, 9, 5, 6]


def test_speed_bound_per_step():
    """The bound behind the fused kernels' check-free path (no check per step for a particle
    whose starting speeds are below the launch's vsafe): one midpoint step is
    v' = v(1 - h + h^2/2) + h u(xm) - (h^2/2) u(x) with h = dt/tau, and 1 - h + h^2/2 > 0,
    so if |v_c| and every |u_c| are at most M then |v'_c| <= M (1 + h^2), times 1 + 2^-23
    for the f32 rounding of v'.  Checked on the oracle's trajectories, per particle, for
    small and large h, negative amplitudes, and speeds on both sides of the flow's
    amplitude bound."""
    rng = np.random.default_rng(11)
    n, nsteps = 4000, 25
    for A, B, C, tau, dt in ((1.0, 1.0, 1.0, 0.1, 1e-3), (1.5, -0.5, 1.3, 0.01, 1e-3),
                             (-1.2, 1.1, 0.6, 0.2, 0.1), (1.0, 1.0, 1.0, 0.05, 0.05),
                             (0.3, 2.0, -1.0, 1.0, 0.5)):
        h = dt / tau
        umax = max(abs(A) + abs(C), abs(B) + abs(A), abs(C) + abs(B))
        pos = [rng.uniform(0.0, TWO_PI, n) for _ in range(3)]
        vel = [(rng.standard_normal(n) * rng.choice([0.1, 1.0, 5.0], n)).astype(np.float32) for _ in range(3)]
        M = np.maximum(np.max(np.abs(np.stack(vel)).astype(np.float64), axis=0), umax)
        grow = (1.0 + h * h) * (1.0 + 2.0 ** -23)
        for s in range(1, nsteps + 1):
            oracle.step_soa(pos, vel, A, B, C, tau, dt, 1)
            speed = np.max(np.abs(np.stack(vel)).astype(np.float64), axis=0)
            assert np.all(speed <= M * grow ** s), (A, B, C, tau, dt, s)
    # The growth factor is needed: with B = C = 0 (u = (A sin z, A cos z, 0)), v_x = A and a
    # half-step shift of -pi in z from 3 pi/2, u_x(x) = -A and u_x(xm) = +A, so
    # v'_x = A (1 - h + h^2/2) + h A + (h^2/2) A = A (1 + h^2) exactly in real arithmetic.
    A, tau, dt = 2 * math.pi, 1.0, 1.0
    h = dt / tau
    pos = [np.array([0.5]), np.array([0.5]), np.array([1.5 * math.pi])]
    vel = [np.array([A], np.float32), np.array([0.0], np.float32), np.array([-A], np.float32)]
    M = max(float(np.abs(vel[0][0])), float(np.abs(vel[2][0])), A)
    oracle.step_soa(pos, vel, A, 0.0, 0.0, tau, dt, 1)
    vx = float(vel[0][0])
    assert M * (1.0 + h * h) * (1.0 - 1e-6) < vx <= M * (1.0 + h * h) * (1.0 + 2.0 ** -23)


def test_f64state_threads_do_not_change_bits():
    """Threads only split the particle range: one thread and many give the same bits."""
    d = soax_inputs.basic_set(5000, 11)
    outs = []
    for threads in (1, 7):
        p = [a.copy() for a in d["pos"]]
        v = [a.astype(np.float64) for a in d["vel"]]
        oracle.step_f64state(p, v, 1.0, 0.9, 1.1, 0.1, 1e-3, 20, threads=threads)
        outs.append(p + v)
    for a, b in zip(*outs):
        assert a.tobytes() == b.tobytes()
