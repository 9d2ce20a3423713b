"""Pins of the oracle's adjoint: central finite differences of the FP64-state forward,
the zero-flow closed form (x_K = x0 + tau v0 (1 - g^K)), zero gradient at the target
parameters, and the f32-stored adjoint staying close to the FP64 one."""
import math

import numpy as np

import oracle
import soax_inputs

TWO_PI = soax_inputs.TWO_PI


def _minimg(d):
    return np.fmod(np.fmod(d + math.pi, TWO_PI) + TWO_PI, TWO_PI) - math.pi


def _loss_f64(pos, vel, xt, A, B, C, tau, dt, K):
    p = [x.copy() for x in pos]
    v = [x.astype(np.float64) for x in vel]
    oracle.step_f64state(p, v, A, B, C, tau, dt, K)
    n = p[0].size
    return sum(float(np.sum(_minimg(p[c] - xt[c]) ** 2)) for c in range(3)) / n


def _problem(n=48, K=60, seed=3):
    d = soax_inputs.basic_set(n, seed)
    pos = [p.copy() for p in d["pos"]]
    vel = [v.astype(np.float64) for v in d["vel"]]
    xt = [p.copy() for p in pos]
    vt = [v.copy() for v in vel]
    oracle.step_f64state(xt, vt, 1.1, 1.0, 1.0, 0.1, 1e-3, K)
    return pos, vel, xt


def test_param_gradients_match_central_fd():
    K, dt, eps = 60, 1e-3, 1e-6
    pos, vel, xt = _problem(K=K)
    th = [1.0, 0.9, 1.05, 0.12]
    loss, _, _, g = oracle.adjoint(pos, vel, xt, *th, dt, K, f32v=False)
    assert abs(loss - _loss_f64(pos, vel, xt, *th, dt, K)) < 1e-15
    for k in range(4):
        tp, tm = list(th), list(th)
        tp[k] += eps
        tm[k] -= eps
        fd = (_loss_f64(pos, vel, xt, *tp, dt, K) - _loss_f64(pos, vel, xt, *tm, dt, K)) / (2 * eps)
        assert abs(g[k] - fd) <= 1e-6 * max(abs(fd), 1e-8), (k, g[k], fd)


def test_state_gradients_match_central_fd():
    K, dt, eps = 60, 1e-3, 1e-6
    pos, vel, xt = _problem(K=K)
    th = [1.0, 0.9, 1.05, 0.12]
    _, xb, vb, _ = oracle.adjoint(pos, vel, xt, *th, dt, K, f32v=False)
    for i in (0, 7, 31):
        for c in range(3):
            for which, arr, grad in (("x", pos, xb), ("v", vel, vb)):
                ap = [a.copy() for a in arr]
                am = [a.copy() for a in arr]
                ap[c][i] += eps
                am[c][i] -= eps
                if which == "x":
                    lp = _loss_f64(ap, vel, xt, *th, dt, K)
                    lm = _loss_f64(am, vel, xt, *th, dt, K)
                else:
                    lp = _loss_f64(pos, ap, xt, *th, dt, K)
                    lm = _loss_f64(pos, am, xt, *th, dt, K)
                fd = (lp - lm) / (2 * eps)
                # FD round-off floor: |L| * 2^-52 / eps is about 1e-13 here.
                assert abs(grad[c][i] - fd) <= 1e-6 * abs(fd) + 1e-12, (which, i, c, grad[c][i], fd)


def test_zero_flow_closed_form_gradients():
    n, K, dt, tau = 40, 80, 1e-3, 0.1
    d = soax_inputs.basic_set(n, 5)
    pos = [p.copy() for p in d["pos"]]
    vel = [v.astype(np.float64) for v in d["vel"]]
    xt = [np.ascontiguousarray(np.fmod(p + 0.01, TWO_PI)) for p in pos]
    h = dt / tau
    g = 1 - h + h * h / 2
    loss, xb, vb, gr = oracle.adjoint(pos, vel, xt, 0.0, 0.0, 0.0, tau, dt, K, f32v=False)
    dg = dt / tau ** 2 - dt ** 2 / tau ** 3       # dg/dtau
    dfac = (1 - g ** K) - tau * K * g ** (K - 1) * dg  # d/dtau [tau (1 - g^K)]
    gt = 0.0
    for c in range(3):
        xk = pos[c] + tau * vel[c] * (1 - g ** K)
        dd = _minimg(xk - xt[c])
        assert np.allclose(xb[c], 2 * dd / n, rtol=1e-9, atol=1e-15)
        assert np.allclose(vb[c], 2 * dd / n * tau * (1 - g ** K), rtol=1e-9, atol=1e-15)
        gt += float(np.sum(2 * dd / n * vel[c] * dfac))
    assert abs(gr[3] - gt) <= 1e-9 * abs(gt)


def test_zero_gradient_at_target():
    n, K = 32, 50
    d = soax_inputs.basic_set(n, 6)
    pos, vel = d["pos"], d["vel"]
    xt = [p.copy() for p in pos]
    vt = [v.copy() for v in vel]
    oracle.step_soa(xt, vt, 1.1, 1.0, 1.0, 0.1, 1e-3, K)
    loss, xb, vb, gr = oracle.adjoint(pos, vel, xt, 1.1, 1.0, 1.0, 0.1, 1e-3, K, f32v=True)
    assert loss == 0.0 and np.all(gr == 0.0)
    assert all(np.all(a == 0.0) for a in xb + vb)


def test_f32_storage_adjoint_close_to_f64():
    K = 60
    pos, vel, xt = _problem(K=K)
    vel32 = [v.astype(np.float32) for v in vel]
    th = [1.0, 0.9, 1.05, 0.12]
    _, xa, va, ga = oracle.adjoint(pos, vel32, xt, *th, 1e-3, K, f32v=True)
    _, xd, vd, gd = oracle.adjoint(pos, [v.astype(np.float64) for v in vel32], xt, *th, 1e-3, K, f32v=False)
    assert np.allclose(ga, gd, rtol=1e-4)
    for c in range(3):
        assert np.allclose(xa[c], xd[c], rtol=1e-4, atol=1e-9)
