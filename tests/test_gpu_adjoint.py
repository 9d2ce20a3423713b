"""GPU checkpointed forward and adjoint against the oracle's adjoint (f32-stored forward,
same arithmetic) and against central finite differences; the autograd Function."""
import numpy as np
import pytest
import torch

import oracle
import paper_1710_03462_b300 as sx
import soax_inputs
from parity import audit_particle_fused

pytestmark = pytest.mark.gpu

SCHEMA = [("pos", "f64", 3, "P"), ("vel", "f32", 3, "V")]


def _target(d, K, A=1.1, tau=0.1, dt=1e-3):
    xt = [a.copy() for a in d["pos"]]
    vt = [a.copy() for a in d["vel"]]
    oracle.step_soa(xt, vt, A, 1.0, 1.0, tau, dt, K)
    return xt


def _gpu_adjoint(d, xt, K, C, th, dt=1e-3):
    n = d["pos"][0].size
    p = sx.Particles(SCHEMA, n, shadow=False)
    p.load({"pos": d["pos"], "vel": d["vel"]})
    f = sx.Flow(A=th[0], B=th[1], C=th[2], tau=th[3], dt=dt)
    ws = p.adjoint_workspace(K, C)
    p.step_checkpointed(f, K, C, ws)
    xtg = [torch.from_numpy(a).cuda() for a in xt]
    loss, xbK = p.minimage_loss(xtg, ws)
    xb0, vb0, g = p.step_adjoint(f, K, C, ws, xbK)
    return (p, float(loss.item()), [t.cpu().numpy() for t in xb0], [t.cpu().numpy() for t in vb0],
            g.cpu().numpy())


def _diverged(p, d, th, K, dt=1e-3, max_frac=1e-3):
    """Particles whose forward state after K steps differs from the oracle's by more than
    f64 rounding: their f32 velocity took the other side of a rounding midpoint at some
    step.  The forward is soax_step_fused's arithmetic, so each is replayed on its own
    trajectory (parity.audit_particle_fused) and must be a legitimate midpoint flip; their
    gradients then follow a slightly different trajectory and are left out of the
    element-wise comparison."""
    opos = [a.copy() for a in d["pos"]]
    ovel = [a.copy() for a in d["vel"]]
    oracle.step_soa(opos, ovel, *th, dt, K)
    g = p.numpy()
    bad = np.zeros(opos[0].size, bool)
    for c in range(3):
        dx = np.abs(g["pos"][c] - opos[c])
        bad |= np.minimum(dx, sx.TWO_PI - dx) > 1e-12
        bad |= g["vel"][c] != ovel[c]
    idx = np.flatnonzero(bad)
    assert idx.size <= max(2, max_frac * bad.size), f"{idx.size} diverged particles"
    for i in idx:
        audit_particle_fused([d["pos"][c][i] for c in range(3)], [d["vel"][c][i] for c in range(3)], *th[:3], th[3],
                             dt, K)
    return bad


@pytest.mark.parametrize("n,K,C", [(1, 5, 32), (1000, 70, 32), (4099, 100, 32), (513, 64, 8), (700, 10, 1)])
def test_adjoint_vs_oracle(n, K, C):
    d = soax_inputs.basic_set(n, n)
    xt = _target(d, K)
    th = [1.0, 0.95, 1.05, 0.12]
    p, loss, xb, vb, g = _gpu_adjoint(d, xt, K, C, th)
    ol, oxb, ovb, og = oracle.adjoint(d["pos"], d["vel"], xt, *th, 1e-3, K, f32v=True)
    ok = ~_diverged(p, d, th, K)
    assert abs(loss - ol) <= 1e-9 * abs(ol)
    assert np.allclose(g, og, rtol=1e-8, atol=0)
    for c in range(3):
        scale = max(np.abs(oxb[c]).max(), 1e-300)
        assert np.max(np.abs(xb[c] - oxb[c])[ok]) <= 1e-9 * scale
        scale = max(np.abs(ovb[c]).max(), 1e-300)
        assert np.max(np.abs(vb[c] - ovb[c])[ok]) <= 1e-9 * scale


@pytest.mark.parametrize("th", [[0.0, 0.95, 1.05, 0.12], [1.0, 1e-7, 1.05, 0.12], [-1.0, 0.95, -1.05, 0.2]])
def test_adjoint_vs_oracle_amplitude_forms(th):
    """The reverse runs on amplitude-scaled tables when every |amplitude| >= 2^-20 (the
    gradients come out times their amplitude and are divided once per particle) and on the
    plain table otherwise: a zero and a tiny amplitude (plain table; dL/dA is still
    defined at A = 0) and negative ones (scaled) against the oracle."""
    n, K, C = 1000, 70, 32
    d = soax_inputs.basic_set(n, 7)
    xt = _target(d, K)
    p, loss, xb, vb, g = _gpu_adjoint(d, xt, K, C, th)
    ol, oxb, ovb, og = oracle.adjoint(d["pos"], d["vel"], xt, *th, 1e-3, K, f32v=True)
    ok = ~_diverged(p, d, th, K)
    assert abs(loss - ol) <= 1e-9 * abs(ol)
    assert np.all(np.isfinite(g))
    assert np.allclose(g, og, rtol=1e-8, atol=0), (g, og)
    for c in range(3):
        scale = max(np.abs(oxb[c]).max(), 1e-300)
        assert np.max(np.abs(xb[c] - oxb[c])[ok]) <= 1e-9 * scale
        scale = max(np.abs(ovb[c]).max(), 1e-300)
        assert np.max(np.abs(vb[c] - ovb[c])[ok]) <= 1e-9 * scale


def test_adjoint_scaled_and_plain_forms_agree():
    """An amplitude just at 2^-20 (scaled tables) and the next binary64 below it (plain
    table) differ by one ulp of the amplitude: the two reverse forms give the same
    gradients to float-pair accuracy."""
    n, K, C = 2000, 40, 16
    d = soax_inputs.basic_set(n, 3)
    xt = _target(d, K)
    a = 2.0 ** -20
    _, _, xb1, vb1, g1 = _gpu_adjoint(d, xt, K, C, [1.0, a, 1.05, 0.12])
    _, _, xb2, vb2, g2 = _gpu_adjoint(d, xt, K, C, [1.0, np.nextafter(a, 0.0), 1.05, 0.12])
    assert np.allclose(g1, g2, rtol=1e-9, atol=0), (g1, g2)
    for c in range(3):
        assert np.max(np.abs(xb1[c] - xb2[c])) <= 1e-10 * np.abs(xb1[c]).max()
        assert np.max(np.abs(vb1[c] - vb2[c])) <= 1e-10 * np.abs(vb1[c]).max()


def test_checkpointed_forward_equals_fused_step():
    """The checkpointed forward is soax_step_fused's arithmetic: the same bits as one fused
    launch of K steps."""
    n, K = 20000, 77
    d = soax_inputs.basic_set(n, 3)
    a = sx.Particles(SCHEMA, n, shadow=False)
    a.load({"pos": d["pos"], "vel": d["vel"]})
    b = sx.Particles(SCHEMA, n, shadow=False)
    b.load({"pos": d["pos"], "vel": d["vel"]})
    f = sx.Flow()
    a.step_fused(f, K)
    ws = b.adjoint_workspace(K, 32)
    b.step_checkpointed(f, K, 32, ws)
    x, y = a.numpy(), b.numpy()
    for k in x:
        for u, v in zip(x[k], y[k]):
            assert u.tobytes() == v.tobytes()


def test_checkpointed_forward_with_acceleration_equals_fused_step():
    """With an acceleration field the checkpointed forward (its ACC kernel) stores the
    same positions, velocities and last-stage accelerations as the fused step, and the
    adjoint still runs (the acceleration is an output only, not differentiated)."""
    n, K = 5003, 40
    d = soax_inputs.wide_set(n, 6)
    schema = [("pos", "f64", 3, "P"), ("vel", "f32", 3, "V"), ("acc", "f32", 3, "A")]
    a = sx.Particles(schema, n, shadow=False)
    b = sx.Particles(schema, n, shadow=False)
    for q in (a, b):
        q.load({"pos": d["pos"], "vel": d["vel"], "acc": d["acc"]})
    f = sx.Flow(tau=0.15, dt=1e-3, acc="acc")
    a.step_fused(f, K)
    ws = b.adjoint_workspace(K, 16)
    b.step_checkpointed(f, K, 16, ws)
    x, y = a.numpy(), b.numpy()
    for k in ("pos", "vel", "acc"):
        for u, v in zip(x[k], y[k]):
            assert u.tobytes() == v.tobytes(), k
    assert not np.array_equal(y["acc"][0], d["acc"][0])
    xt = [torch.from_numpy(p.copy()).cuda() for p in d["pos"]]
    _, xb = b.minimage_loss(xt, ws)
    _, _, g = b.step_adjoint(f, K, 16, ws, xb)
    assert np.all(np.isfinite(g.cpu().numpy()))


def test_zero_steps_passes_the_seed_through():
    """K = 0: no step, so x̄0 = x̄K and v̄0 = v̄K (to the float-pair precision the reverse
    carries adjoints in: 48 significant bits, so binary64 seeds come back within 2^-47
    relative, and exactly where they fit in 48 bits) and the parameter gradients are zero."""
    n = 3000
    d = soax_inputs.basic_set(n, 8)
    p = sx.Particles(SCHEMA, n, shadow=False)
    p.load({"pos": d["pos"], "vel": d["vel"]})
    f = sx.Flow()
    ws = p.adjoint_workspace(0, 32)
    p.step_checkpointed(f, 0, 32, ws)
    xt = [torch.from_numpy(np.roll(a, 1).copy()).cuda() for a in d["pos"]]
    _, xb = p.minimage_loss(xt, ws)
    vk = [torch.full((n,), 0.25, dtype=torch.float64, device="cuda") for _ in range(3)]
    xb0, vb0, g = p.step_adjoint(f, 0, 32, ws, xb, vk)
    for c in range(3):
        assert torch.allclose(xb0[c], xb[c], rtol=2.0 ** -47, atol=0.0)
        assert torch.equal(vb0[c], vk[c])  # 0.25 fits in 48 bits
    assert np.all(g.cpu().numpy() == 0.0)
    g2 = p.numpy()
    for c in range(3):
        assert np.array_equal(g2["pos"][c], d["pos"][c]) and np.array_equal(g2["vel"][c], d["vel"][c])


def test_zero_gradient_at_target():
    """Targets from the same forward: the loss and every gradient are exactly zero."""
    n, K = 2000, 64
    d = soax_inputs.basic_set(n, 4)
    t = sx.Particles(SCHEMA, n, shadow=False)
    t.load({"pos": d["pos"], "vel": d["vel"]})
    t.step_fused(sx.Flow(A=1.1), K)
    xt = t.numpy()["pos"]
    ot = [a.copy() for a in d["pos"]]
    oracle.step_soa(ot, [a.copy() for a in d["vel"]], 1.1, 1.0, 1.0, 0.1, 1e-3, K)
    assert all(np.max(np.abs(a - b)) < 1e-9 for a, b in zip(xt, ot))
    p, loss, xb, vb, g = _gpu_adjoint(d, xt, K, 32, [1.1, 1.0, 1.0, 0.1])
    assert loss == 0.0 and np.all(g == 0.0)
    assert all(np.all(a == 0) for a in xb + vb)


def test_gradients_vs_central_fd_of_fp64_forward():
    """The GPU adjoint (f32-stored v) against finite differences of the oracle's FP64-state
    forward; the gap is set by the f32 storage, hence the 1e-4 tolerance."""
    n, K, eps = 256, 200, 1e-6
    d = soax_inputs.basic_set(n, 6)
    xt = _target(d, K)
    th = [1.0, 1.0, 1.0, 0.1]
    _, loss, xb, vb, g = _gpu_adjoint(d, xt, K, 32, th)

    def L(t, vel=None):
        p = [a.copy() for a in d["pos"]]
        v = [a.astype(np.float64) for a in (vel or d["vel"])]
        oracle.step_f64state(p, v, *t, 1e-3, K)
        return sum(float(np.sum(((p[c] - xt[c] + np.pi) % (2 * np.pi) - np.pi) ** 2)) for c in range(3)) / n
    for k in range(4):
        tp, tm = list(th), list(th)
        tp[k] += eps
        tm[k] -= eps
        fd = (L(tp) - L(tm)) / (2 * eps)
        assert abs(g[k] - fd) <= 1e-4 * abs(fd) + 1e-10, (k, g[k], fd)


def test_autograd_function():
    n, K = 3000, 50
    d = soax_inputs.basic_set(n, 7)
    xt = _target(d, K)
    x0 = torch.from_numpy(np.stack(d["pos"])).cuda().requires_grad_()
    v0 = torch.from_numpy(np.stack(d["vel"]).astype(np.float64)).cuda().requires_grad_()
    theta = torch.tensor([1.0, 0.9, 1.1, 0.1], dtype=torch.float64, device="cuda", requires_grad=True)
    xk = sx.SoaxRK2.apply(x0, v0, theta, 1e-3, K, 32)
    dd = xk - torch.from_numpy(np.stack(xt)).cuda()
    dd = torch.remainder(dd + np.pi, 2 * np.pi) - np.pi
    loss = (dd * dd).sum() / n
    loss.backward()
    ol, oxb, ovb, og = oracle.adjoint(d["pos"], d["vel"], xt, 1.0, 0.9, 1.1, 0.1, 1e-3, K, f32v=True)
    p = sx.Particles([("pos", "f64", 3, "P"), ("vel", "f32", 3, "V")], n, shadow=False)
    p.load({"pos": d["pos"], "vel": d["vel"]})
    p.step_fused(sx.Flow(A=1.0, B=0.9, C=1.1, tau=0.1), K)
    ok = ~_diverged(p, d, [1.0, 0.9, 1.1, 0.1], K)
    assert np.allclose(theta.grad.cpu().numpy(), og, rtol=1e-8)
    assert np.allclose(v0.grad.cpu().numpy()[:, ok], np.stack(ovb)[:, ok], rtol=1e-8, atol=1e-14)
    assert np.allclose(x0.grad.cpu().numpy()[:, ok], np.stack(oxb)[:, ok], rtol=1e-8, atol=1e-14)


def _target64(d, K, A, tau, dt, threads=None):
    """x_target of the adjoint workload: the oracle's FP64-state forward (v never rounded
    to f32) from the same initial state, with A = A_target."""
    xt = [a.copy() for a in d["pos"]]
    vt = [a.astype(np.float64) for a in d["vel"]]
    oracle.step_f64state(xt, vt, A, 1.0, 1.0, tau, dt, K, threads=threads)
    return xt


def test_adjoint_workload_n1M_k1000():
    """The adjoint workload as it is stated: 1,048,576 particles, K = 1000 steps,
    checkpoints every 32, the target from the oracle's FP64-state forward at A = 1.1.
    Over ALL particles: the loss and the four parameter gradients against the oracle's
    adjoint of the f32-stored forward (rtol 1e-9 and 1e-8), and every particle's x̄0 and
    v̄0 (1e-9 of the largest), except particles whose f32 velocity took the other side of a
    rounding midpoint at some step, each audited as a legitimate flip."""
    w = soax_inputs.WORKLOADS["adjoint_n1M"]
    n, K, C = w["n"], w["K"], w["ckpt_every"]
    d = soax_inputs.basic_set(n, w["seed"])
    xt = _target64(d, K, w["A_target"], w["tau"], w["dt"])
    th = [w["A"], w["B"], w["C"], w["tau"]]
    p, loss, xb, vb, g = _gpu_adjoint(d, xt, K, C, th, dt=w["dt"])
    ol, oxb, ovb, og = oracle.adjoint(d["pos"], d["vel"], xt, *th, w["dt"], K, f32v=True)
    assert np.all(np.isfinite(g)) and np.all(g != 0.0)
    assert abs(loss - ol) <= 1e-9 * abs(ol), (loss, ol)
    assert np.allclose(g, og, rtol=1e-8, atol=0), (g, og)
    ok = ~_diverged(p, d, th, K, dt=w["dt"], max_frac=1e-4)
    for c in range(3):
        assert np.max(np.abs(xb[c] - oxb[c])[ok]) <= 1e-9 * np.abs(oxb[c]).max()
        assert np.max(np.abs(vb[c] - ovb[c])[ok]) <= 1e-9 * np.abs(ovb[c]).max()
    torch.cuda.empty_cache()


def test_adjoint_workload_subset_vs_fd_k1000():
    """The parameter gradients of the adjoint workload (K = 1000, checkpoints every 32,
    the FP64-state target at A = 1.1) on a deterministic subset of 4096 of its particles
    (every 256th), run as a set of its own: against the oracle's adjoint of the f32-stored
    forward (rtol 1e-8), and against central finite differences of the oracle's FP64-state
    forward with eps = 1e-6 (rtol 1e-4: the gap the f32 storage of v opens)."""
    w = soax_inputs.WORKLOADS["adjoint_n1M"]
    n, K, C, eps = w["n"], w["K"], w["ckpt_every"], w["fd_eps"]
    full = soax_inputs.basic_set(n, w["seed"])
    idx = np.arange(0, n, 256)
    d = {k: [np.ascontiguousarray(a[idx]) for a in full[k]] for k in ("pos", "vel")}
    m = idx.size
    xt = _target64(d, K, w["A_target"], w["tau"], w["dt"])
    th = [w["A"], w["B"], w["C"], w["tau"]]
    _, loss, _, _, g = _gpu_adjoint(d, xt, K, C, th, dt=w["dt"])
    ol, _, _, og = oracle.adjoint(d["pos"], d["vel"], xt, *th, w["dt"], K, f32v=True)
    assert abs(loss - ol) <= 1e-9 * abs(ol)
    assert np.allclose(g, og, rtol=1e-8, atol=0), (g, og)

    def L(t):
        x = [a.copy() for a in d["pos"]]
        v = [a.astype(np.float64) for a in d["vel"]]
        oracle.step_f64state(x, v, *t, w["dt"], K)
        return sum(float(np.sum(((x[c] - xt[c] + np.pi) % (2 * np.pi) - np.pi) ** 2)) for c in range(3)) / m
    for k in range(4):
        tp, tm = list(th), list(th)
        tp[k] += eps
        tm[k] -= eps
        fd = (L(tp) - L(tm)) / (2 * eps)
        assert abs(g[k] - fd) <= 1e-4 * abs(fd), (k, g[k], fd)
