"""Zero flow (A = B = C = 0), the method's degenerate case: u = 0, so every step only
multiplies v by g = 1 - h + h^2/2 (h = dt/tau) before its f32 rounding and the positions
follow x_K = x0 + tau v0 (1 - g^K).  The amplitude-scaled tables are all zero and the
adjoint takes the plain table (every amplitude below 2^-20).  Every form against the
oracle, and the adjoint's gradients with respect to the amplitudes (still defined: the
flow's sensitivity to switching it on)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1710_03462_b300 as sx
import soax_inputs
from parity import assert_parity, assert_parity_fused

pytestmark = pytest.mark.gpu

A = B = C = 0.0
TAU, DT, STEPS = 0.1, 1e-3, 20


def _data(n, seed):
    return soax_inputs.basic_set(n, seed)


def _oracle(d, steps=STEPS):
    opos = [a.copy() for a in d["pos"]]
    ovel = [a.copy() for a in d["vel"]]
    oracle.step_soa(opos, ovel, A, B, C, TAU, DT, steps)
    return opos, ovel


@pytest.mark.parametrize("form", ["one_pass", "fused", "aos"])
def test_zero_flow_steps(form):
    n = 20001
    d = _data(n, 61)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    p.load(d)
    f = sx.Flow(A=A, B=B, C=C, tau=TAU, dt=DT)
    if form == "one_pass":
        p.step(f, STEPS)
    elif form == "fused":
        p.step_fused(f, STEPS)
    else:
        aos = p.to_aos()
        p.step_aos(aos, f, STEPS)
        p.from_aos(aos)
    g = p.numpy()
    opos, ovel = _oracle(d)
    taus = np.full(n, TAU)
    check = assert_parity_fused if form == "fused" else assert_parity
    check(g["pos"], g["vel"], opos, ovel, d["pos"], d["vel"], taus, A, B, C, DT, STEPS)
    # The closed form of the positions, up to the f32 roundings of v along the way: after
    # n steps v is off v0 g^n by at most n 2^-24 |v|, which moves x by at most
    # dt K^2/2 2^-24 max|v| (7e-9 here).
    h = DT / TAU
    gk = (1 - h + h * h / 2) ** STEPS
    vmax = max(float(np.abs(v).max()) for v in d["vel"])
    for c in range(3):
        x = d["pos"][c] + TAU * d["vel"][c].astype(np.float64) * (1 - gk)
        dx = np.abs(g["pos"][c] - np.mod(x, sx.TWO_PI))
        assert np.max(np.minimum(dx, sx.TWO_PI - dx)) <= DT * STEPS ** 2 / 2 * 2.0 ** -24 * vmax * 1.01


def test_zero_flow_adjoint():
    n, K, Ck = 2000, 40, 16
    d = _data(n, 62)
    xt = [a.copy() for a in d["pos"]]
    vt = [a.copy() for a in d["vel"]]
    oracle.step_soa(xt, vt, 0.3, 0.0, 0.0, TAU, DT, K)  # targets from a weak flow
    p = sx.Particles([("pos", "f64", 3, "P"), ("vel", "f32", 3, "V")], n, shadow=False)
    p.load({"pos": d["pos"], "vel": d["vel"]})
    f = sx.Flow(A=A, B=B, C=C, tau=TAU, dt=DT)
    ws = p.adjoint_workspace(K, Ck)
    p.step_checkpointed(f, K, Ck, ws)
    loss, xb = p.minimage_loss([torch.from_numpy(a).cuda() for a in xt], ws)
    xb0, vb0, g = p.step_adjoint(f, K, Ck, ws, xb)
    ol, oxb, ovb, og = oracle.adjoint(d["pos"], d["vel"], xt, A, B, C, TAU, DT, K, f32v=True)
    assert abs(float(loss.item()) - ol) <= 1e-9 * abs(ol)
    g = g.cpu().numpy()
    assert np.all(np.isfinite(g)) and np.all(g[:3] != 0.0)
    assert np.allclose(g, og, rtol=1e-8, atol=0)
    # The target flow moves x and y only, so the z adjoints are zero up to rounding: the
    # tolerance is scaled by the largest adjoint over all components.
    sx_ = max(float(np.abs(a).max()) for a in oxb)
    sv_ = max(float(np.abs(a).max()) for a in ovb)
    for c in range(3):
        assert np.allclose(xb0[c].cpu().numpy(), oxb[c], rtol=1e-9, atol=1e-9 * sx_)
        assert np.allclose(vb0[c].cpu().numpy(), ovb[c], rtol=1e-9, atol=1e-9 * sv_)
