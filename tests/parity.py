"""Shared helpers of the GPU parity tests: compare a GPU state with the oracle's and
audit every particle outside the tolerance.

Tolerances (100-step state): positions max |dx| <= 1e-11; velocities
|dv| <= 1e-5 |v_ref| with a floor of 1e-9 absolute (v0 ~ N(0, 0.1^2) can be near 0).

Audit: the f32 storage of v makes the path sensitive to f64 differences of a few ulp
that move v + dt a2 across an f32 rounding midpoint; one such flip changes v by one
f32 ulp and the position by ~tau * ulp.  A particle out of tolerance is replayed one
step at a time on the GPU and in the oracle from the same state; every step must give
positions within 1e-13, and a velocity that differs must be the f32 rounding of some
value near the oracle's binary64 one (rounds_within): within 1e-14 of it relative to the
value, or within the GPU step's absolute error bound, whichever is larger
(flip_window).  Where one f32 ulp exceeds that window this says the two are one ulp
apart with the oracle's value within the window of the midpoint between them.  The bound is an absolute one because the step's error is: v' = v + (dt/tau)
w1 is formed from the flow terms in float pairs (2^-48 relative precision), so its error
before the f32 rounding is at most about (dt/tau) x 2^10 x 2^-53 x the largest amplitude
(some 32 float-pair roundings of terms of that size), plus a few units of 2^-53 from the
update itself; a relative window alone would shrink to nothing for a velocity near zero.
"""
import numpy as np
import torch

import oracle
import paper_1710_03462_b300 as sx

POS_TOL = 1e-11
VEL_RTOL = 1e-5
VEL_ATOL = 1e-9


def flip_window(ovn, A, B, C, tau, dt):
    """Largest accepted distance of the oracle's binary64 v' from the f32 midpoint that
    the GPU rounded across: 1e-14 relative, with the absolute floor of the step's error
    bound, (4 + 2^10 (dt/tau) max(|A|, |B|, |C|)) units of 2^-53."""
    floor = (4.0 + 1024.0 * (dt / tau) * max(abs(A), abs(B), abs(C))) * 2.0 ** -53
    return max(1e-14 * abs(ovn), floor)


def rounds_within(gv, ovn, window):
    """True when the f32 gv is the rounding to nearest of some value within window of the
    oracle's binary64 ovn: gv lies between RN32(ovn - window) and RN32(ovn + window).
    Where one f32 ulp exceeds the window this is the midpoint rule (gv one ulp from
    RN32(ovn), with the midpoint between them within the window of ovn); for a velocity
    near zero, where f32 ulps are finer than the window, it admits every rounding the
    window reaches."""
    return bool(np.float32(ovn - window) <= gv <= np.float32(ovn + window))


def out_of_tolerance(gpos, gvel, opos, ovel):
    """Boolean mask of particles whose GPU state misses the tolerance."""
    bad = np.zeros(gpos[0].size, bool)
    for c in range(3):
        d = np.abs(gpos[c] - opos[c])
        d = np.minimum(d, sx.TWO_PI - d)  # the same point seen across the periodic wrap
        bad |= d > POS_TOL
        bad |= np.abs(gvel[c].astype(np.float64) - ovel[c]) > np.maximum(VEL_RTOL * np.abs(ovel[c]), VEL_ATOL)
    return bad


def assert_acc(gacc, oacc, gpos, gvel, opos, ovel):
    """The stored acceleration is f32(a2) of the last step: one rounding of a
    binary64-accurate value.  On particles whose stored velocities equal the oracle's bit
    for bit and whose positions agree within 1e-12, it must equal the oracle's f32 value
    or be one f32 ulp away (a2 within the step's error of a rounding midpoint).  A particle
    that took an accepted velocity flip (audited through its position and velocity) follows
    the flipped trajectory: a one-ulp change of v moves a2 by about ulp(v)/tau, so there
    acc is held to the velocity tolerance, 1e-5 relative with a 1e-6 absolute floor."""
    same = np.ones(gacc[0].size, bool)
    for c in range(3):
        d = np.abs(gpos[c] - opos[c])
        same &= np.minimum(d, sx.TWO_PI - d) <= 1e-12
        same &= gvel[c] == ovel[c]
    for c in range(3):
        g = np.ascontiguousarray(gacc[c], np.float32)
        o = np.ascontiguousarray(oacc[c], np.float32)
        up = np.nextafter(o, np.float32(np.inf))
        dn = np.nextafter(o, np.float32(-np.inf))
        ulp_ok = (g == o) | (g == up) | (g == dn)
        assert np.all(ulp_ok[same]), f"acc[{c}]: {np.count_nonzero(~ulp_ok[same])} particles beyond one f32 ulp"
        near = np.abs(g.astype(np.float64) - o) <= 1e-5 * np.abs(o) + 1e-6
        assert np.all(near[~same]), f"acc[{c}]: a flipped particle beyond the velocity tolerance"
    return int(np.count_nonzero(same))


def gpu_one_step(x3, v3, A, B, C, tau, dt):
    p = sx.Particles([("pos", "f64", 3, "P"), ("vel", "f32", 3, "V")], 1, shadow=False)
    p.load({"pos": [np.array([x]) for x in x3], "vel": [np.array([v], np.float32) for v in v3]})
    p.step(sx.Flow(A=A, B=B, C=C, tau=tau, dt=dt), 1)
    d = p.numpy()
    return np.array([a[0] for a in d["pos"]]), np.array([a[0] for a in d["vel"]], np.float32)


def audit_particle(x0, v0, A, B, C, tau, dt, steps):
    """Replay one particle; returns the number of accepted midpoint flips or raises."""
    x = np.array(x0, np.float64)
    v = np.array(v0, np.float32)
    flips = 0
    for s in range(steps):
        gx, gv = gpu_one_step(x, v, A, B, C, tau, dt)
        ox, ovn, _ = oracle.step_one_detail(A, B, C, tau, dt, x, v)
        ov = ovn.astype(np.float32)
        dx = np.abs(gx - ox)
        dx = np.minimum(dx, sx.TWO_PI - dx)
        assert np.all(dx <= 1e-13), f"step {s}: position differs by {dx.max()}"
        for c in range(3):
            if gv[c] != ov[c]:
                assert rounds_within(gv[c], ovn[c], flip_window(ovn[c], A, B, C, tau, dt)), \
                    f"step {s}: velocity {gv[c]!r} is no rounding of the oracle's {ovn[c]!r} within the window"
                flips += 1
        x, v = ox, ov
    return flips


def assert_parity(gpos, gvel, opos, ovel, x0, v0, taus, A, B, C, dt, steps, max_audit=20):
    """Tolerance check, with an audit of each particle out of tolerance."""
    bad = np.flatnonzero(out_of_tolerance(gpos, gvel, opos, ovel))
    assert bad.size <= max_audit, f"{bad.size} particles out of tolerance"
    for i in bad:
        audit_particle([x0[c][i] for c in range(3)], [v0[c][i] for c in range(3)], A, B, C, float(taus[i]), dt, steps)
    return bad.size


def gpu_fused_steps(x3, v3, A, B, C, tau, dt, steps):
    """One particle advanced `steps` steps in one soax_step_fused launch."""
    p = sx.Particles([("pos", "f64", 3, "P"), ("vel", "f32", 3, "V")], 1, shadow=False)
    p.load({"pos": [np.array([x]) for x in x3], "vel": [np.array([v], np.float32) for v in v3]})
    p.step_fused(sx.Flow(A=A, B=B, C=C, tau=tau, dt=dt), steps)
    d = p.numpy()
    return np.array([a[0] for a in d["pos"]]), np.array([a[0] for a in d["vel"]], np.float32)


def audit_particle_fused(x0, v0, A, B, C, tau, dt, steps):
    """Audit of a particle that soax_step_fused left out of tolerance.  The fused kernel
    keeps its position between steps in fixed point, so it is replayed on its own
    trajectory: the first s steps of a fused launch are the state a launch of s steps
    returns.  Up to the first step whose f32 velocity differs from the oracle's, positions
    must agree within 1e-13 per step; at that step each differing velocity must be the
    f32 rounding of a value within flip_window of the oracle's binary64 one (rounds_within).
    Later steps follow from that flip.  A particle out of tolerance with no such
    flip fails."""
    x = np.array(x0, np.float64)
    v = np.array(v0, np.float32)
    for s in range(1, steps + 1):
        ox, ovn, _ = oracle.step_one_detail(A, B, C, tau, dt, x, v)
        ov = ovn.astype(np.float32)
        gx, gv = gpu_fused_steps(x0, v0, A, B, C, tau, dt, s)
        dx = np.abs(gx - ox)
        dx = np.minimum(dx, sx.TWO_PI - dx)
        assert np.all(dx <= 1e-13 * s), f"step {s}: position differs by {dx.max()}"
        if not np.array_equal(gv, ov):
            for c in range(3):
                if gv[c] != ov[c]:
                    assert rounds_within(gv[c], ovn[c], flip_window(ovn[c], A, B, C, tau, dt)), \
                        f"step {s}: velocity {gv[c]!r} is no rounding of the oracle's {ovn[c]!r} within the window"
            return 1
        x, v = ox, ov
    raise AssertionError("out of tolerance without a velocity flip")


def assert_parity_fused(gpos, gvel, opos, ovel, x0, v0, taus, A, B, C, dt, steps, max_audit=20):
    """assert_parity for soax_step_fused results (audit_particle_fused)."""
    bad = np.flatnonzero(out_of_tolerance(gpos, gvel, opos, ovel))
    assert bad.size <= max_audit, f"{bad.size} particles out of tolerance"
    for i in bad:
        audit_particle_fused([x0[c][i] for c in range(3)], [v0[c][i] for c in range(3)], A, B, C, float(taus[i]),
                             dt, steps)
    return bad.size
