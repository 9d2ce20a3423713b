"""The GPU parity helpers' host-side rules without a GPU: the flip audit's window."""
import numpy as np

from parity import flip_window, rounds_within


def test_flip_window_floor_and_relative_part():
    u = 2.0 ** -53
    # The workloads (dt/tau = 0.01, unit amplitudes): 4 + 10.24 units of 2^-53 absolute.
    assert flip_window(1e-4, 1.0, 1.0, 1.0, 0.1, 1e-3) == (4.0 + 10.24) * u
    # Large velocities keep the relative 1e-14 window.
    assert flip_window(2.0, 1.0, 1.0, 1.0, 0.1, 1e-3) == 2e-14
    # The floor grows with dt/tau and the largest amplitude.
    assert flip_window(0.0, 1.4, 0.6, -1.5, 0.004, 2e-3) == (4.0 + 1024.0 * 0.5 * 1.5) * u
    # A GPU error of 1e-12 at the workloads (a real arithmetic fault, ~9000 units) is
    # outside the window: such a flip fails the audit.
    assert flip_window(0.1, 1.0, 1.0, 1.0, 0.1, 1e-3) < 1e-12 / 100
    assert np.isfinite(flip_window(0.0, 0.0, 0.0, 0.0, 0.1, 1e-3))


def test_rounds_within():
    w = 14.24 * 2.0 ** -53
    # One ulp apart, the midpoint within the window: accepted; farther: rejected.
    x = np.float64(np.float32(0.1)) + np.float64(np.spacing(np.float32(0.1))) / 2 - 0.5 * w
    assert rounds_within(np.nextafter(np.float32(0.1), np.float32(1)), x, w)
    assert not rounds_within(np.nextafter(np.float32(0.1), np.float32(1)), x - 2 * w, w)
    # Two ulps apart at an ordinary magnitude: never.
    assert not rounds_within(np.float32(0.1) + 2 * np.spacing(np.float32(0.1)), 0.1, w)
    # Near zero the window spans many f32 values: each rounding it reaches is accepted.
    assert rounds_within(np.float32(-1.7332225e-10), -1.7332234390047305e-10, w)
    assert not rounds_within(np.float32(-1.7e-10), -1.7332234390047305e-10, w)
