"""Seeded synthetic particle sets -- shared by the tests, the bench and smoke().

This module only draws random numbers; it holds none of the method's arithmetic, so
both the CUDA path and the CPU oracle can take their inputs from it without sharing
code.  The paper benchmarks on synthetic particles (Sec. 2: positions and velocities of
a set of particles advanced by Eq. 1); these sets follow the same idea with the
workloads' record types and sizes.

Draw order (numpy PCG64, default_rng(seed)):
  * id = arange(n)                                  (i32, or i64 for the wide record)
  * pos = uniform(0, 2pi, (3, n)) clamped below 2pi (f64)
  * vel = normal(0, 0.1, (3, n)).astype(f32)
  * wide record only: acc = 0 (f32 x 3); mass = exp(uniform(ln 0.1, ln 10, n)) as f32;
    tag = integers(0, 8, n) as u8.
"""
import math

import numpy as np

TWO_PI = 6.283185307179586
_BELOW_TWO_PI = np.nextafter(TWO_PI, 0.0)

# Workload parameters (flow amplitudes, tau, dt, steps, sort grid and cadence).
WORKLOADS = {
    "plain_n65536": dict(n=65536, A=1.0, B=1.0, C=1.0, tau=0.1, dt=1e-3, steps=100, seed=0),
    "sorted_n16M": dict(n=16777216, A=1.0, B=1.0, C=1.0, tau=0.1, dt=1e-3, steps=1000, grid=32,
                        sort_every=10, seed=0),
    "wide_n64M": dict(n=67108864, A=1.0, B=1.0, C=1.0, tau_scale=0.1, dt=5e-4, steps=200, grid=64,
                      sort_every=20, seed=0),
    "adjoint_n1M": dict(n=1048576, A=1.0, B=1.0, C=1.0, tau=0.1, dt=1e-3, K=1000, ckpt_every=32,
                        A_target=1.1, fd_eps=1e-6, seed=0),
    "batched_512": dict(nens=512, nmin=1024, nmax=4194304, dt=1e-3, steps=200, seed=0),
}


def basic_set(n, seed=0, id_dtype=np.int32):
    """id, pos[3], vel[3] for n particles (the record {int id; double pos[3]; float vel[3]})."""
    rng = np.random.default_rng(seed)
    ids = np.arange(n, dtype=id_dtype)
    pos = rng.uniform(0.0, TWO_PI, (3, n))
    pos = np.minimum(pos, _BELOW_TWO_PI)
    vel = rng.normal(0.0, 0.1, (3, n)).astype(np.float32)
    return {"id": [ids], "pos": [np.ascontiguousarray(p) for p in pos],
            "vel": [np.ascontiguousarray(v) for v in vel]}


def wide_set(n, seed=0):
    """The wide heterogeneous record: i64 id, f64 pos[3], f32 vel[3], f32 acc[3], f32 mass,
    u8 tag."""
    rng = np.random.default_rng(seed)
    ids = np.arange(n, dtype=np.int64)
    pos = np.minimum(rng.uniform(0.0, TWO_PI, (3, n)), _BELOW_TWO_PI)
    vel = rng.normal(0.0, 0.1, (3, n)).astype(np.float32)
    acc = np.zeros((3, n), np.float32)
    mass = np.exp(rng.uniform(math.log(0.1), math.log(10.0), n)).astype(np.float32)
    tag = rng.integers(0, 8, n, dtype=np.uint8)
    return {"id": [ids], "pos": [np.ascontiguousarray(p) for p in pos],
            "vel": [np.ascontiguousarray(v) for v in vel], "acc": [np.ascontiguousarray(a) for a in acc],
            "mass": [mass], "tag": [tag]}


def ensembles(nens=512, nmin=1024, nmax=4194304, seed=0):
    """Per-ensemble sizes (log-uniform), tau ~ U[0.01, 1] and (A, B, C) ~ U[0.5, 1.5]."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), nens))).astype(np.int64)
    tau = rng.uniform(0.01, 1.0, nens)
    abc = rng.uniform(0.5, 1.5, (nens, 3))
    return sizes, tau, abc


def ensemble_set(e, n):
    """Particles of ensemble e: the basic generator with seed 1000 + e."""
    return basic_set(int(n), seed=1000 + int(e))
