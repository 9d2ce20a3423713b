"""ctypes wrapper around libsoax_oracle.so (test infrastructure only).

Numpy in, numpy out.  Every function here only marshals arguments; the arithmetic is
in soax_oracle.c.  Functions:

  flow(A, B, C, x, y, z)                    ABC flow u(x) (workload definition)
  step_soa(pos, vel, A, B, C, tau, dt, n)   midpoint-RK2 steps on SoA planes, in place
  step_aos(rec, rb, pos_off, vel_off, ...)  the same on AoS records, in place
  step_one_detail(...)                      one step of one particle, f64 v before rounding
  step_f64state(...)                        FP64-state forward (v never rounded)
  cell_keys(px, py, pz, G)                  linear cell index on a G^3 grid
  stable_argsort(keys)                      stable ascending argsort (+ sorted keys)
  permute(planes, perm)                     out[i] = in[perm[i]] for every plane
  aos_layout(elem_bytes, ncomp)             natural C struct layout (Listing 1, 4)
  soa_to_aos / aos_to_soa                   byte-exact transposes (Listing 6)
  adjoint(...)                              loss and reverse-mode gradients
  euler_f32(x, v, dt)                       the paper's Eq. 1 step
  euler_aos_f32(rec, rb, x_off, v_off, dt)  the same on Particle<SIZE> records (Listing 4)
  fill(plane, value)                        SetToValue on one array (Listing 7)
  lincomb(dst, srcs, coefs, constant)       dst = constant + sum coef_k src_k (Listing 5)
  remove(planes, idx)                       removal by overwriting with the last ones (Sec. 2)
  expr(program, compute, out_dtype)         a postfix expression over whole arrays (Sec. 4.2)
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

TWO_PI = 6.283185307179586

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        p, i64, d = C.c_void_p, C.c_int64, C.c_double
        L.orc_flow.argtypes = [d, d, d, i64, p, p, p, p, p, p]
        L.orc_step_soa.argtypes = [i64, p, p, p, p, p, p, p, p, p, p, d, d, d, d, d, d, C.c_int, C.c_int]
        L.orc_step_aos.argtypes = [i64, p, i64, i64, i64, i64, i64, d, d, d, d, d, d, C.c_int, C.c_int]
        L.orc_step_one_detail.argtypes = [d, d, d, d, d, p, p, p, p]
        L.orc_step_f64state.argtypes = [i64, p, p, p, p, p, p, d, d, d, d, d, C.c_int, C.c_int]
        L.orc_cell_keys.argtypes = [i64, p, p, p, C.c_int, p]
        L.orc_stable_argsort.argtypes = [i64, p, p, p]
        L.orc_stable_argsort.restype = C.c_int
        L.orc_permute.argtypes = [i64, C.c_int, p, p, p, p]
        L.orc_aos_layout.argtypes = [C.c_int, p, p, p]
        L.orc_aos_layout.restype = i64
        L.orc_soa_to_aos.argtypes = [i64, C.c_int, p, p, p, p]
        L.orc_aos_to_soa.argtypes = [i64, C.c_int, p, p, p, p]
        L.orc_adjoint.argtypes = ([i64] + [p] * 3 + [p] * 3 + [p] * 3 + [p] * 3 + [d] * 5 +
                                  [C.c_int, C.c_int] + [p] * 6 + [p, p, C.c_int])
        L.orc_adjoint.restype = C.c_int
        L.orc_euler_f32.argtypes = [i64, p, p, C.c_float]
        L.orc_euler_aos_f32.argtypes = [i64, p, i64, i64, i64, C.c_float]
        L.orc_fill.argtypes = [i64, p, C.c_int, d]
        L.orc_remove.argtypes = [i64, C.c_int, p, p, p, i64]
        L.orc_remove.restype = i64
        L.orc_lincomb.argtypes = [i64, C.c_int, p, C.c_int, p, p, d]
        L.orc_expr.argtypes = [i64, C.c_int, C.c_int, p, p, p, p, p, C.c_int]
        _lib = L
    return _lib


def default_threads():
    return max(1, os.cpu_count() or 1)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _need(a, dtype):
    if not (isinstance(a, np.ndarray) and a.dtype == dtype and a.flags.c_contiguous):
        raise TypeError(f"expected contiguous {np.dtype(dtype)} array")
    return a


def flow(A, B, C_, x, y, z):
    x, y, z = (np.ascontiguousarray(a, np.float64) for a in (x, y, z))
    n = x.size
    ux, uy, uz = np.empty(n), np.empty(n), np.empty(n)
    lib().orc_flow(A, B, C_, n, _p(x), _p(y), _p(z), _p(ux), _p(uy), _p(uz))
    return ux, uy, uz


def step_soa(pos, vel, A, B, C_, tau, dt, nsteps, acc=None, mass=None, tau_scale=0.0,
             threads=None):
    """pos: 3 f64 planes, vel: 3 f32 planes (modified in place); acc: 3 f32 planes or
    None; mass: f32 plane or None (then tau is uniform, else tau_i = tau_scale*mass_i)."""
    px, py, pz = (_need(a, np.float64) for a in pos)
    vx, vy, vz = (_need(a, np.float32) for a in vel)
    ax, ay, az = (None, None, None) if acc is None else tuple(_need(a, np.float32) for a in acc)
    if mass is not None:
        _need(mass, np.float32)
    n = px.size
    lib().orc_step_soa(n, _p(px), _p(py), _p(pz), _p(vx), _p(vy), _p(vz), _p(ax), _p(ay),
                       _p(az), _p(mass), A, B, C_, tau, tau_scale, dt, int(nsteps),
                       threads or default_threads())


def step_aos(rec, record_bytes, pos_off, vel_off, A, B, C_, tau, dt, nsteps, acc_off=-1,
             mass_off=-1, tau_scale=0.0, threads=None):
    _need(rec, np.uint8)
    n = rec.size // record_bytes
    lib().orc_step_aos(n, _p(rec), record_bytes, pos_off, vel_off, acc_off, mass_off, A, B,
                       C_, tau, tau_scale, dt, int(nsteps), threads or default_threads())


def step_one_detail(A, B, C_, tau, dt, x3, v3):
    """One step of one particle. Returns (x' f64[3], v' before f32 rounding f64[3], a2)."""
    x = np.array(x3, np.float64)
    v = np.array(v3, np.float32)
    vn, a2 = np.empty(3), np.empty(3)
    lib().orc_step_one_detail(A, B, C_, tau, dt, _p(x), _p(v), _p(vn), _p(a2))
    return x, vn, a2


def step_f64state(pos, vel, A, B, C_, tau, dt, nsteps, threads=None):
    px, py, pz = (_need(a, np.float64) for a in pos)
    vx, vy, vz = (_need(a, np.float64) for a in vel)
    lib().orc_step_f64state(px.size, _p(px), _p(py), _p(pz), _p(vx), _p(vy), _p(vz), A, B, C_,
                            tau, dt, int(nsteps), threads or default_threads())


def cell_keys(px, py, pz, G):
    px, py, pz = (_need(a, np.float64) for a in (px, py, pz))
    keys = np.empty(px.size, np.uint32)
    lib().orc_cell_keys(px.size, _p(px), _p(py), _p(pz), int(G), _p(keys))
    return keys


def stable_argsort(keys):
    keys = _need(keys, np.uint32)
    perm = np.empty(keys.size, np.uint32)
    sk = np.empty(keys.size, np.uint32)
    if lib().orc_stable_argsort(keys.size, _p(keys), _p(perm), _p(sk)) != 0:
        raise MemoryError("oracle argsort")
    return perm, sk


def permute(planes, perm):
    perm = _need(perm, np.uint32)
    planes = [np.ascontiguousarray(a) for a in planes]
    outs = [np.empty_like(a) for a in planes]
    k = len(planes)
    ins = (C.c_void_p * k)(*[a.ctypes.data for a in planes])
    ous = (C.c_void_p * k)(*[a.ctypes.data for a in outs])
    eb = np.array([a.dtype.itemsize for a in planes], np.int32)
    lib().orc_permute(perm.size, k, ins, ous, _p(eb), _p(perm))
    return outs


def aos_layout(elem_bytes, ncomp):
    eb = np.array(elem_bytes, np.int32)
    nc = np.array(ncomp, np.int32)
    offs = np.empty(len(eb), np.int64)
    rb = lib().orc_aos_layout(len(eb), _p(eb), _p(nc), _p(offs))
    return int(rb), [int(o) for o in offs]


def soa_to_aos(planes, elem_bytes, ncomp):
    """planes: one array per (field, component) in schema order."""
    eb = np.array(elem_bytes, np.int32)
    nc = np.array(ncomp, np.int32)
    rb, _ = aos_layout(elem_bytes, ncomp)
    n = planes[0].size
    planes = [np.ascontiguousarray(a) for a in planes]
    rec = np.empty(n * rb, np.uint8)
    arr = (C.c_void_p * len(planes))(*[a.ctypes.data for a in planes])
    lib().orc_soa_to_aos(n, len(eb), _p(eb), _p(nc), arr, _p(rec))
    return rec


def aos_to_soa(rec, elem_bytes, ncomp, dtypes):
    """dtypes: numpy dtype per field; returns one plane per (field, component)."""
    eb = np.array(elem_bytes, np.int32)
    nc = np.array(ncomp, np.int32)
    rb, _ = aos_layout(elem_bytes, ncomp)
    rec = _need(rec, np.uint8)
    n = rec.size // rb
    planes = []
    for f, dt in enumerate(dtypes):
        for _ in range(int(nc[f])):
            planes.append(np.empty(n, dt))
    arr = (C.c_void_p * len(planes))(*[a.ctypes.data for a in planes])
    lib().orc_aos_to_soa(n, len(eb), _p(eb), _p(nc), _p(rec), arr)
    return planes


def adjoint(pos0, vel0, xtgt, A, B, C_, tau, dt, K, f32v=True, threads=None):
    """Returns (loss, xbar0 [3 planes], vbar0 [3 planes], grad[A, B, C, tau]).
    f32v: velocity stored as f32 each step (vel0 must be f32), else FP64 state."""
    x0 = [_need(a, np.float64) for a in pos0]
    xt = [_need(a, np.float64) for a in xtgt]
    n = x0[0].size
    if f32v:
        vf = [_need(a, np.float32) for a in vel0]
        vd = [None] * 3
    else:
        vd = [_need(a, np.float64) for a in vel0]
        vf = [None] * 3
    xb = [np.empty(n) for _ in range(3)]
    vb = [np.empty(n) for _ in range(3)]
    grad = np.empty(4)
    loss = np.empty(1)
    rc = lib().orc_adjoint(n, *[_p(a) for a in x0], *[_p(a) for a in vf], *[_p(a) for a in vd],
                           *[_p(a) for a in xt], A, B, C_, tau, dt, int(K), 1 if f32v else 0,
                           *[_p(a) for a in xb], *[_p(a) for a in vb], _p(grad), _p(loss),
                           threads or default_threads())
    if rc != 0:
        raise MemoryError("oracle adjoint")
    return float(loss[0]), xb, vb, grad


def euler_f32(x, v, dt):
    _need(x, np.float32)
    _need(v, np.float32)
    lib().orc_euler_f32(x.size, _p(x), _p(v), np.float32(dt))


def euler_aos_f32(rec, record_bytes, x_off, v_off, dt):
    _need(rec, np.uint8)
    lib().orc_euler_aos_f32(rec.size // record_bytes, _p(rec), record_bytes, x_off, v_off, np.float32(dt))


_TCODES = {np.dtype(np.int32): 0, np.dtype(np.int64): 1, np.dtype(np.uint8): 2, np.dtype(np.float32): 3,
           np.dtype(np.float64): 4}


def fill(plane, value):
    plane = np.ascontiguousarray(plane)
    lib().orc_fill(plane.size, _p(plane), _TCODES[plane.dtype], float(value))
    return plane


def lincomb(dst, srcs, coefs, constant=0.0):
    is32 = dst.dtype == np.float32
    srcs = [_need(a, dst.dtype) for a in srcs]
    _need(dst, dst.dtype)
    arr = (C.c_void_p * max(1, len(srcs)))(*[a.ctypes.data for a in srcs])
    cf = np.array(coefs, np.float64)
    lib().orc_lincomb(dst.size, 1 if is32 else 0, _p(dst), len(srcs), arr, _p(cf), float(constant))
    return dst


def remove(planes, idx):
    """Returns the planes after removing the particles at the ascending distinct indices
    idx: removed positions below n - k receive the surviving particles of the last k
    positions, both in ascending order."""
    planes = [np.ascontiguousarray(a).copy() for a in planes]
    idx = np.ascontiguousarray(idx, np.uint32)
    n = planes[0].size
    k = len(planes)
    arr = (C.c_void_p * k)(*[a.ctypes.data for a in planes])
    eb = np.array([a.dtype.itemsize for a in planes], np.int32)
    m = lib().orc_remove(n, k, arr, _p(eb), _p(idx), idx.size)
    return [a[:m].copy() for a in planes]


_EXPR_OPS = {"load": 0, "const": 1, "add": 2, "sub": 3, "mul": 4, "div": 5, "neg": 6, "abs": 7, "sqrt": 8,
             "min": 9, "max": 10, "fma": 11}


def expr(program, compute="f64", out_dtype=np.float64, n=None):
    """Evaluate a postfix program element by element (orc_expr).  program: a list of
    ("load", array), ("const", value) or an operator name (add, sub, mul, div, neg, abs,
    sqrt, min, max, fma); compute: "f32" or "f64"; every loaded array has n elements (n
    may be omitted when the program loads an array).  Returns the result array of
    out_dtype (float32 or float64)."""
    ops, vals, srcs, codes, keep = [], [], [], [], []
    for item in program:
        name, arg = (item, None) if isinstance(item, str) else item
        ops.append(_EXPR_OPS[name])
        vals.append(float(arg) if name == "const" else 0.0)
        if name == "load":
            a = np.ascontiguousarray(arg)
            n = a.size if n is None else n
            if a.size != n:
                raise ValueError("expr: loaded arrays differ in length")
            keep.append(a)
            srcs.append(a.ctypes.data)
            codes.append(_TCODES[a.dtype])
        else:
            srcs.append(None)
            codes.append(0)
    n = 0 if n is None else n
    out = np.empty(n, out_dtype)
    op = np.array(ops, np.int32)
    val = np.array(vals, np.float64)
    code = np.array(codes, np.int32)
    arr = (C.c_void_p * len(srcs))(*srcs)
    lib().orc_expr(n, 1 if compute == "f32" else 0, len(ops), _p(op), _p(val), arr, _p(code), _p(out),
                   1 if np.dtype(out_dtype) == np.float32 else 0)
    return out
