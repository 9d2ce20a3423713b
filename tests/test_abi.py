"""The C ABI without a GPU: the library builds and loads, exports every symbol that
include/*.h declare, and validates arguments on the host (no device work)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

import paper_1710_03462_b300 as sx
from paper_1710_03462_b300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = "".join(open(f).read() for f in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(soax_\w+)\s*\(", src, re.M)))


def test_exports_every_declared_symbol():
    L = sx.lib()
    names = _declared()
    assert len(names) >= 25
    for n in names:
        assert hasattr(L, n), n
    assert sorted(_abi.EXPORTS) == names


def _create(schema, n):
    descs = (_abi.soax_field_desc * len(schema))()
    keep = []
    for k, (name, dt, nc, tag) in enumerate(schema):
        b = name.encode()
        keep.append(b)
        descs[k] = _abi.soax_field_desc(b, _abi.DTYPES.get(dt, 99), nc, tag.encode())
    h = C.c_void_p()
    rc = sx.lib().soax_create(descs, len(schema), n, C.byref(h))
    return rc, h


def test_version_and_layout():
    L = sx.lib()
    assert L.soax_version() == 1
    rc, h = _create(sx.WIDE_SCHEMA, 10)
    assert rc == 0
    rb = C.c_int64()
    offs = (C.c_int64 * 6)()
    assert L.soax_aos_layout(h, C.byref(rb), offs) == 0
    assert (rb.value, list(offs)) == (64, [0, 8, 32, 44, 56, 60])
    n, nf, npl = C.c_int64(), C.c_int32(), C.c_int32()
    assert L.soax_size(h, C.byref(n), C.byref(nf), C.byref(npl)) == 0
    assert (n.value, nf.value, npl.value) == (10, 6, 12)
    assert L.soax_destroy(h) == 0


@pytest.mark.parametrize("schema,n", [
    ([("a", "f99", 1, "x")], 4),
    ([("a", "f32", 0, "x")], 4),
    ([("a", "f32", 17, "x")], 4),
    ([("a", "f32", 1, "x"), ("a", "f64", 1, "y")], 4),
    ([("", "f32", 1, "x")], 4),
    ([(f"f{k}", "f32", 16, "x") for k in range(5)], 4),
])
def test_bad_schemas(schema, n):
    rc, h = _create(schema, n)
    assert rc == -2 and not h.value


def test_bad_sizes():
    assert _create(sx.BASIC_SCHEMA, -1)[0] == -1
    assert _create(sx.BASIC_SCHEMA, 2 ** 31)[0] == -1


def test_bind_validation_and_step_validation_without_gpu():
    L = sx.lib()
    rc, h = _create(sx.BASIC_SCHEMA, 100)
    assert L.soax_bind(h, 1, 0, 0, C.c_void_p(0x1008)) == -3   # misaligned
    assert L.soax_bind(h, 1, 3, 0, C.c_void_p(0x1000)) == -1   # bad component
    assert L.soax_bind(h, 5, 0, 0, C.c_void_p(0x1000)) == -1   # bad field
    assert L.soax_bind(h, 1, 0, 2, C.c_void_p(0x1000)) == -1   # bad buffer
    assert L.soax_bind(h, 1, 0, 0, None) == -1
    fl = _abi.soax_flow(1, 1, 1, 0.1, 1e-3, 0.0, -1, 1, 2, -1)
    assert L.soax_step(h, C.byref(fl), 1, None) == -8           # planes not bound
    bad = _abi.soax_flow(1, 1, 1, 0.1, 1e-3, 0.0, -1, 2, 1, -1)  # pos/vel swapped
    assert L.soax_step(h, C.byref(bad), 1, None) == -2
    neg = _abi.soax_flow(1, 1, 1, -0.1, 1e-3, 0.0, -1, 1, 2, -1)
    assert L.soax_step(h, C.byref(neg), 1, None) == -1
    assert L.soax_step(h, C.byref(fl), -1, None) == -1
    assert b"nsteps" in L.soax_last_error()
    assert L.soax_step(None, C.byref(fl), 1, None) == -1
    # The fused step validates the same way, before any launch.
    assert L.soax_step_fused(h, C.byref(fl), 1, None) == -8
    assert L.soax_step_fused(h, C.byref(bad), 1, None) == -2
    assert L.soax_step_fused(h, C.byref(neg), 1, None) == -1
    assert L.soax_step_fused(h, C.byref(fl), -1, None) == -1
    assert b"nsteps" in L.soax_last_error()
    assert L.soax_step_fused(None, C.byref(fl), 1, None) == -1
    # soax_copy_plane validates before any copy: field, component, direction, host
    # pointer, and that the plane is bound.
    buf = (C.c_double * 100)()
    assert L.soax_copy_plane(h, 5, 0, buf, 1, None) == -1          # bad field
    assert L.soax_copy_plane(h, 1, 3, buf, 1, None) == -1          # bad component
    assert L.soax_copy_plane(h, 1, 0, buf, 2, None) == -1          # bad direction
    assert L.soax_copy_plane(h, 1, 0, None, 0, None) == -1         # NULL host
    assert L.soax_copy_plane(h, 1, 0, buf, 1, None) == -1          # plane not bound
    assert b"not bound" in L.soax_last_error()
    assert L.soax_copy_plane(None, 1, 0, buf, 1, None) == -1
    L.soax_destroy(h)


def test_empty_handle_is_a_no_op():
    L = sx.lib()
    rc, h = _create(sx.BASIC_SCHEMA, 0)
    fl = _abi.soax_flow(1, 1, 1, 0.1, 1e-3, 0.0, -1, 1, 2, -1)
    assert L.soax_step(h, C.byref(fl), 3, None) == 0
    # The keyed fused step and the keyed sort check the grid before anything else.
    assert L.soax_step_fused_keys(h, C.byref(fl), 1, 0, None, None) == -1
    assert L.soax_step_fused_keys(h, C.byref(fl), 1, 2000, None, None) == -1
    assert L.soax_step_fused_keys(h, C.byref(fl), 1, 32, None, None) == 0
    assert L.soax_sort_by_keys(h, 0, None, None, 0, None) == -1
    assert L.soax_sort_by_keys(h, 32, None, None, 0, None) == 0
    assert L.soax_sort_perm(h, 0, None, None, 0, None) == -1
    assert L.soax_sort_perm(h, 32, None, None, 0, None) == 0
    cur = C.c_int32()
    assert L.soax_permute_step_fused(h, None, C.byref(fl), 1, 2000, None, None) == -1
    assert L.soax_permute_step_fused(h, None, C.byref(fl), -1, 0, None, None) == -1
    assert L.soax_current(h, C.byref(cur)) == 0 and cur.value == 0
    assert L.soax_permute_step_fused(h, None, C.byref(fl), 1, 0, None, None) == 0  # n = 0: flips only
    assert L.soax_current(h, C.byref(cur)) == 0 and cur.value == 1
    assert L.soax_step_fused(h, C.byref(fl), 3, None) == 0
    assert L.soax_soa_to_aos(h, None, None) == 0
    L.soax_destroy(h)


def test_step_host_validation_without_gpu():
    # soax_step_host checks everything on the host before any event, copy or launch.
    L = sx.lib()
    fl = _abi.soax_flow(1, 1, 1, 0.1, 1e-3, 0.0, -1, 1, 2, -1)
    bad = _abi.soax_flow(1, 1, 1, 0.1, 1e-3, 0.0, -1, 2, 1, -1)  # pos/vel swapped
    rc, h0 = _create(sx.BASIC_SCHEMA, 100)
    assert L.soax_step_host(h0, (C.c_void_p * 7)(*([0x1000] * 7)), C.byref(fl), 10, 32, 0, 0, C.c_void_p(0x10000),
                            1 << 30, None, None, None) == -8    # planes not bound
    L.soax_destroy(h0)
    rc, h = _create(sx.BASIC_SCHEMA, 100)
    for f, nc in enumerate((1, 3, 3)):                            # fake device addresses, never touched
        for c in range(nc):
            for b in (0, 1):
                assert L.soax_bind(h, f, c, b, C.c_void_p(0x100000 * (1 + 8 * f + 2 * c + b))) == 0
    host = (C.c_void_p * 7)(*([0x1000] * 7))
    ws = C.c_void_p(0x10000)
    args = lambda **k: dict(dict(host=host, fl=C.byref(fl), nsteps=10, grid=32, nchunks=0, defer=0, ws=ws,
                                 wsb=1 << 30), **k)

    def call(**k):
        a = args(**k)
        return L.soax_step_host(h, a["host"], a["fl"], a["nsteps"], a["grid"], a["nchunks"], a.get("defer", 0),
                                a["ws"], a["wsb"], None, None, None)
    assert call(nsteps=-1) == -1
    assert call(grid=0) == -1 and call(grid=1025) == -1
    assert call(nchunks=-1) == -1 and call(nchunks=1025) == -1
    assert b"nchunks" in L.soax_last_error()
    assert call(defer=2) == -1 and b"defer" in L.soax_last_error()
    assert call(fl=C.byref(bad)) == -2
    assert call(host=None) == -1
    holes = (C.c_void_p * 7)(*([0x1000] * 6 + [0]))
    assert call(host=holes) == -1 and b"host plane 6" in L.soax_last_error()
    assert call(wsb=16) == -6
    assert call(ws=C.c_void_p(0x10008)) == -3
    assert L.soax_step_host(None, host, C.byref(fl), 1, 32, 0, 0, ws, 1 << 30, None, None, None) == -1
    assert L.soax_step_host_finish(None, None) == -1
    assert L.soax_step_host_finish(h, None) == 0                 # nothing deferred: no work
    L.soax_destroy(h)
    # An empty set moves nothing: the live set flips, as after soax_permute.
    rc, h = _create(sx.BASIC_SCHEMA, 0)
    cur = C.c_int32()
    assert L.soax_step_host(h, None, C.byref(fl), 10, 32, 0, 1, None, 0, None, None, None) == 0
    assert L.soax_current(h, C.byref(cur)) == 0 and cur.value == 1
    L.soax_destroy(h)


def test_workspace_sizes():
    L = sx.lib()
    assert L.soax_batched_forget(None) == 0  # unknown workspace: no effect
    b = C.c_size_t()
    assert L.soax_radix_workspace_bytes(1 << 24, 15, C.byref(b)) == 0
    # 2 passes: counts (512 x 4096 x 4) + totals + one ping-pong pair of n u32.
    assert b.value >= 2 * 4 * (1 << 24)
    assert L.soax_radix_workspace_bytes(10, 0, C.byref(b)) == -1
    rc, h = _create(sx.BASIC_SCHEMA, 1000)
    assert L.soax_sort_workspace_bytes(h, 32, C.byref(b)) == 0 and b.value > 3 * 4000
    assert L.soax_adjoint_workspace_bytes(h, 1000, 32, C.byref(b)) == 0
    assert b.value >= (32 + 32) * 36 * 1000
    L.soax_destroy(h)


def test_expr_validation_without_gpu():
    """soax_expr checks its program on the host before any launch (an empty set still
    validates it)."""
    L = sx.lib()
    rc, h = _create(sx.WIDE_SCHEMA, 0)
    assert rc == 0

    def run(ops, dst=(1, 0), compute=4):
        arr = (_abi.soax_expr_op * max(1, len(ops)))()
        for j, (op, f, c, v) in enumerate(ops):
            arr[j].op, arr[j].field, arr[j].comp, arr[j].value = op, f, c, v
        return L.soax_expr(h, dst[0], dst[1], arr, len(ops), compute, None)
    load_pos, const, add, fma = (0, 1, 0, 0.0), (1, 0, 0, 2.0), (2, 0, 0, 0.0), (11, 0, 0, 0.0)
    assert run([load_pos, const, add]) == 0
    assert run([load_pos, add]) == -1                   # underflow
    assert run([load_pos, const]) == -1                 # two values left
    assert run([load_pos, const, fma]) == -1            # fma needs three
    assert run([(99, 0, 0, 0.0)]) == -1                 # unknown operation
    assert run([load_pos], compute=0) == -1             # compute type
    assert run([load_pos], dst=(5, 0)) == -2            # u8 destination
    assert run([(0, 1, 3, 0.0)]) == -1                  # bad component
    assert run([const] * 17 + [add] * 16) == -1         # deeper than 16
    assert run([const] * 65) == -1                      # more than 64 operations
    L.soax_destroy(h)
