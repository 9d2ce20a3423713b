"""soax_sort_by_cell_noalloc, the cell sort for hosts that cannot allocate device memory
(C or Fortran codes without a device allocator of their own, or time-step loops that
forbid cudaMalloc because it can synchronise the device and breaks a fixed memory
budget).  Called through the C ABI, it must leave every plane and the permutation
bit-identical to soax_sort_by_cell with a caller workspace, on two calls in a row (the
second one reuses the static scratch that the first call left filled), and must reject
sizes beyond its static limit.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_1710_03462_b300 as sx
import soax_inputs

pytestmark = pytest.mark.gpu


def _planes(p):
    return [t.cpu().numpy().tobytes() for name, _, _, _ in p.schema for t in p.field(name)]


def test_noalloc_sort_matches_workspace_sort_twice():
    L = sx.lib()
    n, grid = 300007, 32
    d = soax_inputs.basic_set(n, 11)
    ref = sx.Particles(sx.BASIC_SCHEMA, n)
    got = sx.Particles(sx.BASIC_SCHEMA, n)
    ref.load(d)
    got.load(d)
    ws = ref.sort_workspace(grid)
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        assert L.soax_sort_by_cell(ref.h, grid, C.c_void_p(ws.data_ptr()), ws.numel(), stream) == 0
        rc = L.soax_sort_by_cell_noalloc(got.h, grid, C.c_void_p(perm.data_ptr()), stream)
        assert rc == 0, L.soax_last_error()
        assert L.soax_sync(stream) == 0
        assert got.current == ref.current
        _, ref_perm = ref.sort_results(grid, ws)
        assert torch.equal(perm, ref_perm), f"call {call}: permutation differs"
        assert _planes(got) == _planes(ref), f"call {call}: planes differ"
        # Move the particles so that the second call sorts a different order.
        ref.step(sx.Flow(), 3)
        got.step(sx.Flow(), 3)


def test_noalloc_sort_wide_record_grid64():
    L = sx.lib()
    n = 1 << 20  # the largest size the static scratch takes
    d = soax_inputs.wide_set(n, 12)
    ref = sx.Particles(sx.WIDE_SCHEMA, n)
    got = sx.Particles(sx.WIDE_SCHEMA, n)
    ref.load(d)
    got.load(d)
    ref.sort_by_cell(64)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.soax_sort_by_cell_noalloc(got.h, 64, None, stream) == 0, L.soax_last_error()
    assert L.soax_sync(stream) == 0
    assert _planes(got) == _planes(ref)


def test_noalloc_sort_rejects_sizes_beyond_the_limit():
    L = sx.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    big = sx.Particles(sx.BASIC_SCHEMA, (1 << 20) + 1, shadow=False)
    assert L.soax_sort_by_cell_noalloc(big.h, 32, None, stream) == -1
    assert b"1048576" in L.soax_last_error()
    small = sx.Particles(sx.BASIC_SCHEMA, 1000)
    assert L.soax_sort_by_cell_noalloc(small.h, 65, None, stream) == -1
    assert b"grid" in L.soax_last_error()
