"""soax_copy_plane: the live planes to and from host memory, byte for byte, for every
field type, asynchronously from pinned memory on a stream, and following the live buffer
set after a sort flips it."""
import numpy as np
import pytest
import torch

import paper_1710_03462_b300 as sx
import soax_inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("schema,maker", [(sx.BASIC_SCHEMA, soax_inputs.basic_set),
                                          (sx.WIDE_SCHEMA, soax_inputs.wide_set)])
@pytest.mark.parametrize("n", [1, 1000, 65537])
def test_round_trip_every_plane(schema, maker, n):
    d = maker(n, 3)
    p = sx.Particles(schema, n)
    s = torch.cuda.Stream()
    host = {k: [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in v] for k, v in d.items()}
    for k, v in host.items():
        for c, t in enumerate(v):
            p.copy_plane(k, c, t, True, stream=s)
    s.synchronize()
    g = p.numpy()
    for k, v in d.items():
        for c, a in enumerate(v):
            assert g[k][c].tobytes() == np.ascontiguousarray(a).tobytes(), (k, c)
    back = {k: [torch.empty_like(t).pin_memory() for t in v] for k, v in host.items()}
    for k, v in back.items():
        for c, t in enumerate(v):
            p.copy_plane(k, c, t, False, stream=s)
    s.synchronize()
    for k, v in d.items():
        for c, a in enumerate(v):
            assert back[k][c].numpy().tobytes() == np.ascontiguousarray(a).tobytes(), (k, c)


def test_copies_follow_the_live_set():
    n = 5000
    d = soax_inputs.basic_set(n, 9)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    p.load(d)
    _, perm = p.sort_by_cell(32)
    assert p.current == 1
    perm = perm.cpu().numpy().view(np.uint32)
    out = np.empty(n, np.float64)
    p.copy_plane("pos", 2, out, False)          # pageable memory: returns after the copy
    assert np.array_equal(out, d["pos"][2][perm])
    new = np.arange(n, dtype=np.int32)
    p.copy_plane("id", 0, new, True)
    torch.cuda.synchronize()
    assert np.array_equal(p.field("id")[0].cpu().numpy(), new)
    assert np.array_equal(p.field("id", buf=0)[0].cpu().numpy(), d["id"][0])  # the other set is untouched


def test_rejects_bad_host_buffers():
    p = sx.Particles(sx.BASIC_SCHEMA, 100)
    with pytest.raises(ValueError):
        p.copy_plane("pos", 0, np.empty(100, np.float32), True)     # wrong element size
    with pytest.raises(ValueError):
        p.copy_plane("pos", 0, np.empty(50, np.float64), True)      # too short
    with pytest.raises(ValueError):
        p.copy_plane("pos", 0, torch.empty(100, dtype=torch.float64, device="cuda"), True)  # not host memory
