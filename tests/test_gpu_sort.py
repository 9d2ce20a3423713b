"""GPU cell keys, radix sort, permute and sort_by_cell: bit-exact against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_1710_03462_b300 as sx
import soax_inputs

pytestmark = pytest.mark.gpu


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("G", [1, 7, 32, 64])
def test_cell_keys_bit_exact(G):
    n = 100003
    d = soax_inputs.basic_set(n, G)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    p.load(d)
    k = _u32(p.cell_keys(G))
    assert np.array_equal(k, oracle.cell_keys(*d["pos"], G))


def test_cell_keys_boundaries():
    G = 64
    below = np.nextafter(sx.TWO_PI, 0.0)
    pos = [np.array([0.0, below, 0.0, 0.0, 1e-300]), np.array([0.0, 0.0, below, 0.0, 3.0]),
           np.array([0.0, 0.0, 0.0, below, 6.0])]
    p = sx.Particles([("pos", "f64", 3, "P")], 5)
    p.load({"pos": pos})
    assert np.array_equal(_u32(p.cell_keys(G)), oracle.cell_keys(*pos, G))


@pytest.mark.parametrize("n,bits", [(1, 15), (5, 3), (4095, 9), (4097, 10), (100000, 15), (250001, 18),
                                    (70000, 32), (33, 1)])
def test_radix_sort_pairs_vs_oracle(n, bits):
    rng = np.random.default_rng(n + bits)
    keys = rng.integers(0, 2 ** bits, n, dtype=np.uint64).astype(np.uint32)
    kt = torch.from_numpy(keys.view(np.int32)).cuda()
    ko, vo = sx.radix_sort_pairs(kt, key_bits=bits)
    perm, sk = oracle.stable_argsort(keys)
    assert np.array_equal(_u32(vo), perm)
    assert np.array_equal(_u32(ko), sk)


def test_radix_sort_with_values_and_sorted_input():
    n = 300000
    keys = np.sort(np.random.default_rng(1).integers(0, 2 ** 15, n)).astype(np.uint32)  # already sorted
    vals = np.random.default_rng(2).integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    ko, vo = sx.radix_sort_pairs(torch.from_numpy(keys.view(np.int32)).cuda(), torch.from_numpy(vals.view(np.int32)).cuda(),
                                 key_bits=15)
    perm, sk = oracle.stable_argsort(keys)
    assert np.array_equal(_u32(vo), vals[perm])
    assert np.array_equal(_u32(ko), sk)


def _check_sort_by_cell(d, schema, G):
    n = d["pos"][0].size
    p = sx.Particles(schema, n)
    p.load(d)
    kt, pt = p.sort_by_cell(G)
    assert p.current == 1
    keys = oracle.cell_keys(*d["pos"], G)
    perm, sk = oracle.stable_argsort(keys)
    assert np.array_equal(_u32(pt), perm)
    assert np.array_equal(_u32(kt), sk)
    g = p.numpy()
    for name, _, nc, _ in schema:
        outs = oracle.permute(d[name], perm)
        for a, b in zip(g[name], outs):
            assert a.tobytes() == b.tobytes(), name
    return p


@pytest.mark.parametrize("n", [1, 2, 4099, 123457])
def test_sort_by_cell_basic(n):
    _check_sort_by_cell(soax_inputs.basic_set(n, 5), sx.BASIC_SCHEMA, 32)


def test_sort_by_cell_wide_grid64():
    _check_sort_by_cell(soax_inputs.wide_set(200003, 6), sx.WIDE_SCHEMA, 64)


def test_sort_twice_flips_back_and_is_stable():
    n = 50000
    d = soax_inputs.basic_set(n, 8)
    p = _check_sort_by_cell(d, sx.BASIC_SCHEMA, 32)
    p.sort_by_cell(32)
    assert p.current == 0
    ids = p.numpy()["id"][0]
    k = oracle.cell_keys(*p.numpy()["pos"], 32)
    assert np.all(np.diff(k.astype(np.int64)) >= 0)
    same = k[1:] == k[:-1]
    assert np.all(ids[1:][same] > ids[:-1][same])


def test_full_size_sorted_n16M_sort():
    w = soax_inputs.WORKLOADS["sorted_n16M"]
    d = soax_inputs.basic_set(w["n"], w["seed"])
    p = _check_sort_by_cell(d, sx.BASIC_SCHEMA, w["grid"])
    del p
    torch.cuda.empty_cache()


def test_full_size_wide_n64M_sort():
    w = soax_inputs.WORKLOADS["wide_n64M"]
    n = w["n"]
    d = soax_inputs.wide_set(n, w["seed"])
    p = sx.Particles(sx.WIDE_SCHEMA, n)
    p.load(d)
    kt, pt = p.sort_by_cell(w["grid"])
    perm = _u32(pt)
    ref, _ = oracle.stable_argsort(oracle.cell_keys(*d["pos"], w["grid"]))
    assert np.array_equal(perm, ref)
    g = p.numpy()
    pi = perm.astype(np.int64)
    for name, _, nc, _ in sx.WIDE_SCHEMA:
        for a, b in zip(g[name], d[name]):
            assert np.array_equal(a, b[pi]), name
    del p, g
    torch.cuda.empty_cache()


@pytest.mark.parametrize("G", [32, 64, 1000])
def test_cell_keys_near_every_boundary(G):
    """Positions within a few ulps of every cell boundary: the product x * (G/2pi) must
    round (then truncate) exactly as binary64 arithmetic does."""
    c = G / sx.TWO_PI
    base = np.arange(G + 1) / c
    xs = [base]
    up, dn = base.copy(), base.copy()
    for _ in range(6):
        up = np.nextafter(up, np.inf)
        dn = np.nextafter(dn, -np.inf)
        xs += [up.copy(), dn.copy()]
    x = np.concatenate(xs)
    x = x[(x >= 0) & (x < sx.TWO_PI)]
    rng = np.random.default_rng(G)
    pos = [np.ascontiguousarray(rng.permutation(x)) for _ in range(3)]
    p = sx.Particles([("pos", "f64", 3, "P")], x.size)
    p.load({"pos": pos})
    assert np.array_equal(_u32(p.cell_keys(G)), oracle.cell_keys(*pos, G))


def test_permute_reports_an_index_out_of_range():
    """A bad permutation entry is not read; the kernel records EINVAL in the device status
    word and soax_sync reports it (and clears it)."""
    n = 1000
    d = soax_inputs.basic_set(n, 9)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    p.load(d)
    perm = torch.arange(n, dtype=torch.int32, device="cuda")
    perm[517] = n + 12345
    p.permute(perm)
    with pytest.raises(sx.SoaxError) as ei:
        sx.sync()
    assert ei.value.code == -1
    sx.sync()  # cleared
    g = p.numpy()
    assert g["id"][0][517] == d["id"][0][0]
    assert np.array_equal(np.delete(g["id"][0], 517), np.delete(d["id"][0], 517))


def test_bench_step_captured_in_a_cuda_graph():
    """10 RK2 steps and a cell sort captured in one CUDA graph (no allocation or host
    synchronisation inside the calls) give the same bits as the eager calls."""
    n = 200003
    d = soax_inputs.basic_set(n, 13)
    eager = sx.Particles(sx.BASIC_SCHEMA, n)
    graph = sx.Particles(sx.BASIC_SCHEMA, n)
    eager.load(d)
    graph.load(d)
    f = sx.Flow()
    ws_e, ws_g = eager.sort_workspace(32), graph.sort_workspace(32)
    eager.sort_by_cell(32, ws_e)  # first use sets kernel attributes outside any capture
    graph.sort_by_cell(32, ws_g)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    start = graph.current
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            graph.step(f, 10, stream=s)
            graph.sort_by_cell(32, ws_g, stream=s)
            graph.step(f, 10, stream=s)
            graph.sort_by_cell(32, ws_g, stream=s)  # two flips: the live set is back to start
    torch.cuda.current_stream().wait_stream(s)
    graph.set_current(start)
    for _ in range(3):
        g.replay()
        for _ in range(2):
            eager.step(f, 10)
            eager.sort_by_cell(32, ws_e)
    torch.cuda.synchronize()
    a, b = eager.numpy(), graph.numpy()
    for k in a:
        for x, y in zip(a[k], b[k]):
            assert x.tobytes() == y.tobytes()
