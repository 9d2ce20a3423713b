"""The cell counting sort (grids up to 64^3: counts, bucket scan, scatter of equal-key
groups, per-key order of the groups by segment) and its fallback to the radix passes
(the body of the sort graph's conditional node, or gated on a stream being captured),
bit-exact against the oracle's stable argsort: near-sorted keys (the bench's case: a
sorted set stepped again), random keys, keys at the per-key capacity (2048 particles,
256 groups), keys beyond it (one key holding most particles: the radix passes sort),
tiny and ragged sizes, the sorted keys written beside the permutation, one graph serving
many key sets, more buffer sets than the graph cache, and the sort inside a caller's
captured graph."""
import numpy as np
import pytest
import torch

import oracle
import paper_1710_03462_b300 as sx
import soax_inputs

pytestmark = pytest.mark.gpu


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _sort_keys(keys, grid, with_keys=True):
    """sort_by_keys / sort_perm of the given u32 keys on a set of that size."""
    n = keys.size
    p = sx.Particles([("pos", "f64", 3, "P")], n)
    kt = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    if with_keys:
        sk, perm = p.sort_by_keys(grid, kt)
        out = _u32(sk), _u32(perm)
    else:
        _, perm = p.sort_perm(grid, kt)
        out = None, _u32(perm)
    sx.sync()
    return out


def _check(keys, grid, with_keys=True):
    sk, perm = _sort_keys(keys, grid, with_keys)
    ref, rsk = oracle.stable_argsort(keys)
    assert np.array_equal(perm, ref)
    if with_keys:
        assert np.array_equal(sk, rsk)


@pytest.mark.parametrize("n,grid", [(1, 32), (2, 1), (31, 7), (33, 32), (4097, 64), (100003, 32), (250001, 64)])
def test_random_keys(n, grid):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, grid ** 3, n, dtype=np.uint32)
    _check(keys, grid)
    _check(keys, grid, with_keys=False)


def test_near_sorted_keys_after_steps():
    """The bench's case: a set sorted by cell, stepped 10 times, keyed again in its
    sorted order (most keys in runs, a tenth of them moved to neighbouring cells)."""
    n, grid = 1 << 20, 32
    d = soax_inputs.basic_set(n, 3)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    p.load(d)
    p.sort_by_cell(grid)
    keys = p.step_fused(sx.Flow(), 10, grid=grid)
    k = _u32(keys).copy()
    moved = np.count_nonzero(np.diff(k.astype(np.int64)) != 0)
    assert moved > n // 100  # not trivially sorted
    ws = p.sort_workspace(grid)
    _, perm = p.sort_perm(grid, keys, ws)
    sx.sync()
    ref, _ = oracle.stable_argsort(k)
    assert np.array_equal(_u32(perm), ref)


def test_capacity_edges():
    """A key with exactly 2048 particles in 64 groups (the counting path), a key with 2049
    (the radix passes), and a key with 257 groups of one particle (the radix passes)."""
    grid = 16
    base = np.repeat(np.arange(grid ** 3, dtype=np.uint32), 3)
    k1 = np.sort(np.concatenate([base, np.full(2048 - 3, 77, np.uint32)]), kind="stable")
    _check(k1, grid)
    k2 = np.sort(np.concatenate([base, np.full(2049 - 3, 77, np.uint32)]), kind="stable")
    _check(k2, grid)
    # 257 groups of key 5: one per 32-key segment, the rest of each segment other keys.
    k3 = np.arange(grid ** 3, dtype=np.uint32) % 4000 + 10
    k3 = np.resize(k3, 257 * 32).copy()
    k3[::32] = 5
    _check(k3, grid)


def test_one_cell_holds_most_particles():
    """Clustered input beyond the per-key capacity: the gate hands the sort to the radix
    passes, which give the same permutation."""
    rng = np.random.default_rng(9)
    n, grid = 300001, 32
    keys = rng.integers(0, grid ** 3, n, dtype=np.uint32)
    keys[rng.random(n) < 0.5] = 12345
    _check(keys, grid)


def test_grid_beyond_the_counting_sort():
    """Grids above 64^3 (more than 18 key bits) sort with the radix passes alone."""
    rng = np.random.default_rng(4)
    keys = rng.integers(0, 100 ** 3, 70001, dtype=np.uint32)
    _check(keys, 100)


def test_unordered_then_near_sorted_sets():
    """A set in no particular order (the probe hands it to the radix passes) and then the
    same set sorted and stepped (the counting sort): both give the oracle's permutation."""
    n, grid = 400003, 32
    d = soax_inputs.basic_set(n, 12)
    p = sx.Particles(sx.BASIC_SCHEMA, n)
    p.load(d)
    ws = p.sort_workspace(grid)
    keys = p.cell_keys(grid)
    _, perm = p.sort_perm(grid, keys, ws)
    sx.sync()
    assert np.array_equal(_u32(perm), oracle.stable_argsort(_u32(keys).copy())[0])
    p.sort_by_cell(grid, ws)
    keys = p.step_fused(sx.Flow(), 10, grid=grid)
    _, perm = p.sort_perm(grid, keys, ws)
    sx.sync()
    assert np.array_equal(_u32(perm), oracle.stable_argsort(_u32(keys).copy())[0])


def test_graph_reused_across_key_sets_in_the_same_buffers():
    """One graph serves every call with the same pointers and sizes: the same key buffer
    filled with near-sorted keys, keys beyond the per-key capacity (the conditional body
    runs the radix passes) and near-sorted keys again.  Exactly one graph is built for
    the five calls, and no build fails."""
    n, grid = 200003, 32
    rng = np.random.default_rng(17)
    p = sx.Particles([("pos", "f64", 3, "P")], n)
    ws = p.sort_workspace(grid)
    kt = torch.empty(n, dtype=torch.int32, device="cuda")
    base = np.sort(rng.integers(0, grid ** 3, n, dtype=np.uint32))
    crowded = base.copy()
    crowded[rng.random(n) < 0.3] = 777
    built0, failed0 = sx.sort_graph_counts()
    for keys in (base, crowded, np.roll(base, 5000), crowded[::-1].copy(), base):
        kt.copy_(torch.from_numpy(keys.view(np.int32)))
        _, perm = p.sort_perm(grid, kt, ws)
        sx.sync()
        assert np.array_equal(_u32(perm), oracle.stable_argsort(keys)[0])
    built1, failed1 = sx.sort_graph_counts()
    assert (built1 - built0, failed1 - failed0) == (1, 0)


def test_more_pointer_sets_than_the_graph_cache():
    """Ten workspaces used in turn, twice (more than the graphs kept): each call still
    gives the oracle's permutation."""
    n, grid = 50001, 16
    rng = np.random.default_rng(18)
    p = sx.Particles([("pos", "f64", 3, "P")], n)
    wss = [p.sort_workspace(grid) for _ in range(10)]
    kt = torch.empty(n, dtype=torch.int32, device="cuda")
    for rep in range(2):
        for j, ws in enumerate(wss):
            keys = np.sort(rng.integers(0, grid ** 3, n, dtype=np.uint32))
            if (j + rep) % 3 == 0:
                keys = rng.permutation(keys)  # in no particular order: the radix passes
            kt.copy_(torch.from_numpy(keys.view(np.int32)))
            _, perm = p.sort_perm(grid, kt, ws)
            sx.sync()
            assert np.array_equal(_u32(perm), oracle.stable_argsort(keys)[0]), (rep, j)


def test_sort_inside_a_captured_graph():
    """A caller capturing its own CUDA graph gets the sort's kernels on its stream (the
    radix passes gated): replays of the captured sort give the oracle's permutation for
    the keys in the buffer at replay time."""
    n, grid = 100003, 32
    rng = np.random.default_rng(19)
    p = sx.Particles([("pos", "f64", 3, "P")], n)
    ws = p.sort_workspace(grid)
    kt = torch.empty(n, dtype=torch.int32, device="cuda")
    kt.copy_(torch.from_numpy(np.sort(rng.integers(0, grid ** 3, n, dtype=np.uint32)).view(np.int32)))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        p.sort_perm(grid, kt, ws, stream=s)  # warm-up outside the capture (builds the sort's graph)
    s.synchronize()
    counts = sx.sort_graph_counts()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        _, perm = p.sort_perm(grid, kt, ws, stream=s)
    assert sx.sort_graph_counts() == counts  # inside the capture: no graph built
    for keys in (np.sort(rng.integers(0, grid ** 3, n, dtype=np.uint32)),
                 rng.integers(0, grid ** 3, n, dtype=np.uint32)):
        kt.copy_(torch.from_numpy(keys.view(np.int32)))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(_u32(perm), oracle.stable_argsort(keys)[0])


def test_two_threads_sharing_the_graph_cache():
    """Two host threads sort on their own streams with six workspaces each (twelve
    buffer sets against a cache of eight: graphs are evicted while the other thread
    launches its own); every permutation is the oracle's."""
    import threading

    n, grid = 40009, 16
    errors = []

    def worker(seed):
        try:
            rng = np.random.default_rng(seed)
            s = torch.cuda.Stream()
            p = sx.Particles([("pos", "f64", 3, "P")], n)
            wss = [p.sort_workspace(grid) for _ in range(6)]
            kt = torch.empty(n, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            for rep in range(3):
                for j, ws in enumerate(wss):
                    keys = np.sort(rng.integers(0, grid ** 3, n, dtype=np.uint32))
                    if (j + rep) % 4 == 0:
                        keys = rng.permutation(keys)
                    with torch.cuda.stream(s):
                        kt.copy_(torch.from_numpy(keys.view(np.int32)))
                        _, perm = p.sort_perm(grid, kt, ws, stream=s)
                        got = perm.cpu()  # on s: after the sort
                    s.synchronize()
                    if not np.array_equal(got.numpy().view(np.uint32), oracle.stable_argsort(keys)[0]):
                        errors.append((seed, rep, j))
        except Exception as e:  # reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(s,)) for s in (31, 32)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    sx.sync()
