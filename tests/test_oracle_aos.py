"""Pins of the oracle's AoS layout and transposes: the paper's own structs
(tests/golden/aos_layouts.txt), numpy's and ctypes' independent computation of C struct
layouts, byte equality with a numpy structured array (zero padding), and the round
trip."""
import ctypes
import os

import numpy as np
import pytest

import oracle
import soax_inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "aos_layouts.txt")
SIZES = {"i32": 4, "i64": 8, "u8": 1, "f32": 4, "f64": 8}
NP = {"i32": "<i4", "i64": "<i8", "u8": "u1", "f32": "<f4", "f64": "<f8"}
CT = {"i32": ctypes.c_int32, "i64": ctypes.c_int64, "u8": ctypes.c_uint8, "f32": ctypes.c_float,
      "f64": ctypes.c_double}


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, fields, rb, offs, cite = [x.strip() for x in line.split("|")]
        fl = [(f.split(":")[0], int(f.split(":")[1])) for f in fields.split()]
        rows.append((name, fl, int(rb), [int(o) for o in offs.split()], cite))
    return rows


@pytest.mark.parametrize("row", _golden(), ids=lambda r: r[0])
def test_paper_layouts(row):
    name, fl, rb, offs, _ = row
    got_rb, got_offs = oracle.aos_layout([SIZES[t] for t, _ in fl], [n for _, n in fl])
    assert (got_rb, got_offs) == (rb, offs)


SCHEMAS = [
    [("i32", 1), ("f64", 3), ("f32", 3)],
    [("i64", 1), ("f64", 3), ("f32", 3), ("f32", 3), ("f32", 1), ("u8", 1)],
    [("u8", 1), ("f64", 1), ("u8", 3), ("i32", 2)],
    [("f32", 3), ("u8", 1)],
]


@pytest.mark.parametrize("schema", SCHEMAS)
def test_layout_matches_numpy_and_ctypes(schema):
    rb, offs = oracle.aos_layout([SIZES[t] for t, _ in schema], [n for _, n in schema])
    dt = np.dtype([(f"f{k}", NP[t], (n,)) for k, (t, n) in enumerate(schema)], align=True)
    assert dt.itemsize == rb
    assert [dt.fields[f"f{k}"][1] for k in range(len(schema))] == offs

    class S(ctypes.Structure):
        _fields_ = [(f"f{k}", CT[t] * n) for k, (t, n) in enumerate(schema)]
    assert ctypes.sizeof(S) == rb
    assert [getattr(S, f"f{k}").offset for k in range(len(schema))] == offs


def _planes_for(schema, n, rng):
    planes = []
    for t, nc in schema:
        for _ in range(nc):
            if t == "u8":
                planes.append(rng.integers(0, 256, n, dtype=np.uint8))
            elif t in ("i32", "i64"):
                planes.append(rng.integers(-2**31, 2**31 - 1, n).astype(NP[t]))
            else:
                planes.append(rng.standard_normal(n).astype(NP[t]))
    return planes


@pytest.mark.parametrize("schema", SCHEMAS)
def test_soa_to_aos_matches_numpy_struct_bytes(schema):
    rng = np.random.default_rng(1)
    n = 777
    planes = _planes_for(schema, n, rng)
    rec = oracle.soa_to_aos(planes, [SIZES[t] for t, _ in schema], [n_ for _, n_ in schema])
    dt = np.dtype([(f"f{k}", NP[t], (nc,)) for k, (t, nc) in enumerate(schema)], align=True)
    ref = np.zeros(n, dt)  # padding bytes stay zero
    p = 0
    for k, (t, nc) in enumerate(schema):
        for c in range(nc):
            ref[f"f{k}"][:, c] = planes[p]
            p += 1
    assert rec.tobytes() == ref.tobytes()


@pytest.mark.parametrize("schema", SCHEMAS)
def test_round_trip_identity(schema):
    rng = np.random.default_rng(2)
    n = 1001
    planes = _planes_for(schema, n, rng)
    eb, nc = [SIZES[t] for t, _ in schema], [x for _, x in schema]
    rec = oracle.soa_to_aos(planes, eb, nc)
    back = oracle.aos_to_soa(rec, eb, nc, [NP[t] for t, _ in schema])
    assert all(a.tobytes() == b.tobytes() for a, b in zip(planes, back))
    rec2 = oracle.soa_to_aos(back, eb, nc)
    assert rec.tobytes() == rec2.tobytes()


def test_basic_set_record():
    d = soax_inputs.basic_set(10)
    rec = oracle.soa_to_aos(d["id"] + d["pos"] + d["vel"], [4, 8, 4], [1, 3, 3])
    r = rec.reshape(10, 48)
    assert np.all(r[:, 4:8] == 0) and np.all(r[:, 44:48] == 0)
    assert np.array_equal(r[:, 8:16].copy().view("<f8")[:, 0], d["pos"][0])
