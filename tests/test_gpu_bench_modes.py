"""The profiling entry points of bench.py (--only euler|aos|fixed|adjoint|batched), the
commands profiles/ cites, run at tiny sizes and print one JSON line with their rows."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("argv,keys", [
    (["--only", "euler", "--n", "65536"], ["soa_fused_GB/s", "aos32_over_soa_per_component"]),
    (["--only", "aos", "--n", "65536"], ["aos_soa_roundtrip", "aos_step"]),
    (["--only", "fixed", "--n", "65536"], ["gather+keys", "fused+keys", "fused"]),
    (["--only", "adjoint", "--n", "4096"], ["fwd_ms", "adj_ms", "roofline"]),
    (["--only", "batched", "--nens", "3", "--fixed-tune"], ["persistent", "fused", "plain_launches"]),
])
def test_only_modes(argv, keys, capsys):
    assert bench.main(argv) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["only"] == argv[1]
    for k in keys:
        assert k in line["row"], k
    if argv[1] == "fixed":
        r = line["row"]["gather+keys"]
        assert r["ms_per_step"] > 0 and set(r["ms_per_launch"]) == {"10", "20"}
