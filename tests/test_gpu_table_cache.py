"""On-disk table cache: a plan's tables written to a file and read back give
bit-identical transforms; plan creation with ST_TABLE_CACHE builds the tables
once, later creations load them; a file of another plan, or a damaged one, is
refused and leaves the plan's tables as they were."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_1908_06096_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _round_trip(p, a):
    g = p.inv(a)
    s = p.dir(g)
    torch.cuda.synchronize()
    return g.cpu().numpy(), s.cpu().numpy()


def test_save_load_round_trip_is_bitwise(st_mod, tmp_path):
    T = 47
    path = str(tmp_path / "t47.bin")
    a = torch.from_numpy(inputs.spectra(T, 3, seed=61)).to("cuda", torch.float32)
    p = st_mod.Plan(T, "octahedral", precision="bf16x3", max_fields=3)
    ref = _round_trip(p, a)
    p.save_tables(path)
    q = st_mod.Plan(T, "octahedral", precision="bf16x3", max_fields=3)
    q.load_tables(path)
    got = _round_trip(q, a)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    # another plan's file is refused; a damaged file too
    r = st_mod.Plan(T, "regular", precision="bf16x3", max_fields=3)
    with pytest.raises(st_mod.STError):
        r.load_tables(path)
    with open(path, "r+b") as fh:
        fh.seek(-5, os.SEEK_END)
        b = fh.read(1)
        fh.seek(-5, os.SEEK_END)
        fh.write(bytes([b[0] ^ 0x40]))
    with pytest.raises(st_mod.STError):
        q.load_tables(path)
    assert np.array_equal(_round_trip(q, a)[0], ref[0])  # untouched by the refused load
    for x in (p, q, r):
        x.close()


CHILD = r"""
import sys, json
sys.path.insert(0, sys.argv[1])
from paper_1908_06096_gb300 import st
st.ensure_built()
p = st.Plan(63, "octahedral", precision="tf32x3", max_fields=2)
print(json.dumps({"tables": p.timings().get("plan_tables", {"launches": 0})["launches"]}))
"""


def test_env_cache_builds_once(st_mod, tmp_path):
    """Two processes create the same plan with ST_TABLE_CACHE set: the first
    builds the tables (one table launch) and writes the file, the second
    loads it (no table launch)."""
    import json
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, ST_TABLE_CACHE=str(tmp_path))
    runs = []
    for _ in range(2):
        out = subprocess.run([sys.executable, "-c", CHILD, root], env=env, capture_output=True, text=True,
                             timeout=300)
        assert out.returncode == 0, out.stderr[-2000:]
        runs.append(json.loads(out.stdout.strip().splitlines()[-1])["tables"])
    assert runs == [1, 0]
    assert any(f.startswith("st_tables_T63_") for f in os.listdir(tmp_path))
