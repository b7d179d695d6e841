"""Batched execution (st_batch_*): every request's result inside a mixed
batch of truncations, grids and precisions is the same as the request run
alone (within the split-precision tolerance), with and without graph replay."""
import numpy as np
import pytest
import torch

from paper_1908_06096_gb300 import inputs
from tests.conftest import per_field_max_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


REQS = [
    # T, grid, precision, nfields, direction
    (79, "regular", "bf16x3", 5, "round"),
    (63, "octahedral", "bf16x3", 17, "round"),
    (31, "regular", "fp64", 3, "inv"),
    (47, "octahedral", "tf32x3", 9, "dir"),
    (95, "octahedral", "bf16x3", 1, "round"),
    (31, "octahedral", "fp32", 4, "round"),
]


def _make(st_mod, idx, T, grid, prec, nf, direction):
    p = st_mod.Plan(T, grid, precision=prec, max_fields=nf)
    spec = torch.from_numpy(inputs.spectra(T, nf, seed=500 + idx)).to("cuda", p.dtype)
    g = torch.zeros((nf, p.npts), dtype=p.dtype, device="cuda")
    if direction == "dir":
        g = p.inv(spec).clone()
    out = torch.zeros((nf, p.nspec, 2), dtype=p.dtype, device="cuda")
    return p, spec, g, out


@pytest.mark.parametrize("graph", [False, True])
def test_batch_matches_individual_calls(st_mod, graph):
    setups = [_make(st_mod, i, *r) for i, r in enumerate(REQS)]
    refs = []
    for (p, spec, g, out), r in zip(setups, REQS):
        d = r[4]
        if d == "inv":
            refs.append((p.inv(spec).clone(), None))
        elif d == "dir":
            refs.append((None, p.dir(g).clone()))
        else:
            gg = p.inv(spec).clone()
            refs.append((gg, p.dir(gg).clone()))
    torch.cuda.synchronize()
    items = [(p, r[4], spec if r[4] != "dir" else None, g, out if r[4] != "inv" else None)
             for (p, spec, g, out), r in zip(setups, REQS)]
    batch = st_mod.Batch(items)
    for _ in range(2):                      # a second run replays the graph
        for (p, spec, g, out), r in zip(setups, REQS):
            if r[4] != "dir":
                g.zero_()
            out.zero_()
        batch.run(graph=graph)
        torch.cuda.synchronize()
        for (p, spec, g, out), r, (gref, sref) in zip(setups, REQS, refs):
            tol = 1e-12 if r[2] == "fp64" else 2e-5
            if gref is not None:
                assert per_field_max_rel(g.double().cpu().numpy(), gref.double().cpu().numpy()) <= tol, r
            if sref is not None:
                assert per_field_max_rel(out.double().cpu().numpy(), sref.double().cpu().numpy()) <= tol, r
    batch.close()
    for p, *_ in setups:
        p.sync()
        p.close()


def test_batch_rejects_duplicate_plan(st_mod):
    p = st_mod.Plan(31, "regular", precision="bf16x3", max_fields=2)
    spec = torch.zeros((2, p.nspec, 2), device="cuda")
    g = torch.zeros((2, p.npts), device="cuda")
    with pytest.raises(st_mod.STError):
        st_mod.Batch([(p, "inv", spec, g, None), (p, "inv", spec, g, None)])
    p.close()
