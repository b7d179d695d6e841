"""Batched execution (st_batch_*).

Every request of a mixed batch of truncations, grids and precisions is
compared with the FP64 oracle (the synthesis and analysis definitions), with
and without graph replay, and with the same request run alone.  A second case
runs requests of the mixed-truncation configuration's sizes (T639 on O640
with 220 fields in BF16x3, T511 on the regular 512 x 1024 grid with 200
fields in 3xTF32) in one batch, sampled fields against the oracle.

Bars: 1e-12 (FP64), 2e-5 (FP32, 3xTF32, BF16x3) normwise per field.
"""
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


def _tol(prec):
    return 1e-12 if prec == "fp64" else 2e-5


def _make(st_mod, idx, T, grid, prec, nf, direction):
    p = st_mod.Plan(T, grid, precision=prec, max_fields=nf)
    spec = torch.from_numpy(inputs.spectra(T, nf, seed=500 + idx)).to("cuda", p.dtype)
    g = torch.zeros((nf, p.npts), dtype=p.dtype, device="cuda")
    if direction == "dir":
        g = p.inv(spec).clone()
    out = torch.zeros((nf, p.nspec, 2), dtype=p.dtype, device="cuda")
    return p, spec, g, out


class _Oracle:
    """Oracle results of one plan's geometry (nodes, rows) on host arrays."""

    def __init__(self, oracle_mod, plan):
        self.o = oracle_mod
        self.T = plan.T
        self.rows = oracle_mod.grid_rows(plan.grid, plan.nlat, plan.nlon)
        self.mu, self.w = oracle_mod.gauss(plan.nlat)

    def inv(self, spec):
        return self.o.inv_trans(self.T, self.rows, self.mu, spec)

    def dir(self, grid):
        return self.o.dir_trans(self.T, self.rows, self.mu, self.w, grid)


def _cplx(s):
    s = np.asarray(s, dtype=np.float64)
    return s[..., 0] + 1j * s[..., 1]


def _check_vs_oracle(orc, prec, spec, grid_in, grid_out, spec_out, direction, pick=None):
    """Compare a request's outputs (host arrays) with the oracle on fields `pick`."""
    pick = list(range(len(spec))) if pick is None else list(pick)
    tol = _tol(prec)
    if direction in ("inv", "round"):
        ref = orc.inv(spec[pick])
        err = per_field_max_rel(grid_out[pick], ref)
        assert err < tol, ("inverse", err)
    if direction in ("dir", "round"):
        src = grid_out if direction == "round" else grid_in
        ref = orc.dir(src[pick])
        err = per_field_max_rel(_cplx(spec_out[pick]), ref)
        assert err < tol, ("direct", err)


@pytest.mark.parametrize("graph", [False, True])
def test_batch_matches_oracle_and_individual_calls(st_mod, oracle_mod, graph):
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
            prec, d = r[2], r[4]
            gh = g.double().cpu().numpy()
            sh = out.double().cpu().numpy()
            # against the oracle
            _check_vs_oracle(_Oracle(oracle_mod, p), prec, spec.double().cpu().numpy(), gh, gh, sh, d)
            # and against the same request run alone on the GPU
            tol = _tol(prec)
            if gref is not None:
                assert per_field_max_rel(gh, gref.double().cpu().numpy()) <= tol, r
            if sref is not None:
                assert per_field_max_rel(sh, sref.double().cpu().numpy()) <= tol, r
    batch.close()
    for p, *_ in setups:
        p.sync()
        p.close()


def test_batch_at_mixed_truncation_sizes_vs_oracle(st_mod, oracle_mod):
    """Requests of the mixed-truncation configuration's largest sizes in one
    graph-replayed batch; fields 0 and the last of each against the oracle."""
    cases = [
        # T, grid, nlat, nlon, precision, nfields, seed
        (639, "octahedral", 1280, 0, "bf16x3", 220, 1103),
        (511, "regular", 512, 1024, "tf32x3", 200, 1104),
        (159, "octahedral", 320, 0, "bf16x3", 37, 1105),
    ]
    setups = []
    for T, grid, nlat, nlon, prec, nf, seed in cases:
        p = st_mod.Plan(T, grid, nlat=nlat, nlon=nlon or None, precision=prec, max_fields=nf)
        a = inputs.spectra(T, nf, seed=seed)
        spec = torch.from_numpy(a).to("cuda", p.dtype)
        g = torch.zeros((nf, p.npts), dtype=p.dtype, device="cuda")
        out = torch.zeros((nf, p.nspec, 2), dtype=p.dtype, device="cuda")
        setups.append((p, a, spec, g, out, prec, nf))
    batch = st_mod.Batch([(p, "round", spec, g, out) for p, a, spec, g, out, prec, nf in setups])
    batch.run(graph=True)
    batch.run(graph=True)
    torch.cuda.synchronize()
    for p, a, spec, g, out, prec, nf in setups:
        pick = [0, nf - 1]
        gh = g[pick].double().cpu().numpy()
        sh = out[pick].double().cpu().numpy()
        orc = _Oracle(oracle_mod, p)
        err = per_field_max_rel(gh, orc.inv(a[pick]))
        assert err < _tol(prec), (p.T, "inverse", err)
        err = per_field_max_rel(_cplx(sh), orc.dir(gh))
        assert err < _tol(prec), (p.T, "direct", err)
    batch.close()
    for p, *_ in setups:
        p.close()


def test_batch_rejects_duplicate_plan(st_mod):
    p = st_mod.Plan(31, "regular", precision="bf16x3", max_fields=2)
    spec = torch.zeros((2, p.nspec, 2), device="cuda")
    g = torch.zeros((2, p.npts), device="cuda")
    with pytest.raises(st_mod.STError):
        st_mod.Batch([(p, "inv", spec, g, None), (p, "inv", spec, g, None)])
    p.close()


PERSIST = [
    # T, grid, nfields, direction
    (79, "regular", 7, "round"),
    (159, "octahedral", 33, "round"),
    (255, "regular", 3, "inv"),
    (127, "octahedral", 12, "dir"),
    (639, "octahedral", 40, "round"),
]


@pytest.mark.parametrize("prec", ["bf16x3"])
def test_persistent_launch_matches_staged_launches(st_mod, oracle_mod, prec):
    """The whole batch in one persistent launch gives the per-stage launches'
    results, on two runs in a row, to within the last bits (its row-FFT
    bodies are separately compiled instances of the same code, so the
    compiler may fuse multiply-adds differently); sampled fields against the
    oracle."""
    reqs = PERSIST if prec == "bf16x3" else PERSIST[:3]
    made = [_make(st_mod, 40 + i, T, grid, prec, nf, d) for i, (T, grid, nf, d) in enumerate(reqs)]
    items = [(p, d, spec if d != "dir" else None, g, out if d != "inv" else None)
             for (p, spec, g, out), (_, _, _, d) in zip(made, reqs)]
    b = st_mod.Batch(items)
    b.run(graph=False)
    torch.cuda.synchronize()
    ref = [(g.clone(), out.clone()) for (_, _, g, out) in made]
    for _ in range(2):
        for (p, spec, g, out), (_, _, _, d) in zip(made, reqs):
            out.zero_()
            if d != "dir":
                g.zero_()
        b.run(persistent=True)
        torch.cuda.synchronize()
        for (p, spec, g, out), (gr, outr), (_, _, _, d) in zip(made, ref, reqs):
            p.sync()
            if d != "dir":
                assert per_field_max_rel(g.double().cpu().numpy(), gr.double().cpu().numpy()) < 1e-6
            if d != "inv":
                assert per_field_max_rel(out.double().cpu().numpy(), outr.double().cpu().numpy()) < 1e-6
    # the staged results themselves, one field of each request, vs the oracle
    for (p, spec, g, out), (T, grid, nf, d) in zip(made, reqs):
        o = _Oracle(oracle_mod, p)
        a = spec.double().cpu().numpy()
        if d != "dir":
            ref_g = oracle_mod.inv_trans(T, o.rows, o.mu, a[:1])
            assert per_field_max_rel(g[:1].double().cpu().numpy(), ref_g) < _tol(prec)
        if d != "inv":
            ref_s = oracle_mod.dir_trans(T, o.rows, o.mu, o.w, g[:1].double().cpu().numpy())
            got = out[:1].double().cpu().numpy()
            assert per_field_max_rel(got[..., 0] + 1j * got[..., 1], ref_s) < _tol(prec)
    b.close()
    for p, *_ in made:
        p.close()


@pytest.mark.parametrize("precs", [("bf16x3", "fp64"), ("tf32x3", "tf32x3")])
def test_persistent_launch_refuses_other_batches(st_mod, precs):
    """Mixed precisions, or a precision other than BF16x3, run per stage only."""
    made = [_make(st_mod, 60 + i, 31, "regular", pr, 2, "round") for i, pr in enumerate(precs)]
    b = st_mod.Batch([(p, "round", spec, g, out) for (p, spec, g, out) in made])
    with pytest.raises(st_mod.STError):
        b.run(persistent=True)
    b.run(graph=False)
    torch.cuda.synchronize()
    b.close()
    for p, *_ in made:
        p.close()
