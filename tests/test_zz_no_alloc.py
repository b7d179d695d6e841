"""st_inv_trans_static: the inverse transform for callers that cannot
allocate device memory where they run it (real-time loops where an
allocation may stall, frameworks that own all device memory).  Its scratch is
a fixed array inside the library instead of the plan's workspace.

Checked here through the C ABI: two calls in a row agree with st_inv_trans
(within the split-precision tolerance the other parity tests use), a call
after another plan with a different layout and precision has used the array
still agrees, more fields than the plan's max_fields work while the array
holds them, the launches are counted with the plan's, and a request too
large for the array is refused.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1908_06096_gb300 import inputs
from tests.conftest import max_rel

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "bf16x3": 2e-5, "tf32x3": 2e-5, "fp32": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _spec(T, nf, seed, dtype):
    return torch.from_numpy(inputs.spectra(T, nf, seed=seed)).to("cuda", dtype)


def _static_call(st_mod, plan, spec, out):
    lib = st_mod.load()
    nf = spec.numel() // (plan.nspec * 2)
    return lib.st_inv_trans_static(plan.handle, ctypes.c_void_p(spec.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                   nf, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("T,grid,prec,nf", [(63, "octahedral", "bf16x3", 5), (31, "regular", "fp64", 3)])
def test_static_scratch_matches_workspace_path_twice(st_mod, T, grid, prec, nf):
    plan = st_mod.Plan(T, grid, precision=prec, max_fields=nf)
    for seed in (11, 12):                      # two calls in a row, different inputs
        spec = _spec(T, nf, seed, plan.dtype)
        ref = plan.inv(spec).clone()
        out = torch.full_like(ref, float("nan"))
        rc = _static_call(st_mod, plan, spec, out)
        assert rc == 0, st_mod.load().st_last_error()
        torch.cuda.synchronize()
        assert max_rel(out.double().cpu().numpy(), ref.double().cpu().numpy()) <= TOL[prec]
    plan.close()


def test_static_scratch_after_other_layouts(st_mod):
    """The array keeps the previous call's bytes; a call on a plan with another
    truncation, precision and field count in between must not leak into it."""
    a = st_mod.Plan(63, "octahedral", precision="bf16x3", max_fields=7)
    b = st_mod.Plan(47, "regular", precision="tf32x3", max_fields=2)
    sa = _spec(63, 7, 21, torch.float32)
    sb = _spec(47, 2, 22, torch.float32)
    ref_a = a.inv(sa).clone()
    ref_b = b.inv(sb).clone()
    out_a1 = a.inv_static(sa).clone()
    out_b = b.inv_static(sb).clone()
    out_a2 = a.inv_static(sa).clone()
    torch.cuda.synchronize()
    for out, ref in ((out_a1, ref_a), (out_b, ref_b), (out_a2, ref_a)):
        assert torch.isfinite(out).all()
        assert max_rel(out.double().cpu().numpy(), ref.double().cpu().numpy()) <= TOL["bf16x3"]
    a.close()
    b.close()


def test_static_scratch_rejects_oversize(st_mod):
    lib = st_mod.load()
    limit = int(lib.st_static_scratch_bytes())
    assert limit == 32 << 20
    plan = st_mod.Plan(255, "regular", precision="bf16x3", max_fields=64)
    spec = _spec(255, 64, 5, torch.float32)
    out = torch.empty((64, plan.npts), device="cuda")
    rc = _static_call(st_mod, plan, spec, out)
    assert rc == 1  # ST_ERR_ARG
    assert b"static scratch" in lib.st_last_error()
    plan.close()


def test_static_scratch_beyond_max_fields_and_counted(st_mod):
    """nfields above the plan's max_fields (the array, not the plan's
    workspace, bounds the static call) agrees with a plan sized for them; the
    call's three launches are counted with the plan's."""
    small = st_mod.Plan(31, "regular", precision="bf16x3", max_fields=2)
    big = st_mod.Plan(31, "regular", precision="bf16x3", max_fields=5)
    spec = _spec(31, 5, 31, torch.float32)
    ref = big.inv(spec).clone()
    small.reset_timings()
    out = torch.full_like(ref, float("nan"))
    rc = _static_call(st_mod, small, spec, out)
    assert rc == 0, st_mod.load().st_last_error()
    torch.cuda.synchronize()
    assert max_rel(out.double().cpu().numpy(), ref.double().cpu().numpy()) <= TOL["bf16x3"]
    counts = {k: v["launches"] for k, v in small.timings().items()}
    assert counts.get("pack_spectra") == 1 and counts.get("fft_inverse") == 1
    assert counts.get("legendre_inverse_tcgen05") == 1
    small.close()
    big.close()
