"""Failure detection without a GPU fault: a bounded device-side wait that
nothing can satisfy runs out, the kernel records it and exits cleanly, the
host sees ST_ERR_TIMEOUT, and the plan keeps working afterwards."""
import pytest
import torch

from paper_1908_06096_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_bounded_wait_times_out_and_plan_recovers(st_mod, prec):
    lib = st_mod.load()
    p = st_mod.Plan(63, "octahedral", precision=prec, max_fields=4)
    spec = torch.from_numpy(inputs.spectra(63, 4, seed=77)).to("cuda", torch.float32)
    ref = p.inv(spec).clone()
    p.sync()
    assert lib.st_plan_inject(p.handle, 1, 100) == 0
    p.inv(spec)                                   # this launch withholds its copies
    with pytest.raises(st_mod.STError) as ex:
        p.sync()
    assert ex.value.code == 4                     # ST_ERR_TIMEOUT
    p.sync()                                      # the error word was cleared
    again = p.inv(spec)
    p.sync()
    assert torch.equal(again, ref)
    p.close()


def test_inject_rejects_bad_arguments(st_mod):
    lib = st_mod.load()
    p = st_mod.Plan(31, "regular", precision="fp64", max_fields=1)
    assert lib.st_plan_inject(p.handle, 1, 100) == 5      # SIMT plan: unsupported
    p.close()
    q = st_mod.Plan(31, "regular", precision="bf16x3", max_fields=1)
    assert lib.st_plan_inject(q.handle, 1, 0) == 1
    assert lib.st_plan_inject(q.handle, 2, 100) == 1
    assert lib.st_plan_inject(q.handle, 0, 0) == 0
    q.close()
