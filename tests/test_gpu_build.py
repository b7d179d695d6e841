"""The library's kernels target the device they run on: compute capability
10.3 (GB300) and sm_103a code, as the CUDA runtime reports them for a kernel
of the library (st_build_info)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_kernels_are_sm103a_code_on_an_sm103_device(st_mod):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    major, minor, binary = st_mod.build_info()
    assert (major, minor) == (10, 3)
    assert binary == 103
