import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU oracle case")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def st_mod():
    """The CUDA library binding; builds the shared library if it is missing."""
    from paper_1908_06096_gb300 import st
    st.ensure_built()
    return st


def max_rel(x, ref):
    """Normwise max relative error: max|x - ref| / max|ref| (per whole array)."""
    import numpy as np
    x = np.asarray(x)
    ref = np.asarray(ref)
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(x - ref)) / (den if den > 0 else 1.0))


def per_field_max_rel(x, ref):
    """Normwise max relative error per field (first axis), worst field."""
    import numpy as np
    x = np.asarray(x).reshape(len(x), -1)
    ref = np.asarray(ref).reshape(len(ref), -1)
    den = np.max(np.abs(ref), axis=1)
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.max(np.abs(x - ref), axis=1) / den))
