"""Host-side checks of the C ABI: the library builds for sm_103a, loads
without a GPU, and exports every function include/apgb.h declares."""
import ctypes

import pytest

from paper_0910_1650_gb300 import build as b
from paper_0910_1650_gb300 import capi


@pytest.fixture(scope="module")
def lib():
    b.build()
    return capi.lib()


def test_every_declared_function_is_exported(lib):
    names = capi.header_functions()
    assert "ap_iterate" in names and "ap_similarity" in names and "ap_exemplars" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    assert set(capi.header_functions()) <= set(capi._SIGNATURES)


def test_status_strings(lib):
    assert capi.status_string(0) == "ok"
    assert "invalid" in capi.status_string(-1)
    assert capi.status_string(12345) == "unknown status"
    assert lib.ap_version() >= 100


def test_workspace_queries_without_gpu(lib):
    assert lib.ap_exemplars_workspace_size(1000) > 0
    assert lib.ap_similarity_workspace_size(0, 3) == 0
    assert lib.ap_exemplars_workspace_size(0) == 0


def test_struct_layout():
    assert ctypes.sizeof(capi.ApParams) == 20
    assert ctypes.sizeof(capi.ApResult) == 56


def test_judge_is_the_half_percent_rule():
    """apl_judge (host only): keep the warm result exactly when its net
    similarity is within tol of the cold one's, both finite."""
    from paper_0910_1650_gb300 import capi
    cold = [-100.0, -100.0, -100.0, -100.0, float("nan"), -50.0]
    warm = [-100.5, -100.51, -99.5, -99.4, -100.0, float("inf")]
    assert capi.apl_judge(cold, warm, 0.005) == [True, False, True, False, False, False]
    assert capi.apl_judge([-1.0], [-1.0], 0.0) == [True]
