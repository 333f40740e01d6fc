"""Host-side logic of the serving path, on the CPU: the closed-form DOF count
used to size requests, the device-memory estimate used for admission, and
the server's refusal to start without a GPU."""
import ctypes

import pytest

from oracle.index_set import IndexSet as OIndex
from paper_1810_11111_gb300 import sgkiif


@pytest.fixture(scope="module")
def lib():
    import os

    from paper_1810_11111_gb300 import build
    if not os.path.exists(sgkiif.LIB_PATH):
        build.build()
    return sgkiif.load()


@pytest.mark.parametrize("d,n,k", [(1, 0, 1), (1, 6, 3), (2, 4, 1), (3, 6, 2), (4, 5, 2), (6, 3, 1), (2, 8, 2)])
def test_dof_formula_matches_oracle_index_set(d, n, k):
    assert sgkiif.dof_of(d, n, k) == OIndex(d, n, k).dof


def test_memory_estimate_shape(lib):
    est = sgkiif.sgk_estimate_bytes
    F64, MIX = sgkiif.SGK_FP64, sgkiif.SGK_MIXED
    assert est(0, 3, 1, 1, 30, F64, 1) == -1 and est(3, 3, 4, 1, 30, F64, 1) == -1
    assert est(3, 3, 1, 1, 0, F64, 1) == -1 and est(3, 3, 1, 5, 30, F64, 1) == -1
    base = est(3, 6, 2, 1, 30, MIX, 1)
    # the finest-grid reaction buffers dominate: (2S+1) H^d values at least
    H = 3 << 6
    assert base >= 3 * H ** 3 * 4
    # mixed keeps the FP64 buffers of F and adds the FP32 ones of the
    # Jacobian products
    assert base > est(3, 6, 2, 1, 30, F64, 1) >= 3 * H ** 3 * 8
    assert est(3, 6, 2, 1, 30, MIX, 0) < base          # no reaction buffers
    assert est(3, 7, 2, 1, 30, MIX, 1) > base          # finer grid
    assert est(3, 6, 2, 1, 60, MIX, 1) > base          # larger Krylov basis
    assert est(3, 6, 2, 2, 30, MIX, 1) > base          # second species
    # the Krylov basis alone: (M + 1) dof doubles
    dof = sgkiif.dof_of(3, 6, 2)
    assert est(3, 6, 2, 1, 30, MIX, 0) >= 31 * dof * 8


def test_server_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert sgkiif.sgk_server_create(0, 2, 0, 0.0, ctypes.byref(h)) == sgkiif.SGK_ECUDA
    assert sgkiif.sgk_server_create(0, 0, 0, 0.0, ctypes.byref(h)) == sgkiif.SGK_EINVAL


def test_batch_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert sgkiif.sgk_batch_create(0, 4, 0, ctypes.byref(h)) == sgkiif.SGK_ECUDA
    assert sgkiif.sgk_batch_create(0, 0, 0, ctypes.byref(h)) == sgkiif.SGK_EINVAL
    assert sgkiif.sgk_batch_count(None) == -1 and sgkiif.sgk_batch_dof(None, 0) == -1


def test_estimates_of_the_interpolation_form(lib):
    # has_reaction = 2 selects the interpolation form of F: no finest-grid
    # buffers, so its memory grows with the sparse-grid DOF only
    est, work = sgkiif.sgk_estimate_bytes, sgkiif.sgk_estimate_work
    MIX = sgkiif.SGK_MIXED
    for d, n, k in ((3, 6, 2), (4, 8, 2), (4, 9, 3)):
        dof = sgkiif.dof_of(d, n, k)
        sparse, quad, none = est(d, n, k, 1, 30, MIX, 2), est(d, n, k, 1, 30, MIX, 1), est(d, n, k, 1, 30, MIX, 0)
        assert none < sparse < quad
        assert sparse - none >= 10 * 8 * dof          # F, the stage buffer, 8 transform buffers
        assert sparse < none + 200 * 8 * dof
        assert 0 < work(d, n, k, 1, 30, 2) < work(d, n, k, 1, 30, 1)
    # the largest served shape fits a GB300 in this form only
    assert est(4, 9, 3, 2, 30, MIX, 2) < 100e9 < est(4, 9, 3, 2, 30, MIX, 1)
