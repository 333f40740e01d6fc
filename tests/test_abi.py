"""Checks of the C ABI: the library builds, loads, and exports every entry
point declared in include/sgkiif.h, and the binding declares exactly the
header's functions (CPU, no compute calls); on a GPU, the runtime loads the
sm_103a image of its kernels."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sgkiif.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sgk_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1810_11111_gb300 import build, sgkiif
    if not os.path.exists(sgkiif.LIB_PATH):
        build.build()
    return sgkiif.load()


def test_header_declares_the_boundary():
    fns = header_functions()
    for name in ["sgk_index_build", "sgk_operator_assemble", "sgk_solver_step", "sgk_solver_get_state",
                 "sgk_matvec", "sgk_reaction_eval", "sgk_krylov_expv", "sgk_expm_e1"]:
        assert name in fns


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_matches_header():
    from paper_1810_11111_gb300 import sgkiif
    assert sgkiif.exported_symbols() == header_functions()


@pytest.mark.gpu
def test_loaded_device_code_is_sm103(lib):
    # the runtime's view of the image it loaded for the library's kernels
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1810_11111_gb300 import sgkiif
    assert sgkiif.binary_arch() == 103


def test_host_dof_count_matches_closed_form(lib):
    from oracle.index_set import IndexSet as OIndex
    from paper_1810_11111_gb300 import sgkiif
    for d, n, k in [(1, 0, 1), (2, 4, 1), (3, 6, 2), (4, 9, 3), (6, 3, 2)]:
        assert sgkiif.dof_of(d, n, k) == OIndex(d, n, k).dof
    assert sgkiif.sgk_dof(0, 3, 1) == -1 and sgkiif.sgk_dof(2, 13, 1) == -1 and sgkiif.sgk_dof(2, 3, 4) == -1


def test_context_creation_without_gpu_fails_cleanly(lib):
    import ctypes

    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1810_11111_gb300 import sgkiif
    h = ctypes.c_void_p()
    assert sgkiif.sgk_ctx_create(ctypes.byref(h), 0, None, 0) == sgkiif.SGK_ECUDA


def test_alu_peak_rejects_bad_arguments(lib):
    import ctypes

    import torch
    from paper_1810_11111_gb300 import sgkiif
    out = ctypes.c_double(0.0)
    assert sgkiif.sgk_alu_peak(0, sgkiif.SGK_PEAK_FP32_FMA, None) == sgkiif.SGK_EINVAL
    assert sgkiif.sgk_alu_peak(0, 7, ctypes.byref(out)) == sgkiif.SGK_EINVAL
    assert sgkiif.sgk_alu_peak(-1, sgkiif.SGK_PEAK_FP64_FMA, ctypes.byref(out)) in (sgkiif.SGK_EINVAL,
                                                                                     sgkiif.SGK_ECUDA)
    if not torch.cuda.is_available():
        assert sgkiif.sgk_alu_peak(0, sgkiif.SGK_PEAK_FP64_FMA, ctypes.byref(out)) in (sgkiif.SGK_EINVAL,
                                                                                        sgkiif.SGK_ECUDA)


def test_iif_alpha_is_adams_moulton(lib):
    # eq. krylov4's weights are the Adams-Moulton coefficients (the same
    # Lagrange integrals; textbook values), computed by the library's host code
    import numpy as np

    from paper_1810_11111_gb300 import sgkiif
    table = {2: (1 / 2, 1 / 2), 3: (5 / 12, 8 / 12, -1 / 12), 4: (9 / 24, 19 / 24, -5 / 24, 1 / 24),
             5: (251 / 720, 646 / 720, -264 / 720, 106 / 720, -19 / 720),
             6: (475 / 1440, 1427 / 1440, -798 / 1440, 482 / 1440, -173 / 1440, 27 / 1440)}
    for r, want in table.items():
        out = np.zeros(r)
        assert sgkiif.sgk_iif_alpha(r, out.ctypes.data) == sgkiif.SGK_OK
        assert np.max(np.abs(out - np.array(want))) < 1e-15, (r, out)
    out = np.zeros(8)
    for r in (1, 7):
        assert sgkiif.sgk_iif_alpha(r, out.ctypes.data) == sgkiif.SGK_EINVAL


def test_cross_blocks_match_the_oracle(lib):
    # the library's host tables for the mixed-derivative terms (built from
    # closed-form Legendre traces in C++) against the oracle's direct
    # evaluation of the hierarchical functions; no GPU involved
    import numpy as np

    from oracle.operator import DIRICHLET0, PERIODIC, cross_blocks_1d
    from paper_1810_11111_gb300 import sgkiif
    for n, k in ((0, 1), (1, 2), (3, 1), (4, 2), (3, 3)):
        for bc, obc in ((sgkiif.SGK_PERIODIC, PERIODIC), (sgkiif.SGK_DIRICHLET0, DIRICHLET0)):
            H = (k + 1) << n
            P = np.zeros(H * H)
            E = np.zeros(H * H)
            assert sgkiif.sgk_cross_blocks_1d(n, k, bc, P.ctypes.data, E.ctypes.data, H * H) == sgkiif.SGK_OK
            Pw, Ew = cross_blocks_1d(n, k, obc)
            for got, want in ((P.reshape(H, H), Pw), (E.reshape(H, H), Ew)):
                assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max()), (n, k, bc)
    out = np.zeros(4)
    assert sgkiif.sgk_cross_blocks_1d(1, 1, 0, out.ctypes.data, out.ctypes.data, 4) == sgkiif.SGK_EINVAL


def test_interp_factors_match_the_oracle(lib):
    # the library's host tables of the interpolation form of the reaction
    # term (each entry from its local formula in long double, C++) against
    # the oracle's (dense evaluation and dense solves, numpy); no GPU involved
    import numpy as np

    from oracle.interp import one_dim_factors
    from paper_1810_11111_gb300 import sgkiif
    for n, k in ((0, 1), (1, 2), (3, 1), (4, 2), (3, 3), (5, 3), (6, 1)):
        want = one_dim_factors(n, k)
        for which in range(4):
            got = sgkiif.interp_factors_1d(n, k, which)
            scale = max(1.0, np.abs(want[which]).max())
            assert np.abs(got - want[which]).max() <= 1e-12 * scale, (n, k, which)
            # the same sparsity: nothing stored where the oracle's entry vanishes
            assert np.all(np.abs(got[np.abs(want[which]) <= 1e-13 * scale]) <= 1e-12 * scale)
    out = np.zeros(4)
    assert sgkiif.sgk_interp_factors_1d(1, 1, 0, out.ctypes.data, 4) == sgkiif.SGK_EINVAL
    assert sgkiif.sgk_interp_factors_1d(1, 1, 4, out.ctypes.data, 16) == sgkiif.SGK_EINVAL
