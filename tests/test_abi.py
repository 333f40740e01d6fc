"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every entry point declared in include/sgkiif.h (no compute calls: there is no
GPU here).  The binding declares exactly the header's functions."""
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


def test_library_is_built_for_sm103a(lib):
    from paper_1810_11111_gb300 import sgkiif
    data = open(sgkiif.LIB_PATH, "rb").read()
    assert b"sm_103a" in data or b"sm_103" in data


def test_context_creation_without_gpu_fails_cleanly(lib):
    import ctypes

    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1810_11111_gb300 import sgkiif
    h = ctypes.c_void_p()
    assert sgkiif.sgk_ctx_create(ctypes.byref(h), 0, None, 0) == sgkiif.SGK_ECUDA
