"""The C-ABI library loads and exports every function declared in include/ift.h
(no compute calls: runs without a GPU)."""

import ctypes
import os
import re

import pytest

from paper_2305_15661_gb300 import ift

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ift_[a-z0-9_]+)\s*\(", text))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ift_set_mesh", "ift_set_bases", "ift_set_eq_weights", "ift_reduced_residual_jacobian",
                     "ift_solve_rom"):
        assert required in names


def test_library_exports_every_declared_symbol():
    if not os.path.exists(ift.LIB_PATH):
        pytest.skip("library not built here")
    lib = ctypes.CDLL(ift.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(ift.EXPORTS) <= declared_functions()


def test_config_defaults_without_gpu():
    if not os.path.exists(ift.LIB_PATH):
        pytest.skip("library not built here")
    lib = ift.load()
    cfg = ift.Config()
    lib.ift_config_default(ctypes.byref(cfg))
    assert cfg.gamma == 1.4 and cfg.eps_g == 1e-8 and cfg.tol == 1e-8 and cfg.max_iters == 200
