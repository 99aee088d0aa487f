"""CPU-side checks of the C ABI: the library builds, loads, and exports every
entry point include/hf.h declares; the binding's signature table covers them;
the oracle stays out of the product package."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "hf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hf_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_paper_calls():
    syms = declared_symbols()
    for name in ("hf_mesh_create", "hf_set_material", "hf_set_injection", "hf_newton_step",
                 "hf_check_fracture_criterion", "hf_get_opening_pressure", "hf_accept_step"):
        assert name in syms


def test_library_builds_loads_and_exports_every_declared_symbol():
    import paper_1911_10275_gb300 as pkg
    lib = pkg.load()
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(declared_symbols()) <= set(pkg.SIGNATURES)


def test_default_options_and_no_device_needed_for_defaults():
    import ctypes
    import paper_1911_10275_gb300 as pkg
    lib = pkg.load()
    o = pkg.hf_solver_opts()
    lib.hf_default_solver_opts(ctypes.byref(o))
    assert o.restart == 60 and o.reorth == 3 and o.scheme == 0 and o.coarse == 1 and o.precision == pkg.HF_PREC_FP64 and o.jacobi_block >= 1
    assert lib.hf_last_error(None) == b"null handle"


def test_product_package_never_imports_the_oracle():
    pkgdir = os.path.join(ROOT, "paper_1911_10275_gb300")
    for dp, _, files in os.walk(pkgdir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dp, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f


def test_invalid_mesh_is_rejected_without_a_device():
    """Malformed descriptors fail with HF_ERR_INVALID_ARG before any CUDA call."""
    import ctypes
    import paper_1911_10275_gb300 as pkg
    lib = pkg.load()
    d = pkg.hf_mesh_desc()
    d.dim = 4
    d.order = 2
    h = ctypes.c_void_p()
    assert lib.hf_mesh_create(ctypes.byref(d), None, ctypes.byref(h)) == -1
    assert not h.value
