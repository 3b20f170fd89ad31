"""The C-ABI library loads and exports every entry point that include/nep.h declares,
and the host-side argument checks answer without touching a GPU."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nep.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2205_10046_gb300 import build, nep
    build.build()
    return nep.load()


def test_header_declares_the_expected_calls():
    names = _declared()
    for must in ("nep_create", "nep_destroy", "nep_compute", "nep_compute_host", "md_init", "md_run",
                 "md_get_state", "nep_last_error", "nep_descriptors"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2205_10046_gb300 import build, nep
    out = subprocess.run(["nm", "-D", "--defined-only", build.OUT], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    declared = _declared()
    missing = [n for n in declared if n not in exported]
    assert not missing, missing
    assert set(declared) == set(nep.EXPORTED)


def test_argument_errors_without_gpu(lib):
    import ctypes as C
    from paper_2205_10046_gb300 import nep
    h = C.c_void_p()
    assert lib.nep_create(None, C.byref(h)) == -1
    assert b"null" in lib.nep_last_error(None)
    p = nep.nep_params()
    p.version = 2
    assert lib.nep_create(C.byref(p), C.byref(h)) == -1
    assert lib.nep_destroy(None) == 0


def test_supported_shapes_cover_the_workload_models(lib):
    from paper_2205_10046_gb300 import nep, workloads as W
    shapes = nep.nep_supported()
    for hyper in (W.SI_MODEL, W.PBTE_MODEL, W.MIXED_MODEL):
        key = (hyper["n_max_radial"], hyper["basis_radial"], hyper["n_max_angular"], hyper["basis_angular"],
               hyper["n_neuron"], hyper["l_max_3b"], hyper["l_max_4b"], hyper["l_max_5b"])
        assert key in shapes
