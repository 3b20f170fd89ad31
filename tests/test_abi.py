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


def test_descriptor_output_shape_is_checked_before_the_library_is_called(monkeypatch):
    """A q of the wrong shape would make the descriptor kernel write past its end: the
    binding refuses it with ValueError before any call into libnep."""
    torch = pytest.importorskip("torch")
    from paper_2205_10046_gb300 import nep, workloads as W

    def no_library(*a, **k):
        raise AssertionError("the library was called")

    monkeypatch.setattr(nep, "load", no_library)
    w = W.si_diamond(1, seed=0, with_velocities=False)  # 8 atoms, N_des = 39
    pos = torch.tensor(w.pos)
    types = torch.tensor(w.types)
    for bad in ((w.n_atoms, w.model.n_des - 1), (w.n_atoms - 1, w.model.n_des), (w.n_atoms * w.model.n_des,)):
        q = torch.zeros(bad, dtype=torch.float64)
        with pytest.raises(ValueError, match="q has shape"):
            nep.nep_descriptors_static(w.model, pos, types, w.box, q)


def test_server_configuration_is_checked_without_gpu(lib):
    """nep_server_create refuses configurations outside the documented ranges before it
    touches a device (workers, precision, compact_every, min_chunk)."""
    from paper_2205_10046_gb300 import nep, workloads as W
    model = W.mixed_model(0)
    for bad in (dict(min_chunk=33), dict(min_chunk=-1), dict(compact_every=-1), dict(compact_every=1025),
                dict(workers=0), dict(precision=3)):
        kw = dict(memory_budget=1 << 30, workers=4)
        kw.update(bad)
        with pytest.raises(nep.NepError) as ei:
            nep.Server(model, **kw)
        assert ei.value.code == -1, bad
