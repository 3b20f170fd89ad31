"""nep_descriptors_static: descriptors for callers that cannot allocate device memory.

It runs the same kernels as nep_descriptors but takes all scratch from a fixed device
array inside the library, so it must give the same descriptors. Two calls in a row (with
different structures) check that the shared scratch does not leak one call's data into the
next. This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2205_10046_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_10046_gb300 import build
    build.build()
    return torch


def _descriptors(torch, fn, model, pos, types, box):
    from paper_2205_10046_gb300 import nep
    q = torch.full((pos.shape[0], model.n_des), float("nan"), dtype=torch.float64, device="cuda")
    p = torch.tensor(pos, device="cuda")
    t = torch.tensor(types, device="cuda")
    if fn == "static":
        nep.nep_descriptors_static(model, p, t, box, q)
    else:
        h = nep.NEP(model)
        nep.nep_descriptors(h.h, p, t, box, q)
        torch.cuda.synchronize()
        h.close()
    torch.cuda.synchronize()
    return q.cpu().numpy()


def test_static_scratch_matches_allocating_entry_point(torch_cuda):
    torch = torch_cuda
    cases = [W.pbte_rocksalt(4, seed=1, with_velocities=False), W.si_diamond(3, seed=0, with_velocities=False)]
    for w in cases:  # two calls in a row through the static scratch
        got = _descriptors(torch, "static", w.model, w.pos, w.types, w.box)
        ref = _descriptors(torch, "handle", w.model, w.pos, w.types, w.box)
        assert np.all(np.isfinite(got))
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= 1e-5, rel
        np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-7)


def test_static_scratch_rejects_oversized_input(torch_cuda):
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    w = W.si_diamond(9, seed=0, with_velocities=False)  # 5832 atoms > NEP_STATIC_MAX_ATOMS
    q = torch.zeros((w.n_atoms, w.model.n_des), dtype=torch.float64, device="cuda")
    with pytest.raises(nep.NepError, match="NEP_STATIC_MAX_ATOMS"):
        nep.nep_descriptors_static(w.model, torch.tensor(w.pos, device="cuda"),
                                   torch.tensor(w.types, device="cuda"), w.box, q)


def test_static_scratch_refuses_lists_that_do_not_fit_then_recovers(torch_cuda):
    """4096 atoms of a dense FCC lattice (a = 2.7 A) with a 3 A skin: every per-atom list stays
    below the 512-entry limit, but the lists of all atoms need more than the 16 MiB scratch.
    The call is refused with NEP_ERR_ARG before any list is written, and a valid call right
    after it still matches the allocating entry point."""
    torch = torch_cuda
    import oracle
    from paper_2205_10046_gb300 import nep
    model = W.si_diamond(1, seed=0, with_velocities=False).model  # r_c 5.0 / 4.0 A
    pos, box, _ = W.lattice("fcc", 2.7, (8, 8, 16))
    pos = W.jitter(pos, 0.05, 7)
    types = np.zeros(pos.shape[0], np.int32)
    skin = 3.0
    # premise, from the oracle's brute-force counts within r_c + skin
    max_r = int(oracle.neighbor_counts(pos, box, model.rc_radial + skin).max())
    max_a = int(oracle.neighbor_counts(pos, box, model.rc_angular + skin).max())
    assert max_r < 512 and max_a < 512
    assert (max_r + 2 * max_a) * 4 * pos.shape[0] > 16 << 20
    q = torch.zeros((pos.shape[0], model.n_des), dtype=torch.float64, device="cuda")
    with pytest.raises(nep.NepError, match="NEP_STATIC_SCRATCH_BYTES") as ei:
        nep.nep_descriptors_static(model, torch.tensor(pos, device="cuda"), torch.tensor(types, device="cuda"),
                                   box, q, skin=skin)
    assert ei.value.code == -1  # NEP_ERR_ARG
    torch.cuda.synchronize()
    w = W.si_diamond(3, seed=0, with_velocities=False)
    got = _descriptors(torch, "static", w.model, w.pos, w.types, w.box)
    ref = _descriptors(torch, "handle", w.model, w.pos, w.types, w.box)
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-7)
