"""The large single-GPU workload: Si diamond, 100^3 conventional cells (8,000,000 atoms), NEP
r_c 5.0/4.0 A, n_max 8/4, 50 neurons, random weights (seed 0), in the launch configuration
the bench times.

The GPU evaluates the whole periodic box. The FP64 oracle evaluates the 4096 atoms of
conventional cells [0, 8)^3, cut out together with every atom within 2 r_c^R (the neighbours
of their neighbours) as an open cluster, so the inner atoms' energies, forces and virials
are exact. Bars: FP32 form relative force RMS <= 1e-5, |sum dU| / 4096 <= 1e-6 eV, per-atom
virial relative RMS <= 1e-5; BF16 forms force RMSE <= 1 meV/A (the relative RMS is printed),
and the split-BF16 form also relative force RMS <= 1e-4.
"""
import numpy as np
import pytest

import oracle
from paper_2205_10046_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL_F = 1e-5
DE_ATOM = 1e-6
F_RMSE_BF16 = 1e-3


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_10046_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def si8m():
    w = W.si_diamond(100, seed=0, with_velocities=False)
    cpos, ctypes, cbox, inner, sel = W.subcell_cluster(w, 100, 8)
    U, F, Wv = oracle.compute(w.model, cpos, ctypes, cbox, sel=inner)
    return w, sel, (U, F, Wv)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _gpu(torch, w, precisions):
    """Per form: FP32 with each per-atom kernel form (keys 0 and 'occ3'), then the BF16 forms."""
    from paper_2205_10046_gb300 import nep
    h = nep.NEP(w.model)
    p = torch.tensor(w.pos, device="cuda")
    t = torch.tensor(w.types, device="cuda")
    out = {}
    for prec in ("occ3",) + tuple(precisions):
        nep.nep_set_tuning(h.h, 0, 0, 0, 3 if prec == "occ3" else 1)
        nep.nep_set_precision(h.h, 0 if prec == "occ3" else prec)
        r = h.compute(p, t, w.box, per_atom_virial=True)
        torch.cuda.synchronize()
        out[prec] = {k: v.cpu().numpy() for k, v in r.items()}
        del r
    h.close()
    return out


def test_si_8m_subcell_against_oracle(torch_cuda, si8m):
    w, sel, (U, F, Wv) = si8m
    assert sel.shape[0] == 4096
    g = _gpu(torch_cuda, w, (0, 1, 2))
    g32 = g[0]
    rel_f = _rel(g32["F"][sel], F)
    de = abs(g32["U"][sel].sum() - U.sum()) / sel.shape[0]
    rel_w = _rel(g32["W"][sel], Wv)
    print(f"FP32: relative force RMS {rel_f:.2e}, |sum dU|/N {de:.2e} eV, virial relative RMS {rel_w:.2e}")
    assert rel_f <= REL_F
    assert de <= DE_ATOM
    np.testing.assert_allclose(g32["U"][sel], U, rtol=0, atol=2e-5)
    assert rel_w <= REL_F
    # properties of the whole box
    assert np.abs(g32["F"].sum(0)).max() < 1e-6 * np.abs(g32["F"]).sum() / 3
    assert abs(g32["E"][0] - g32["U"].sum()) < 1e-9 * abs(g32["E"][0])
    np.testing.assert_allclose(g32["W_total"], g32["W"].sum(0), rtol=1e-9, atol=1e-6)
    # the low-register FP32 kernel form: same bars
    g3 = g["occ3"]
    print(f"FP32 form 3: relative force RMS {_rel(g3['F'][sel], F):.2e}")
    assert _rel(g3["F"][sel], F) <= REL_F
    assert abs(g3["U"][sel].sum() - U.sum()) / sel.shape[0] <= DE_ATOM
    assert _rel(g3["W"][sel], Wv) <= REL_F
    for prec in sorted(k for k in g if k not in (0, "occ3")):
        gb = g[prec]
        rmse = float(np.sqrt(np.mean((gb["F"][sel] - F) ** 2)))
        print(f"BF16 form {prec}: force RMSE {rmse:.2e} eV/A (relative RMS {_rel(gb['F'][sel], F):.2e}, "
              f"|F| rms {np.sqrt(np.mean(F ** 2)):.2e}), |sum dU|/N {abs(gb['U'][sel].sum() - U.sum()) / 4096:.2e} eV")
        assert rmse <= F_RMSE_BF16
        if prec == 2:
            assert _rel(gb["F"][sel], F) <= 1e-4
