"""Neighbour lists, element by element: the library's radial and angular lists (Appendix B's
NN_i and NL_im, exported in caller order with each entry's pair vector) against the oracle's
brute-force search over every atom and every periodic image.

Integer work, so the bar is set equality of the (j, image) pairs of every atom. The image n
of a library entry is recovered from its pair vector: d = r_j - r_i + n H. Pairs whose
distance lies within 1e-4 A of the list radius can fall on either side in FP32 and are
checked only for validity (they are within rounding of the radius); there are few or none.
"""
import numpy as np
import pytest

import oracle
from paper_2205_10046_gb300 import workloads as W

pytestmark = pytest.mark.gpu

AMBIG = 1e-4  # A


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_10046_gb300 import build
    build.build()
    return torch


def _pairs_from_export(pos, box, ex, kind, rows, offset=0):
    """{i: {(j, n0, n1, n2): d}} for the caller rows `rows` (global indices into ex)."""
    inv = np.linalg.inv(box)
    out = {}
    nn, J, D = ex[f"nn_{kind}"], ex[f"j_{kind}"], ex[f"d_{kind}"]
    for i in rows:
        s = {}
        for m in range(nn[i]):
            j = int(J[i, m])
            d = D[i, m].astype(np.float64)
            n = np.rint((d - (pos[j - offset] - pos[i - offset])) @ inv).astype(int)
            key = (j - offset, int(n[0]), int(n[1]), int(n[2]))
            assert key not in s, f"atom {i}: duplicate entry {key}"
            s[key] = d
        out[i - offset] = s
    return out


def _compare(pos, box, got, rl):
    """Every atom's set of (j, n) equals the brute-force set within rl, up to pairs within
    AMBIG of rl; matched pair vectors agree to FP32 rounding."""
    n_pairs = 0
    for i, s in got.items():
        j, n, d = oracle.neighbors(pos, box, rl, i)
        ref = {(int(j[k]), *map(int, n[k])): d[k] for k in range(j.shape[0])}
        for key in set(ref) ^ set(s):
            dd = ref[key] if key in ref else s[key]
            assert abs(np.linalg.norm(dd) - rl) < AMBIG, f"atom {i}: pair {key} at {np.linalg.norm(dd):.6f} A"
        for key in set(ref) & set(s):
            assert np.abs(s[key] - ref[key]).max() < 1e-4, (i, key)
        n_pairs += len(ref)
    return n_pairs


def _lists(torch, model, pos, types, box, skin):
    from paper_2205_10046_gb300 import nep
    h = nep.NEP(model, skin=skin)
    h.compute(torch.tensor(pos, device="cuda"), torch.tensor(types, device="cuda"), box)
    torch.cuda.synchronize()
    ex = nep.nep_export_lists(h.h, pos.shape[0])
    h.close()
    return ex


CASES = [("si216", lambda: W.si_diamond(3, seed=0, with_velocities=False)),
         ("pbte216", lambda: W.pbte_rocksalt(3, seed=1, with_velocities=False))]


@pytest.mark.parametrize("skin", [1e-9, 0.7])
@pytest.mark.parametrize("name,make", CASES)
def test_lists_equal_brute_force(torch_cuda, name, make, skin):
    w = make()
    ex = _lists(torch_cuda, w.model, w.pos, w.types, w.box, skin)
    for kind, rc in (("r", w.model.rc_radial), ("a", w.model.rc_angular)):
        got = _pairs_from_export(w.pos, w.box, ex, kind, range(w.n_atoms))
        assert _compare(w.pos, w.box, got, rc + skin) > 0
    # the radial list is grouped by neighbour type, type 0 first
    for i in range(w.n_atoms):
        tj = w.types[ex["j_r"][i, :ex["nn_r"][i]]]
        assert np.all(np.diff(tj) >= 0)


@pytest.mark.parametrize("seed,n", [(0, 8), (1, 13), (2, 31), (3, 64), (5, 150)])
def test_lists_of_thin_triclinic_cells(torch_cuda, seed, n):
    """Sheared cells thinner than 2 r_c: one atom meets many images of the same neighbour."""
    pos, types, box = W.random_structure(seed, n)
    model = W.random_model(W.MIXED_MODEL, seed, [W.MASS_SI, W.MASS_GE, W.MASS_C])
    ex = _lists(torch_cuda, model, pos, types, box, 1e-9)
    for kind, rc in (("r", model.rc_radial), ("a", model.rc_angular)):
        got = _pairs_from_export(pos, box, ex, kind, range(n))
        assert _compare(pos, box, got, rc) > 0


def test_batch_lists_equal_per_structure_brute_force(torch_cuda):
    """The batched builder (per-structure grids and shift tables): every structure's lists
    against the brute-force search of that structure alone."""
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    b = W.batch_structures(6, seed=11, n_min=8, n_max=120)
    model = W.mixed_model(0)
    h = nep.NEP(model, skin=1e-9)
    h.compute_batch(b.offsets, torch.tensor(b.pos, device="cuda"), torch.tensor(b.types, device="cuda"), b.boxes)
    torch.cuda.synchronize()
    ex = nep.nep_export_lists(h.h, b.n_atoms)
    h.close()
    for s in range(b.n_struct):
        pos, types, box = b.structure(s)
        a0, a1 = int(b.offsets[s]), int(b.offsets[s + 1])
        for kind, rc in (("r", model.rc_radial), ("a", model.rc_angular)):
            # every neighbour of a structure's atom lies in the same structure
            J = ex[f"j_{kind}"][a0:a1]
            for i in range(a1 - a0):
                assert np.all((J[i, :ex[f"nn_{kind}"][a0 + i]] >= a0) & (J[i, :ex[f"nn_{kind}"][a0 + i]] < a1))
            got = _pairs_from_export(pos, box, ex, kind, range(a0, a1), offset=a0)
            assert _compare(pos, box, got, rc) > 0
