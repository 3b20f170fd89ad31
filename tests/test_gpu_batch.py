"""Batched evaluation (nep_compute_batch) against the FP64 oracle, structure by structure.

Every structure of a batch is an independent periodic system (the training set of
Sec. III). Per structure: forces within relative RMS 1e-5 of the oracle, |E_s - E_ref| / N_s
<= 1e-6 eV, per-structure virial error / N_s <= 1e-6 eV, per-atom energies within 2e-5 eV.
A structure evaluated inside a batch takes the same neighbour order and the same per-atom
arithmetic as on its own, so per-atom U, F and W must equal the single-structure call
bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2205_10046_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL_F = 1e-5
DE_ATOM = 1e-6


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_10046_gb300 import build
    build.build()
    return torch


def _dev(torch, b):
    p = torch.tensor(b.pos, dtype=torch.float64, device="cuda")
    t = torch.tensor(b.types, dtype=torch.int32, device="cuda")
    return p, t


def _run_batch(torch, h, b):
    p, t = _dev(torch, b)
    out = h.compute_batch(b.offsets, p, t, b.boxes, per_atom=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _mixed_batch():
    # sizes span the 8-atom cells (several periodic images per axis) up to 512 atoms, with
    # one empty structure in the middle
    sizes = [8, 8, 9, 12, 16, 0, 24, 31, 40, 55, 64, 77, 96, 128, 150, 200, 256, 300, 400, 512, 8]
    parts = []
    for s, n in enumerate(sizes):
        if n == 0:
            parts.append((np.zeros((0, 3)), np.zeros(0, np.int32), np.diag([9.0, 9.5, 10.0])))
        else:
            parts.append(W.random_structure(700 + s, n))
    return W.concat_structures(parts)


def _check_structure(g, b, s, U, F, Wv):
    a, e = int(b.offsets[s]), int(b.offsets[s + 1])
    n = e - a
    if n == 0:
        assert g["E_struct"][s] == 0.0 and np.all(g["W_struct"][s] == 0.0)
        return
    assert _rel(g["F"][a:e], F) <= REL_F, (s, _rel(g["F"][a:e], F))
    assert abs(g["E_struct"][s] - U.sum()) / n <= DE_ATOM, (s, g["E_struct"][s], U.sum())
    np.testing.assert_allclose(g["U"][a:e], U, rtol=0, atol=2e-5)
    assert np.abs(g["W_struct"][s] - Wv.sum(0)).max() / n <= DE_ATOM, s
    assert _rel(g["W"][a:e], Wv) <= REL_F, (s, _rel(g["W"][a:e], Wv))


def test_batch_matches_oracle_per_structure(torch_cuda):
    from paper_2205_10046_gb300 import nep
    model = W.mixed_model(0)
    b = _mixed_batch()
    h = nep.NEP(model)
    g = _run_batch(torch_cuda, h, b)
    for s in range(b.n_struct):
        pos, types, box = b.structure(s)
        if pos.shape[0] == 0:
            _check_structure(g, b, s, None, None, None)
            continue
        U, F, Wv = oracle.compute(model, pos, types, box)
        _check_structure(g, b, s, U, F, Wv)
    h.close()


def test_batch_equals_single_structure_calls(torch_cuda):
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    model = W.mixed_model(1)
    b = _mixed_batch()
    h = nep.NEP(model)
    g = _run_batch(torch, h, b)
    for s in range(b.n_struct):
        pos, types, box = b.structure(s)
        if pos.shape[0] == 0:
            continue
        p = torch.tensor(pos, dtype=torch.float64, device="cuda")
        t = torch.tensor(types, dtype=torch.int32, device="cuda")
        one = {k: v.cpu().numpy() for k, v in h.compute(p, t, box, per_atom_virial=True).items()}
        a, e = int(b.offsets[s]), int(b.offsets[s + 1])
        np.testing.assert_array_equal(g["F"][a:e], one["F"])
        np.testing.assert_array_equal(g["U"][a:e], one["U"])
        np.testing.assert_array_equal(g["W"][a:e], one["W"])
        assert abs(g["E_struct"][s] - one["E"][0]) <= 1e-9 * max(1.0, abs(one["E"][0]))
    h.close()


def test_batch_layout_reuse_and_change(torch_cuda):
    """Same layout twice with new positions (the grids are reused), then another layout."""
    from paper_2205_10046_gb300 import nep
    model = W.mixed_model(2)
    b = W.batch_structures(12, seed=11, n_max=96)
    h = nep.NEP(model)
    g1 = _run_batch(torch_cuda, h, b)
    b2 = W.Batch(b.offsets, b.pos + np.random.default_rng(5).normal(0, 0.05, b.pos.shape), b.types, b.boxes,
                 b.seeds)
    g2 = _run_batch(torch_cuda, h, b2)
    for bb, g in ((b, g1), (b2, g2)):
        for s in (0, 5, 11):
            U, F, Wv = oracle.compute(model, *bb.structure(s))
            _check_structure(g, bb, s, U, F, Wv)
    b3 = b.subset([3, 1, 7])
    g3 = _run_batch(torch_cuda, h, b3)
    for s in range(3):
        U, F, Wv = oracle.compute(model, *b3.structure(s))
        _check_structure(g3, b3, s, U, F, Wv)
    h.close()


def test_batch_forces_sum_to_zero_per_structure(torch_cuda):
    """Newton's third law holds inside every structure (Eq. F_ij), at any batch size."""
    from paper_2205_10046_gb300 import nep
    b = W.batch_structures(256, seed=4)
    h = nep.NEP(W.mixed_model(0))
    g = _run_batch(torch_cuda, h, b)
    for s in range(b.n_struct):
        a, e = int(b.offsets[s]), int(b.offsets[s + 1])
        F = g["F"][a:e]
        assert np.abs(F.sum(0)).max() <= 1e-4 * max(1.0, np.abs(F).max()) * np.sqrt(e - a), s
    h.close()


def test_batch_edge_cases(torch_cuda):
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    h = nep.NEP(W.mixed_model(0))
    lib = nep.load()
    # no structures, and only empty structures
    empty = W.concat_structures([])
    nep.nep_compute_batch(h.h, empty.offsets, torch.zeros((0, 3), dtype=torch.float64, device="cuda"),
                          torch.zeros(0, dtype=torch.int32, device="cuda"), np.zeros((0, 3, 3)))
    parts = [(np.zeros((0, 3)), np.zeros(0, np.int32), np.eye(3) * 10.0)] * 3
    b = W.concat_structures(parts)
    out = h.compute_batch(b.offsets, torch.zeros((0, 3), dtype=torch.float64, device="cuda"),
                          torch.zeros(0, dtype=torch.int32, device="cuda"), b.boxes)
    torch.cuda.synchronize()
    assert np.all(out["E_struct"].cpu().numpy() == 0.0)
    # a cell thinner than a third of r_c + skin is refused on the host, naming the structure
    parts = [W.random_structure(1, 8), (np.zeros((1, 3)), np.zeros(1, np.int32), np.eye(3) * 1.5)]
    b = W.concat_structures(parts)
    p, t = _dev(torch, b)
    with pytest.raises(nep.NepError) as ei:
        h.compute_batch(b.offsets, p, t, b.boxes)
    assert ei.value.code == -6 and "structure 1" in str(ei.value)
    # malformed offsets
    for bad in ([1, 8, 9], [0, 8, 7]):
        off = np.asarray(bad, np.int32)
        rc = lib.nep_compute_batch(h.h, 2, off.ctypes.data, p.data_ptr(), t.data_ptr(),
                                   np.ascontiguousarray(b.boxes).ctypes.data, None, None,
                                   torch.empty((9, 3), dtype=torch.float64, device="cuda").data_ptr(), None, None,
                                   None)
        assert rc == -1
    # the handle still works afterwards
    b = _mixed_batch().subset([0, 1, 2])
    g = _run_batch(torch, h, b)
    U, F, Wv = oracle.compute(h.model, *b.structure(2))
    _check_structure(g, b, 2, U, F, Wv)
    h.close()


def test_full_batch_sampled_structures(torch_cuda):
    """The 4096-structure batch (atom counts uniform in [8, 512]); 24 sampled structures
    are compared with the oracle."""
    from paper_2205_10046_gb300 import nep
    model = W.mixed_model(0)
    b = W.batch_structures(4096, seed=3)
    h = nep.NEP(model)
    g = _run_batch(torch_cuda, h, b)
    rng = np.random.default_rng(0)
    sizes = np.diff(b.offsets)
    sample = list(rng.choice(b.n_struct, 20, replace=False)) + [int(np.argmin(sizes)), int(np.argmax(sizes)), 0,
                                                                  b.n_struct - 1]
    for s in sample:
        U, F, Wv = oracle.compute(model, *b.structure(int(s)))
        _check_structure(g, b, int(s), U, F, Wv)
    h.close()


def test_batch_graph_replay_and_regrow(torch_cuda):
    """Repeated calls on the same arrays replay one captured graph; positions changed in
    place are picked up; a structure compressed beyond the list capacity is caught by the
    status read and evaluated again with grown lists."""
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    model = W.mixed_model(0)
    b = W.batch_structures(16, seed=12, n_max=128)
    h = nep.NEP(model)
    p, t = _dev(torch, b)
    n, ns = b.n_atoms, b.n_struct
    f64 = dict(dtype=torch.float64, device="cuda")
    out = dict(U=torch.empty(n, **f64), E_struct=torch.empty(ns, **f64), F=torch.empty((n, 3), **f64),
               W=torch.empty((n, 9), **f64), W_struct=torch.empty((ns, 9), **f64))

    def call():
        nep.nep_compute_batch(h.h, b.offsets, p, t, b.boxes, out["U"], out["E_struct"], out["F"], out["W"],
                              out["W_struct"])
        torch.cuda.synchronize()
        return {k: v.cpu().numpy().copy() for k, v in out.items()}

    r0, r1 = call(), call()  # eager, eager + capture
    for k in r0:
        np.testing.assert_array_equal(r0[k], r1[k])
    rng = np.random.default_rng(9)
    pos2 = b.pos + rng.normal(0, 0.05, b.pos.shape)
    p.copy_(torch.tensor(pos2, **f64))
    r2, r3 = call(), call()  # replays
    for k in r2:
        np.testing.assert_array_equal(r2[k], r3[k])
    b2 = W.Batch(b.offsets, pos2, b.types, b.boxes, b.seeds)
    for s in (0, 7, 15):
        U, F, Wv = oracle.compute(model, *b2.structure(s))
        _check_structure(r2, b2, s, U, F, Wv)
    # compress structure 3 towards its cell origin: about 4.6 times the neighbours per atom
    a, e = int(b.offsets[3]), int(b.offsets[4])
    pos3 = pos2.copy()
    pos3[a:e] = 0.6 * pos2[a:e]
    p.copy_(torch.tensor(pos3, **f64))
    r4 = call()
    b3 = W.Batch(b.offsets, pos3, b.types, b.boxes, b.seeds)
    for s in (3, 4):
        U, F, Wv = oracle.compute(model, *b3.structure(s))
        _check_structure(r4, b3, s, U, F, Wv)
    h.close()


def test_block_shapes_and_autotune(torch_cuda):
    """Atoms per CTA change the speed only: per-atom and per-structure results are identical
    for every shape the autotuner may pick; the autotuner keeps the fastest of its candidates."""
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    b = W.batch_structures(64, seed=5)
    h = nep.NEP(W.mixed_model(0))
    ref3 = _run_batch(torch, h, b)  # the default: low-register FP32 form on 128-atom CTAs
    nep.nep_set_tuning(h.h, 0, 0, 0, 1)  # the register-resident form runs on 64 and 128
    ref = _run_batch(torch, h, b)
    for k in ref:  # the two forms differ only by FP32 rounding
        np.testing.assert_allclose(ref3[k], ref[k], rtol=1e-6, atol=1e-7, err_msg=k)
    for ab in (64, 128):
        for gb in (64, 128, 256):
            nep.nep_set_tuning(h.h, 0, ab, gb, 1)
            g = _run_batch(torch, h, b)
            for k in ref:
                np.testing.assert_array_equal(g[k], ref[k], err_msg=f"{k} atom_block={ab} gather_block={gb}")
    p, t = _dev(torch, b)
    tune = nep.nep_autotune(h.h, b.offsets, p, t, b.boxes, n_pop=0)
    assert tune["atom_block"] in (64, 128) and tune["gather_block"] in (64, 128, 256)
    assert tune["n_tried"] == 6 and 0 < tune["best_ms"] <= tune["default_ms"]
    g = _run_batch(torch, h, b)
    for k in ref:
        np.testing.assert_array_equal(g[k], ref[k])
    with pytest.raises(nep.NepError):
        nep.nep_set_tuning(h.h, 0, 96, 128)
    # the autotuner keeps the handle's form: only 128-atom CTAs for the low-register form
    nep.nep_set_tuning(h.h, 0, 0, 0, 3)
    tune = nep.nep_autotune(h.h, b.offsets, p, t, b.boxes, n_pop=0)
    assert tune["atom_block"] == 128 and tune["n_tried"] == 3 and tune["atom_form"] == 3
    g = _run_batch(torch, h, b)
    for k in ref3:
        np.testing.assert_array_equal(g[k], ref3[k])
    h.close()
