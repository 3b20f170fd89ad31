"""GPU (libnep, FP32 internals) against the FP64 oracle, through the C ABI.

Tolerances (FP32 path): relative force RMS ||F_gpu - F_ref|| / ||F_ref|| <= 1e-5,
|E_gpu - E_ref| / N <= 1e-6 eV, total-virial error / N <= 1e-6 eV, per-atom virial
relative RMS <= 1e-5, descriptor relative RMS <= 1e-5. Integer work (neighbour counts) is
compared exactly.
"""
import numpy as np
import pytest

import oracle
from paper_2205_10046_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL_F = 1e-5
DE_ATOM = 1e-6
DW_ATOM = 1e-6


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_10046_gb300 import build
    build.build()
    return torch


def _gpu_compute(torch, model, pos, types, box, skin=1.0):
    from paper_2205_10046_gb300 import nep
    h = nep.NEP(model, skin=skin)
    p = torch.tensor(np.ascontiguousarray(pos), dtype=torch.float64, device="cuda")
    t = torch.tensor(np.ascontiguousarray(types), dtype=torch.int32, device="cuda")
    out = h.compute(p, t, box, per_atom_virial=True)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["stats"] = nep.nep_get_stats(h.h)
    h.close()
    return res


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _check_all(g, U, F, Wv, n):
    assert _rel(g["F"], F) <= REL_F, _rel(g["F"], F)
    assert abs(g["E"][0] - U.sum()) / n <= DE_ATOM
    np.testing.assert_allclose(g["U"], U, rtol=0, atol=2e-5)
    assert _rel(g["W"], Wv) <= REL_F, _rel(g["W"], Wv)
    assert np.abs(g["W_total"] - Wv.sum(0)).max() / n <= DW_ATOM


def test_si_diamond_216_matches_oracle(torch_cuda):
    w = W.si_diamond(3, seed=0, with_velocities=False)
    g = _gpu_compute(torch_cuda, w.model, w.pos, w.types, w.box)
    U, F, Wv = oracle.compute(w.model, w.pos, w.types, w.box)
    _check_all(g, U, F, Wv, w.n_atoms)


def test_descriptors_match_oracle(torch_cuda):
    from paper_2205_10046_gb300 import nep
    torch = torch_cuda
    for w in (W.si_diamond(3, seed=0, with_velocities=False), W.pbte_rocksalt(3, seed=1, with_velocities=False)):
        h = nep.NEP(w.model)
        n = w.n_atoms
        q = torch.zeros((n, w.model.n_des), dtype=torch.float64, device="cuda")
        nep.nep_descriptors(h.h, torch.tensor(w.pos, device="cuda"), torch.tensor(w.types, device="cuda"), w.box, q)
        torch.cuda.synchronize()
        qr = oracle.descriptors(w.model, w.pos, w.types, w.box)
        qg = q.cpu().numpy()
        assert _rel(qg, qr) <= 1e-5
        # every component, scaled by its own magnitude over the atoms
        scale = np.abs(qr).max(0) + 1e-12
        assert (np.abs(qg - qr) / scale).max() <= 2e-5
        h.close()


@pytest.mark.parametrize("reps", [2, 3, 4])
def test_pbte_two_species_matches_oracle(torch_cuda, reps):
    """reps = 2 puts many periodic images inside the cutoff (face distance < 2 r_c)."""
    w = W.pbte_rocksalt(reps, seed=1, with_velocities=False)
    g = _gpu_compute(torch_cuda, w.model, w.pos, w.types, w.box)
    U, F, Wv = oracle.compute(w.model, w.pos, w.types, w.box)
    _check_all(g, U, F, Wv, w.n_atoms)


@pytest.mark.parametrize("seed,n", [(0, 8), (1, 13), (2, 31), (3, 64), (4, 97), (5, 150)])
def test_small_triclinic_multi_species_cells(torch_cuda, seed, n):
    """Sheared FCC/BCC/diamond cells of 8..150 atoms with 1..3 species: thin cells where the
    list search spans several images per axis, and ragged atom counts."""
    pos, types, box = W.random_structure(seed, n)
    model = W.random_model(W.MIXED_MODEL, seed, [W.MASS_SI, W.MASS_GE, W.MASS_C])
    g = _gpu_compute(torch_cuda, model, pos, types, box)
    U, F, Wv = oracle.compute(model, pos, types, box)
    _check_all(g, U, F, Wv, n)


def test_neighbour_counts_are_exact(torch_cuda):
    """With skin 0 the library's list lengths are the brute-force counts within r_c."""
    w = W.si_diamond(3, seed=0, with_velocities=False)
    g = _gpu_compute(torch_cuda, w.model, w.pos, w.types, w.box, skin=1e-9)
    counts = oracle.neighbor_counts(w.pos, w.box, w.model.rc_radial)
    st = g["stats"]
    assert st["max_radial"] == counts.max()
    assert st["mean_radial"] * w.n_atoms == pytest.approx(counts.sum(), abs=0.5)
    ca = oracle.neighbor_counts(w.pos, w.box, w.model.rc_angular)
    assert st["max_angular"] == ca.max()
    assert st["mean_angular"] * w.n_atoms == pytest.approx(ca.sum(), abs=0.5)


def test_degenerate_inputs(torch_cuda):
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    m = W.random_model(W.SI_MODEL, 0, [W.MASS_SI])
    h = nep.NEP(m)
    # an isolated atom: no neighbours, U = sum w1 tanh(-b0) - b1, F = 0
    g = h.compute(torch.tensor([[1.0, 2.0, 3.0]], dtype=torch.float64, device="cuda"),
                  torch.zeros(1, dtype=torch.int32, device="cuda"), np.eye(3) * 40.0, per_atom_virial=True)
    U, F, Wv = oracle.compute(m, np.array([[1.0, 2.0, 3.0]]), np.zeros(1, np.int32), np.eye(3) * 40.0)
    assert abs(g["U"].item() - U[0]) < 1e-6
    assert torch.all(g["F"] == 0) and torch.all(g["W"] == 0)
    # empty system
    e = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    nep.nep_compute(h.h, torch.zeros((0, 3), dtype=torch.float64, device="cuda"),
                    torch.zeros(0, dtype=torch.int32, device="cuda"), np.eye(3) * 10.0, None, e,
                    torch.zeros((0, 3), dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert e.item() == 0.0
    # errors are reported, not raised on the device
    pos = torch.tensor([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0]], dtype=torch.float64, device="cuda")
    with pytest.raises(nep.NepError, match="NEP_ERR_ARG"):
        h.compute(pos, torch.tensor([0, 5], dtype=torch.int32, device="cuda"), np.eye(3) * 20.0)
    bad = pos.clone()
    bad[1, 0] = float("nan")
    with pytest.raises(nep.NepError, match="NEP_ERR_NONFINITE"):
        h.compute(bad, torch.zeros(2, dtype=torch.int32, device="cuda"), np.eye(3) * 20.0)
    with pytest.raises(nep.NepError, match="NEP_ERR_ARG"):
        h.compute(pos, torch.zeros(2, dtype=torch.int32, device="cuda"), np.zeros((3, 3)))
    h.close()
    m2 = W.random_model(dict(W.SI_MODEL, n_max_radial=20, basis_radial=20), 0, [W.MASS_SI])
    with pytest.raises(nep.NepError, match="NEP_ERR_UNSUPPORTED"):
        nep.NEP(m2)  # beyond the run-time-shape kernels' n_max <= 19


def test_deterministic_bitwise(torch_cuda):
    w = W.pbte_rocksalt(4, seed=1, with_velocities=False)
    a = _gpu_compute(torch_cuda, w.model, w.pos, w.types, w.box)
    b = _gpu_compute(torch_cuda, w.model, w.pos, w.types, w.box)
    for k in ("U", "E", "F", "W", "W_total"):
        assert np.array_equal(a[k], b[k]), k


def test_host_entry_point_matches_device(torch_cuda):
    from paper_2205_10046_gb300 import nep
    w = W.pbte_rocksalt(3, seed=1, with_velocities=False)
    h = nep.NEP(w.model)
    U, E, F, Wv, Wt = nep.nep_compute_host(h.h, w.pos, w.types, w.box)
    g = _gpu_compute(torch_cuda, w.model, w.pos, w.types, w.box)
    assert np.array_equal(F, g["F"]) and np.array_equal(U, g["U"]) and E == g["E"][0]
    h.close()


def test_pbte_262144_sampled_against_oracle(torch_cuda):
    """The full medium workload (32^3 rocksalt cells) in the launch configuration the bench
    times; forces, energies and virials of sampled atoms against the oracle, plus totals."""
    w = W.pbte_rocksalt(32, seed=1, with_velocities=False)
    g = _gpu_compute(torch_cuda, w.model, w.pos, w.types, w.box)
    rng = np.random.default_rng(0)
    sel = np.sort(rng.choice(w.n_atoms, 24, replace=False))
    sel = np.r_[0, sel, w.n_atoms - 1]
    U, F, Wv = oracle.compute(w.model, w.pos, w.types, w.box, sel=sel)
    assert _rel(g["F"][sel], F) <= REL_F
    np.testing.assert_allclose(g["U"][sel], U, rtol=0, atol=2e-5)
    assert _rel(g["W"][sel], Wv) <= REL_F
    # properties that hold at any size
    assert np.abs(g["F"].sum(0)).max() < 1e-6 * np.abs(g["F"]).sum() / 3
    assert abs(g["E"][0] - g["U"].sum()) < 1e-9 * abs(g["E"][0])
    np.testing.assert_allclose(g["W_total"], g["W"].sum(0), rtol=1e-9, atol=1e-9)


def test_md_matches_oracle_trajectory(torch_cuda):
    """20 NVE steps of the 216-atom Si cell: per-step potential and kinetic energy and the
    final positions/velocities/forces against the FP64 oracle's velocity Verlet."""
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    w = W.si_diamond(3, seed=0)
    n_steps = 20
    h = nep.NEP(w.model)
    nep.md_init(h.h, torch.tensor(w.pos, device="cuda"), torch.tensor(w.types, device="cuda"), w.box,
                torch.tensor(w.vel, device="cuda"))
    th = torch.zeros((n_steps, 4), dtype=torch.float64, device="cuda")
    nep.md_run(h.h, n_steps, 1.0, 1, th)
    pos = torch.zeros((w.n_atoms, 3), dtype=torch.float64, device="cuda")
    vel = torch.zeros_like(pos)
    frc = torch.zeros_like(pos)
    nep.md_get_state(h.h, pos, vel, frc)
    torch.cuda.synchronize()
    p_ref, v_ref, th_ref, f_ref = oracle.md(w.model, w.pos, w.vel, w.types, w.box, n_steps, 1.0)
    thg = th.cpu().numpy()
    n = w.n_atoms
    assert np.abs(thg[:, 0] - th_ref[1:, 0]).max() / n <= 1e-6
    assert np.abs(thg[:, 1] - th_ref[1:, 1]).max() / n <= 1e-6
    np.testing.assert_allclose(thg[:, 2], th_ref[1:, 2], rtol=1e-5)
    L = w.box[0, 0]
    dx = pos.cpu().numpy() - p_ref
    dx -= L * np.round(dx / L)
    assert np.abs(dx).max() < 1e-6
    assert _rel(vel.cpu().numpy(), v_ref) < 1e-5
    assert _rel(frc.cpu().numpy(), f_ref) < 1e-4
    h.close()


def test_md_rebuilds_keep_forces_exact(torch_cuda):
    """A small skin forces neighbour rebuilds inside the captured step graph; after the run
    the forces at the GPU's own positions still match the oracle at those positions."""
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    w = W.pbte_rocksalt(3, seed=1, temperature=1500.0)
    h = nep.NEP(w.model, skin=0.1)
    nep.md_init(h.h, torch.tensor(w.pos, device="cuda"), torch.tensor(w.types, device="cuda"), w.box,
                torch.tensor(w.vel, device="cuda"))
    th = torch.zeros((40, 4), dtype=torch.float64, device="cuda")
    nep.md_run(h.h, 40, 2.0, 1, th)
    pos = torch.zeros((w.n_atoms, 3), dtype=torch.float64, device="cuda")
    frc = torch.zeros_like(pos)
    nep.md_get_state(h.h, pos, None, frc)
    torch.cuda.synchronize()
    st = nep.nep_get_stats(h.h)
    assert st["n_rebuilds"] >= 2, st
    p = pos.cpu().numpy()
    _, F, _ = oracle.compute(w.model, p, w.types, w.box)
    assert _rel(frc.cpu().numpy(), F) <= REL_F
    e = th.cpu().numpy()
    etot = e[:, 0] + e[:, 1]
    assert np.ptp(etot) / w.n_atoms < 1e-4
    h.close()


@pytest.mark.parametrize("seed,n", [(0, 8), (3, 64), (5, 150)])
def test_low_register_atom_form_matches_oracle(torch_cuda, seed, n):
    """The three-CTAs-per-SM form of the FP32 per-atom kernel (nep_tuning.atom_form = 3) on
    the mixed model (S_nk in 128 TMEM columns): same bars as the default form, and an MD run
    whose step graph uses it."""
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    pos, types, box = W.random_structure(seed, n)
    model = W.random_model(W.MIXED_MODEL, seed, [W.MASS_SI, W.MASS_GE, W.MASS_C])
    h = nep.NEP(model)
    nep.nep_set_tuning(h.h, 0, 0, 0, 3)
    assert nep.nep_get_tuning(h.h)["atom_form"] == 3
    p = torch.tensor(pos, device="cuda")
    t = torch.tensor(types, device="cuda")
    g = {k: v.cpu().numpy() for k, v in h.compute(p, t, box, per_atom_virial=True).items()}
    U, F, Wv = oracle.compute(model, pos, types, box)
    _check_all(g, U, F, Wv, n)
    vel = W.maxwell_boltzmann(model.mass[types], 300.0, seed)
    nep.md_init(h.h, p, t, box, torch.tensor(vel, device="cuda"))
    th = torch.zeros((10, 4), dtype=torch.float64, device="cuda")
    nep.md_run(h.h, 10, 1.0, 1, th)
    torch.cuda.synchronize()
    h.close()
    _, _, th_ref, _ = oracle.md(model, pos, vel, types, box, 10, 1.0)
    assert np.abs(th.cpu().numpy()[:, 0] - th_ref[1:, 0]).max() / n <= 1e-6


def test_host_md_entry_points_match_device(torch_cuda):
    """md_init_host / md_get_state_host (host arrays, page-locked or not) give the device
    entry points' trajectory bit for bit, twice in a row on one handle."""
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    w = W.si_diamond(3, seed=0)
    h = nep.NEP(w.model)
    nep.md_init(h.h, torch.tensor(w.pos, device="cuda"), torch.tensor(w.types, device="cuda"), w.box,
                torch.tensor(w.vel, device="cuda"))
    nep.md_run(h.h, 12, 1.0, 1, None)
    ref = [torch.zeros((w.n_atoms, 3), dtype=torch.float64, device="cuda") for _ in range(3)]
    nep.md_get_state(h.h, *ref)
    torch.cuda.synchronize()
    ref = [r.cpu().numpy() for r in ref]
    for pinned in (False, True):
        if pinned:
            pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory().numpy()
            pos, types, vel = pin(w.pos, np.float64), pin(w.types, np.int32), pin(w.vel, np.float64)
            outs = [torch.empty((w.n_atoms, 3), dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
        else:
            pos, types, vel, outs = w.pos, w.types, w.vel, [None, None, None]
        nep.md_init_host(h.h, pos, types, w.box, vel)
        nep.md_run(h.h, 12, 1.0, 1, None)
        torch.cuda.synchronize()
        got = nep.md_get_state_host(h.h, w.n_atoms, *outs)
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a, b)
    h.close()
