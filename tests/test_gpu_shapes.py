"""Model shapes without a compiled kernel instantiation: the run-time-shape kernels against
the FP64 oracle, through the C ABI.

Shapes: the models the paper trains in Sec. III (the MgAlCu NEP3 of Sec. III A, the two
carbon NEPs and the silicon 3-body / 3+4-body variants of Sec. III B), and a small odd shape.
Bars as for the compiled shapes: relative force RMS <= 1e-5, |dE|/N <= 1e-6 eV, total
virial / N <= 1e-6 eV, per-atom virial relative RMS <= 1e-5, descriptors relative RMS <= 1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_2205_10046_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL_F = 1e-5

# (types, rc_R, rc_A, n_R, n_A, K_R, K_A, l3b, l4b, l5b, neurons)
SHAPES = {
    # MgAlCu, Sec. III A: cutoff 6 / 3.5, n_max = basis = 12 / 8, 50 neurons, 3 types
    "mgalcu": (3, 6.0, 3.5, 12, 8, 12, 8, 4, 2, 1, 50),
    # carbon, Sec. III B: 4.2 / 3.7, n_max = basis = 10 / 8, l_max 4/2/1, 100 neurons
    "carbon_4.2": (1, 4.2, 3.7, 10, 8, 10, 8, 4, 2, 1, 100),
    # carbon, second model: 3.7 / 3.2, l_max^5b = 0, 50 neurons
    "carbon_3.7": (1, 3.7, 3.2, 10, 8, 10, 8, 4, 2, 0, 50),
    # silicon, Sec. III B: 5 / 5, n_max = basis = 10, 3-body only, 50 neurons
    "si_3body": (1, 5.0, 5.0, 10, 10, 10, 10, 4, 0, 0, 50),
    # a small odd shape: basis sizes different from n_max, l_max^3b = 2
    "odd": (2, 5.0, 4.0, 3, 2, 5, 3, 2, 0, 0, 7),
}


def _model(name, seed=7):
    T, rcR, rcA, nR, nA, KR, KA, l3, l4, l5, H = SHAPES[name]
    hyper = dict(n_types=T, rc_radial=rcR, rc_angular=rcA, n_max_radial=nR, n_max_angular=nA, basis_radial=KR,
                 basis_angular=KA, l_max_3b=l3, l_max_4b=l4, l_max_5b=l5, n_neuron=H)
    return W.random_model(hyper, seed, [W.MASS_C, W.MASS_SI, W.MASS_GE][:T] if T <= 3 else [12.0] * T)


def _structure(name):
    T = SHAPES[name][0]
    if name.startswith("carbon"):
        pos, box, _ = W.lattice("diamond", 3.567, (3, 3, 3))  # diamond carbon, 216 atoms
        return W.jitter(pos, 0.05, 11), np.zeros(pos.shape[0], np.int32), box
    if name == "si_3body":
        w = W.si_diamond(3, seed=0, with_velocities=False)
        return w.pos, w.types, w.box
    pos, types, box = W.random_structure(23, 200, n_types_model=T)
    return pos, types, box


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_10046_gb300 import build
    build.build()
    return torch


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_published_shapes_are_not_compiled():
    """These shapes run on the run-time-shape kernels, not on an instantiation."""
    pytest.importorskip("torch")
    from paper_2205_10046_gb300 import build, nep
    build.build()
    compiled = set(nep.nep_supported())
    for name, (T, rcR, rcA, nR, nA, KR, KA, l3, l4, l5, H) in SHAPES.items():
        assert (nR, KR, nA, KA, H, l3, l4, l5) not in compiled, name


@pytest.mark.parametrize("name", list(SHAPES))
def test_shape_matches_oracle(torch_cuda, name):
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    model = _model(name)
    pos, types, box = _structure(name)
    n = pos.shape[0]
    h = nep.NEP(model)
    p = torch.tensor(pos, device="cuda")
    t = torch.tensor(types, device="cuda")
    g = {k: v.cpu().numpy() for k, v in h.compute(p, t, box, per_atom_virial=True).items()}
    q = torch.zeros((n, model.n_des), dtype=torch.float64, device="cuda")
    nep.nep_descriptors(h.h, p, t, box, q)
    torch.cuda.synchronize()
    with pytest.raises(nep.NepError, match="NEP_ERR_UNSUPPORTED"):
        nep.nep_set_precision(h.h, 1)
    h.close()
    U, F, Wv = oracle.compute(model, pos, types, box)
    qr = oracle.descriptors(model, pos, types, box)
    print(f"{name}: N_des {model.n_des}, relative force RMS {_rel(g['F'], F):.2e}, "
          f"|dE|/N {abs(g['E'][0] - U.sum()) / n:.2e} eV")
    assert _rel(q.cpu().numpy(), qr) <= 1e-5
    assert _rel(g["F"], F) <= REL_F
    assert abs(g["E"][0] - U.sum()) / n <= 1e-6
    np.testing.assert_allclose(g["U"], U, rtol=0, atol=2e-5)
    assert _rel(g["W"], Wv) <= REL_F
    assert np.abs(g["W_total"] - Wv.sum(0)).max() / n <= 1e-6


def test_shape_md_matches_oracle(torch_cuda):
    """Ten NVE steps with the MgAlCu shape (rebuild inside the step graph included)."""
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    model = _model("mgalcu")
    pos, types, box = _structure("mgalcu")
    vel = W.maxwell_boltzmann(model.mass[types], 600.0, 5)
    h = nep.NEP(model, skin=0.05)
    nep.md_init(h.h, torch.tensor(pos, device="cuda"), torch.tensor(types, device="cuda"), box,
                torch.tensor(vel, device="cuda"))
    th = torch.zeros((10, 4), dtype=torch.float64, device="cuda")
    nep.md_run(h.h, 10, 1.0, 1, th)
    frc = torch.zeros((pos.shape[0], 3), dtype=torch.float64, device="cuda")
    nep.md_get_state(h.h, None, None, frc)
    torch.cuda.synchronize()
    h.close()
    _, _, th_ref, f_ref = oracle.md(model, pos, vel, types, box, 10, 1.0)
    thg = th.cpu().numpy()
    assert np.abs(thg[:, 0] - th_ref[1:, 0]).max() / pos.shape[0] <= 1e-6
    assert np.abs(thg[:, 1] - th_ref[1:, 1]).max() / pos.shape[0] <= 1e-6
    assert _rel(frc.cpu().numpy(), f_ref) < 1e-4


def test_shape_batch_and_population(torch_cuda):
    """The batched run-time-shape kernels: per-structure results and Eq. loss against the oracle."""
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    model = _model("mgalcu")
    b = W.batch_structures(5, seed=21, n_min=8, n_max=90)
    h = nep.NEP(model)
    p = torch.tensor(b.pos, device="cuda")
    t = torch.tensor(b.types, device="cuda")
    out = h.compute_batch(b.offsets, p, t, b.boxes, per_atom=True)
    torch.cuda.synchronize()
    F = out["F"].cpu().numpy()
    e_ref, F_ref, w_ref = oracle.batch_predictions(model, b.offsets, b.pos, b.types, b.boxes)
    assert _rel(F, F_ref) <= REL_F
    cnt = np.diff(b.offsets)
    np.testing.assert_allclose(out["E_struct"].cpu().numpy() / cnt, e_ref, rtol=0, atol=1e-6)
    # two candidates (the model itself and a perturbed one) against the oracle's Eq. loss
    z0 = model.to_vector()
    z = np.stack([z0, z0 + 0.01 * np.random.default_rng(3).standard_normal(z0.shape[0])])
    lam = (1.0, 1.0, 0.0, 0.05, 0.05)
    loss = torch.zeros((2, 6), dtype=torch.float64, device="cuda")
    nep.nep_eval_population(h.h, torch.tensor(z, device="cuda"), b.offsets, p, t, b.boxes,
                            torch.tensor(e_ref, device="cuda"), torch.tensor(F_ref, device="cuda"), None, lam, loss)
    torch.cuda.synchronize()
    h.close()
    lg = loss.cpu().numpy()
    for k in range(2):
        mk = model.with_vector(z[k])
        e_k, F_k, _ = oracle.batch_predictions(mk, b.offsets, b.pos, b.types, b.boxes)
        ref = oracle.eq_loss(e_k, e_ref, F_k, F_ref, z[k], lam)
        np.testing.assert_allclose(lg[k, :3], ref[:3], rtol=1e-4, atol=1e-6)
        np.testing.assert_allclose(lg[k, 4:], ref[4:], rtol=1e-12)


def test_static_descriptors_with_a_run_time_shape(torch_cuda):
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    model = _model("carbon_4.2")
    pos, types, box = _structure("carbon_4.2")
    q = torch.zeros((pos.shape[0], model.n_des), dtype=torch.float64, device="cuda")
    nep.nep_descriptors_static(model, torch.tensor(pos, device="cuda"), torch.tensor(types, device="cuda"), box, q)
    torch.cuda.synchronize()
    assert _rel(q.cpu().numpy(), oracle.descriptors(model, pos, types, box)) <= 1e-5
