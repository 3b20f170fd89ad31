"""Population evaluation (nep_eval_population) against the oracle's Eq. loss.

Targets are FP64 oracle labels of one model (seed 0); the population holds that model
itself (zero energy, force and virial error up to FP32 rounding) and random models. For each
member the GPU loss terms are compared with ``oracle.eq_loss`` of the oracle's predictions
for the same parameters: RMSE terms within 1e-5 relative (plus 1e-6 absolute, the FP32
error of the predictions), regularisers within 1e-12 relative (FP64, same values).
The BF16 form is held to the force bar of the precision form: its force RMSE term moves by
at most 1 meV/A.
"""
import numpy as np
import pytest

import oracle
from paper_2205_10046_gb300 import workloads as W

pytestmark = pytest.mark.gpu

LAMBDAS = (1.0, 1.0, 0.5, 1e-3, 2e-3)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_10046_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def problem():
    label = W.mixed_model(0)
    b = W.batch_structures(10, seed=21, n_max=48)
    e_t, f_t, w_t = oracle.batch_predictions(label, b.offsets, b.pos, b.types, b.boxes)
    members = [label] + [W.mixed_model(100 + p) for p in range(5)]
    z = np.stack([m.to_vector() for m in members])
    ref = []
    for m in members:
        e, f, w = oracle.batch_predictions(m, b.offsets, b.pos, b.types, b.boxes)
        ref.append(oracle.eq_loss(e, e_t, f, f_t, m.to_vector(), LAMBDAS, w, w_t))
    return dict(label=label, b=b, e_t=e_t, f_t=f_t, w_t=w_t, z=z, ref=np.array(ref))


def _eval(torch, p, precision=0, members=0, with_virial=True):
    from paper_2205_10046_gb300 import nep
    h = nep.NEP(p["label"], precision=precision)
    nep.nep_set_tuning(h.h, members)
    b = p["b"]
    dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
    loss = nep.nep_eval_population(h.h, dev(p["z"]), b.offsets, dev(b.pos), dev(b.types, torch.int32), b.boxes,
                                   dev(p["e_t"]), dev(p["f_t"]), dev(p["w_t"]) if with_virial else None, LAMBDAS)
    torch.cuda.synchronize()
    out = loss.cpu().numpy()
    tune = nep.nep_get_tuning(h.h)
    h.close()
    return out, tune


def test_population_loss_matches_oracle(torch_cuda, problem):
    g, _ = _eval(torch_cuda, problem)
    ref = problem["ref"]
    # the label model itself: only rounding remains
    assert g[0, 1] < 1e-6 and g[0, 2] < 1e-5 and g[0, 3] < 1e-5, g[0]
    for c in (1, 2, 3):
        np.testing.assert_allclose(g[:, c], ref[:, c], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(g[:, 4:], ref[:, 4:], rtol=1e-12, atol=0)
    np.testing.assert_allclose(g[:, 0], ref[:, 0], rtol=1e-5, atol=3e-6)


def test_population_without_virial_targets(torch_cuda, problem):
    g, _ = _eval(torch_cuda, problem, with_virial=False)
    ref = problem["ref"]
    assert np.all(g[:, 3] == 0.0)
    lam = LAMBDAS
    expect = lam[0] * ref[:, 1] + lam[1] * ref[:, 2] + lam[3] * ref[:, 4] + lam[4] * ref[:, 5]
    np.testing.assert_allclose(g[:, 0], expect, rtol=1e-5, atol=3e-6)


def test_population_grouping_does_not_change_the_losses(torch_cuda, problem):
    full, t_full = _eval(torch_cuda, problem, members=0)
    assert t_full["last_members"] == problem["z"].shape[0]
    for m in (1, 4):
        g, t = _eval(torch_cuda, problem, members=m)
        assert t["last_members"] == m
        np.testing.assert_array_equal(g, full)


def test_population_bf16_form(torch_cuda, problem):
    g, _ = _eval(torch_cuda, problem, precision=1)
    ref = problem["ref"]
    assert np.all(np.abs(g[:, 2] - ref[:, 2]) <= 1e-3), (g[:, 2], ref[:, 2])
    assert np.all(np.abs(g[:, 1] - ref[:, 1]) <= 2e-3)
    np.testing.assert_allclose(g[:, 4:], ref[:, 4:], rtol=1e-12, atol=0)
    # BF16 members in groups give the same values as one at a time
    g1, _ = _eval(torch_cuda, problem, precision=1, members=1)
    np.testing.assert_array_equal(g1, g)


def test_population_autotuned_shapes(torch_cuda, problem):
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    base, _ = _eval(torch, problem)
    h = nep.NEP(problem["label"])
    b = problem["b"]
    dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
    p, t = dev(b.pos), dev(b.types, torch.int32)
    P = problem["z"].shape[0]
    tune = nep.nep_autotune(h.h, b.offsets, p, t, b.boxes, n_pop=P)
    # gather CTA shapes (the default low-register form keeps 128-atom CTAs), then members
    assert tune["members_per_launch"] in (1, 2, 4) and tune["n_tried"] >= 5
    loss = nep.nep_eval_population(h.h, dev(problem["z"]), b.offsets, p, t, b.boxes, dev(problem["e_t"]),
                                   dev(problem["f_t"]), dev(problem["w_t"]), LAMBDAS).cpu().numpy()
    assert nep.nep_get_tuning(h.h)["last_members"] == tune["members_per_launch"]
    # the force term's block sums follow the gather CTA size: equal up to FP64 summation order
    np.testing.assert_allclose(loss, base, rtol=1e-12, atol=1e-15)
    h.close()


def test_population_16_members_on_64_structures(torch_cuda):
    """A larger sampled case: 16 candidates (the label model and 15 random ones) on 64
    structures of 8-40 atoms, every loss term against the oracle's Eq. loss, in all three
    network forms (the tensor-core forms at their force bars)."""
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    label = W.mixed_model(0)
    b = W.batch_structures(64, seed=33, n_max=40)
    e_t, f_t, w_t = oracle.batch_predictions(label, b.offsets, b.pos, b.types, b.boxes)
    members = [label] + [W.mixed_model(200 + p) for p in range(15)]
    z = np.stack([m.to_vector() for m in members])
    ref = []
    for m in members:
        e, f, w = oracle.batch_predictions(m, b.offsets, b.pos, b.types, b.boxes)
        ref.append(oracle.eq_loss(e, e_t, f, f_t, m.to_vector(), LAMBDAS, w, w_t))
    ref = np.array(ref)
    dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
    for prec in (0, 1, 2):
        h = nep.NEP(label, precision=prec)
        g = nep.nep_eval_population(h.h, dev(z), b.offsets, dev(b.pos), dev(b.types, torch.int32), b.boxes,
                                    dev(e_t), dev(f_t), dev(w_t), LAMBDAS).cpu().numpy()
        h.close()
        np.testing.assert_allclose(g[:, 4:], ref[:, 4:], rtol=1e-12, atol=0)
        if prec == 1:
            assert np.all(np.abs(g[:, 2] - ref[:, 2]) <= 1e-3)
            continue
        for c in (1, 2, 3):
            np.testing.assert_allclose(g[:, c], ref[:, c], rtol=1e-5 if prec == 0 else 1e-4, atol=1e-6)
