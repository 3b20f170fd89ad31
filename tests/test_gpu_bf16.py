"""The precision form: descriptor -> hidden and hidden -> dU/dq as BF16 tensor-core GEMMs
(tcgen05, FP32 accumulation in tensor memory), everything else as in the FP32 path.

Bar: force RMSE against the FP64 oracle <= 1 meV/A; the energy and virial errors are checked
against bounds derived from BF16 rounding (relative 2^-9 per operand) and printed.
"""
import numpy as np
import pytest

import oracle
from paper_2205_10046_gb300 import workloads as W

pytestmark = pytest.mark.gpu

F_RMSE = 1e-3  # eV/A


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_10046_gb300 import build
    build.build()
    return torch


def _run(torch, model, pos, types, box, precision):
    from paper_2205_10046_gb300 import nep
    h = nep.NEP(model, precision=precision)
    out = h.compute(torch.tensor(pos, device="cuda"), torch.tensor(types, device="cuda"), box, per_atom_virial=True)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    h.close()
    return res


CASES = {
    "si216": lambda: W.si_diamond(3, seed=0, with_velocities=False),
    "pbte512": lambda: W.pbte_rocksalt(4, seed=1, with_velocities=False),
    "mixed150": lambda: None,
}


@pytest.mark.parametrize("name", list(CASES))
def test_bf16_network_force_error_below_1_mev_per_angstrom(torch_cuda, name):
    w = CASES[name]()
    if w is None:
        pos, types, box = W.random_structure(5, 150)
        model = W.random_model(W.MIXED_MODEL, 5, [W.MASS_SI, W.MASS_GE, W.MASS_C])
    else:
        pos, types, box, model = w.pos, w.types, w.box, w.model
    n = pos.shape[0]
    U, F, Wv = oracle.compute(model, pos, types, box)
    g = _run(torch_cuda, model, pos, types, box, 1)
    f_rmse = float(np.sqrt(np.mean((g["F"] - F) ** 2)))
    e_err = abs(g["E"][0] - U.sum()) / n
    w_err = float(np.abs(g["W_total"] - Wv.sum(0)).max() / n)
    print(f"{name}: BF16 force RMSE {f_rmse:.2e} eV/A (|F| rms {np.sqrt(np.mean(F**2)):.2e}), "
          f"|dE|/N {e_err:.2e} eV, |dW|/N {w_err:.2e} eV")
    assert f_rmse <= F_RMSE
    assert e_err <= 2e-3 and w_err <= 2e-3
    # the tensor-core form is not the FP32 form
    g32 = _run(torch_cuda, model, pos, types, box, 0)
    assert not np.array_equal(g["F"], g32["F"])


def test_bf16_network_md_conserves_energy(torch_cuda):
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    w = W.pbte_rocksalt(4, seed=1)
    h = nep.NEP(w.model, precision=1)
    nep.md_init(h.h, torch.tensor(w.pos, device="cuda"), torch.tensor(w.types, device="cuda"), w.box,
                torch.tensor(w.vel, device="cuda"))
    th = torch.zeros((100, 4), dtype=torch.float64, device="cuda")
    nep.md_run(h.h, 100, 2.0, 1, th)
    torch.cuda.synchronize()
    e = th.cpu().numpy()
    etot = e[:, 0] + e[:, 1]
    assert np.all(np.isfinite(e))
    # the BF16 network is a slightly different (but smooth) potential: energy stays conserved
    assert np.ptp(etot) / w.n_atoms < 1e-4, np.ptp(etot) / w.n_atoms
    h.close()
