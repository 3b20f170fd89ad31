"""Heat current (Eqs. Ji, J-1) and the Bussi-Donadio-Parrinello thermostat on the GPU against
the oracle.

Per-atom heat currents within relative RMS 1e-5 of the oracle's W_i . v_i; over 10 NVE steps
the total heat current of every step within 1e-5 relative; over 40 thermostatted steps with
the same random numbers, positions within 1e-5 A, velocities within 1e-6 A/fs and kinetic
energies within 1e-6 relative of the oracle's velocity Verlet + BDP.
"""
import numpy as np
import pytest

import oracle
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


def _min_image(d, box):
    f = d @ np.linalg.inv(box)
    f -= np.round(f)
    return f @ box


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_per_atom_heat_current(torch_cuda):
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    m = W.mixed_model(0)
    pos, types, box = W.random_structure(61, 150)
    v = W.maxwell_boltzmann(m.mass[types], 600.0, 4)
    J_ref, Jt_ref = oracle.heat_current(m, pos, types, box, v)
    h = nep.NEP(m)
    dev = lambda a: torch.tensor(a, device="cuda")
    J = torch.empty((150, 3), dtype=torch.float64, device="cuda")
    Jt = torch.empty(3, dtype=torch.float64, device="cuda")
    nep.nep_heat_current(h.h, dev(pos), dev(types), box, dev(v), J, Jt)
    torch.cuda.synchronize()
    assert _rel(J.cpu().numpy(), J_ref) <= 1e-5
    assert _rel(Jt.cpu().numpy(), Jt_ref) <= 1e-5
    h.close()


def test_heat_current_along_nve(torch_cuda):
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    m = W.mixed_model(0)
    pos, types, box = W.random_structure(62, 96)
    v = W.maxwell_boltzmann(m.mass[types], 300.0, 5)
    _, _, th_ref, J_ref = oracle.md_bdp(m, pos, v, types, box, 10, 1.0, 0.0, 100.0, None)
    h = nep.NEP(m)
    dev = lambda a: torch.tensor(a, device="cuda")
    nep.md_init(h.h, dev(pos), dev(types), box, dev(v))
    th = torch.zeros((10, 4), dtype=torch.float64, device="cuda")
    J = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    nep.md_run_ex(h.h, 10, 1.0, 1, th, J)
    torch.cuda.synchronize()
    Jg = J.cpu().numpy()
    for k in range(10):
        assert _rel(Jg[k], J_ref[k]) <= 1e-5, (k, Jg[k], J_ref[k])
    assert np.abs(th.cpu().numpy()[:, 0] - th_ref[:, 0]).max() / 96 <= 1e-6
    h.close()


def test_bdp_thermostat_follows_the_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    m = W.mixed_model(0)
    pos, types, box = W.random_structure(63, 80)
    n = pos.shape[0]
    v = W.maxwell_boltzmann(m.mass[types], 100.0, 6)
    rng = np.random.default_rng(8)
    steps, T0, tau = 40, 600.0, 20.0
    rand = np.stack([rng.normal(size=steps), rng.chisquare(3 * n - 4, size=steps)], axis=1)
    x_ref, v_ref, th_ref, J_ref = oracle.md_bdp(m, pos, v, types, box, steps, 1.0, T0, tau, rand)
    h = nep.NEP(m)
    dev = lambda a: torch.tensor(a, device="cuda")
    nep.md_init(h.h, dev(pos), dev(types), box, dev(v))
    th = torch.zeros((steps, 4), dtype=torch.float64, device="cuda")
    J = torch.zeros((steps, 3), dtype=torch.float64, device="cuda")
    nep.md_run_ex(h.h, steps, 1.0, 1, th, J, temperature=T0, tau_fs=tau, bdp_random=dev(rand))
    p = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    vv = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    nep.md_get_state(h.h, pos=p, vel=vv)
    torch.cuda.synchronize()
    thg = th.cpu().numpy()
    np.testing.assert_allclose(thg[:, 1], th_ref[:, 1], rtol=1e-6)
    np.testing.assert_allclose(thg[:, 2], th_ref[:, 2], rtol=1e-6)
    assert np.abs(_min_image(p.cpu().numpy() - x_ref, box)).max() <= 1e-5
    assert np.abs(vv.cpu().numpy() - v_ref).max() <= 1e-6
    for k in range(steps):
        assert _rel(J.cpu().numpy()[k], J_ref[k]) <= 1e-5
    # the thermostat heated the system towards T0 from 100 K
    assert thg[-1, 2] > 200.0
    # a later plain md_run on the same state is NVE again (no rescaling)
    th2 = torch.zeros((5, 4), dtype=torch.float64, device="cuda")
    nep.md_run(h.h, 5, 1.0, 1, th2)
    torch.cuda.synchronize()
    e = th2.cpu().numpy()
    assert np.abs((e[:, 0] + e[:, 1]) - (e[0, 0] + e[0, 1])).max() / n < 1e-4
    h.close()
