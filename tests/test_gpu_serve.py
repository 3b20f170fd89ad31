"""FIRE relaxation and the serving loop (nep_server_*) against the oracle and themselves.

FIRE (fire_run) follows the oracle's FIRE step for step: the same number of steps, energies
within 1e-5 eV/atom and positions within 1e-4 A after 30 steps (FP32 forces against FP64).
Serving: each job's result does not depend on the jobs around it (alone and in a mix of 20
jobs sharing one batch: equal within the FP32 bar); single-point and NVE jobs match the oracle at the
FP32 bar; admission never reserves more than the memory budget and every job's share of the
workspace stays within its admission estimate; a bad job (a wrong type, a job larger than the
budget or than the 2^23 atoms a batch can index) is refused and the server carries on.
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


def test_fire_follows_the_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    model = W.mixed_model(0)
    pos, types, box = W.random_structure(31, 64)
    xo, Eo, Fo, steps_o, en_o = oracle.fire(model, pos, types, box, 30, 1.0, 0.05)
    h = nep.NEP(model)
    nep.md_init(h.h, torch.tensor(pos, device="cuda"), torch.tensor(types, device="cuda"), box)
    th = torch.zeros((30, 4), dtype=torch.float64, device="cuda")
    steps = nep.fire_run(h.h, 30, 1.0, 0.05, th)
    p = torch.zeros((64, 3), dtype=torch.float64, device="cuda")
    nep.md_get_state(h.h, pos=p)
    torch.cuda.synchronize()
    assert steps == steps_o
    e = th.cpu().numpy()[:steps, 0]
    assert np.abs(e - np.array(en_o)).max() / 64 <= 1e-5
    assert np.abs(_min_image(p.cpu().numpy() - xo, box)).max() <= 1e-4
    # the relaxation lowered the energy
    assert en_o[-1] < oracle.energy(model, pos, types, box)
    h.close()


def test_fire_stops_at_once_when_already_relaxed(torch_cuda):
    torch = torch_cuda
    from paper_2205_10046_gb300 import nep
    model = W.mixed_model(0)
    pos, types, box = W.random_structure(32, 40)
    h = nep.NEP(model)
    nep.md_init(h.h, torch.tensor(pos, device="cuda"), torch.tensor(types, device="cuda"), box)
    assert nep.fire_run(h.h, 10, 1.0, 1e6) == 0
    p = torch.zeros((40, 3), dtype=torch.float64, device="cuda")
    nep.md_get_state(h.h, pos=p)
    torch.cuda.synchronize()
    assert np.abs(_min_image(p.cpu().numpy() - pos, box)).max() < 1e-12
    h.close()


def _jobs(seed):
    """A mix of single-point, FIRE and NVE jobs on structures of 32-1500 atoms."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(17):
        n = int(np.exp(rng.uniform(np.log(32), np.log(1500))))
        pos, types, box = W.random_structure(1000 + 17 * seed + k, n)
        kind = int(rng.choice([0, 0, 1, 2]))
        vel = W.maxwell_boltzmann(W.mixed_model(0).mass[types], 300.0, 5000 + k) if kind == 2 else None
        out.append(dict(kind=kind, pos=pos, types=types, box=box, n_steps=int(rng.integers(5, 40)), dt_fs=1.0,
                        fmax=0.05, vel=vel))
    return out


def _targets():
    m = W.mixed_model(0)
    p1, t1, b1 = W.random_structure(41, 64)
    p2, t2, b2 = W.random_structure(42, 100)
    p3, t3, b3 = W.random_structure(43, 300)
    v2 = W.maxwell_boltzmann(m.mass[t2], 300.0, 77)
    return [dict(kind=1, pos=p1, types=t1, box=b1, n_steps=20, dt_fs=1.0, fmax=0.05, vel=None),
            dict(kind=2, pos=p2, types=t2, box=b2, n_steps=50, dt_fs=1.0, fmax=0.0, vel=v2),
            dict(kind=0, pos=p3, types=t3, box=b3, n_steps=0, dt_fs=1.0, fmax=0.0, vel=None)]


def _run(server, jobs):
    ids = [server.submit(**j) for j in jobs]
    res = {}
    while len(res) < len(ids):
        r = server.wait(120.0)
        assert r is not None, "server stalled"
        res[r["id"]] = r
    arr = {i: server.arrays(i) if res[i]["status"] == 0 else None for i in ids}
    return [(res[i], arr[i]) for i in ids]


@pytest.mark.parametrize("compact_every,min_chunk", [(0, 0), (4, 0), (4, 4)])
def test_results_are_the_same_alone_and_in_a_mix(torch_cuda, compact_every, min_chunk):
    """compact_every = 4: finished jobs stay frozen in the batch until they are a quarter of it
    (lazy leaving); min_chunk = 4: at least four iterations between two reads of the job
    states (a job finishing inside a chunk waits frozen); the results are the same."""
    from paper_2205_10046_gb300 import nep
    model = W.mixed_model(0)
    targets = _targets()
    alone = []
    for j in targets:
        s = nep.Server(model, memory_budget=8 << 30, workers=1)
        alone.append(_run(s, [j])[0])
        s.close()
    mix = _jobs(3)
    order = mix[:4] + [targets[0]] + mix[4:9] + [targets[1]] + mix[9:13] + [targets[2]] + mix[13:]
    s = nep.Server(model, memory_budget=8 << 30, workers=8, compact_every=compact_every, min_chunk=min_chunk)
    out = _run(s, order)
    st = s.stats()
    s.close()
    assert st["completed"] == len(order) and st["failed"] == 0
    pos_t = [next(k for k, o in enumerate(order) if o is t) for t in targets]
    for (ra, aa), k, t in zip(alone, pos_t, targets):
        rm, am = out[k]
        assert ra["status"] == 0 and rm["status"] == 0, (ra["message"], rm["message"])
        n = t["pos"].shape[0]
        # the neighbour lists of a job are rebuilt when any atom of the batch has moved far
        # enough, so alone and in the mix its pair sums may run in different orders: equal
        # within the FP32 bar, not bit for bit
        assert ra["steps"] == rm["steps"]
        assert abs(ra["energy"] - rm["energy"]) / n <= 1e-6
        assert np.abs(ra["virial"] - rm["virial"]).max() / n <= 1e-6
        pa, fa, va = aa
        pm, fm, vm = am
        assert np.abs(_min_image(pa - pm, t["box"])).max() <= 1e-6
        assert np.linalg.norm(fa - fm) <= 1e-5 * np.linalg.norm(fa)
        assert np.abs(va - vm).max() <= 1e-7
    # the jobs overlapped: some job started before an earlier-submitted one had finished
    starts = sorted((r["t_start"], r["t_done"]) for r, _ in out)
    assert any(starts[i + 1][0] < starts[i][1] for i in range(len(starts) - 1))


def test_server_single_point_and_nve_match_the_oracle(torch_cuda):
    from paper_2205_10046_gb300 import nep
    model = W.mixed_model(0)
    targets = _targets()
    s = nep.Server(model, memory_budget=8 << 30, workers=4)
    (r_fire, a_fire), (r_nve, a_nve), (r_sp, a_sp) = _run(s, targets)
    s.close()
    # single point
    j = targets[2]
    U, F, Wv = oracle.compute(model, j["pos"], j["types"], j["box"])
    n = j["pos"].shape[0]
    assert abs(r_sp["energy"] - U.sum()) / n <= 1e-6
    assert np.linalg.norm(a_sp[1] - F) / np.linalg.norm(F) <= 1e-5
    assert np.abs(r_sp["virial"] - Wv.sum(0)).max() / n <= 1e-6
    # NVE: 50 steps of 1 fs against the oracle's velocity Verlet
    j = targets[1]
    xo, vo, thermo, fo = oracle.md(model, j["pos"], j["vel"], j["types"], j["box"], 50, 1.0)
    assert np.abs(_min_image(a_nve[0] - xo, j["box"])).max() <= 1e-5
    assert np.abs(a_nve[2] - vo).max() <= 1e-6
    assert abs(r_nve["energy"] - thermo[-1, 0]) / j["pos"].shape[0] <= 1e-6


def test_memory_budget_admission_and_failures(torch_cuda):
    from paper_2205_10046_gb300 import nep
    model = W.mixed_model(0)
    jobs = _jobs(5)
    probe = nep.Server(model, memory_budget=64 << 30, workers=1)
    big = max(jobs, key=lambda j: j["pos"].shape[0])
    r = _run(probe, [big])[0][0]
    probe.close()
    est = r["workspace_est"]
    assert r["workspace_used"] <= est  # alone, the batch workspace is the job's
    # a budget that holds the largest job about 1.5 times: admission keeps within it
    budget = int(1.5 * est)
    s = nep.Server(model, memory_budget=budget, workers=8)
    out = _run(s, jobs)
    st = s.stats()
    assert st["peak_bytes_reserved"] <= budget
    for res, _ in out:
        assert res["status"] == 0, res["message"]
    # the batch's actual workspace never exceeded the budget
    assert st["peak_workspace_bytes"] <= budget
    # a job with a type outside the model's 3 types is refused at submission
    bad = dict(jobs[0])
    bad["types"] = np.full_like(bad["types"], 7)
    with pytest.raises(nep.NepError) as ei:
        s.submit(**bad)
    assert ei.value.code == -1
    # the server keeps serving after the failed job
    again = _run(s, [jobs[1]])[0][0]
    assert again["status"] == 0
    # a job that alone exceeds the budget is refused at submission
    huge = W.random_structure(9, 8000)
    with pytest.raises(nep.NepError) as ei:
        s.submit(0, *huge)
    assert ei.value.code == -2
    # a job above the 2^23 atoms a batch can index is refused at submission
    n_big = (1 << 23) + 1
    with pytest.raises(nep.NepError) as ei:
        s.submit(0, np.zeros((n_big, 3)), np.zeros(n_big, np.int32), np.eye(3) * 2000.0)
    assert ei.value.code == -6
    s.close()


def test_partial_builds_keep_every_job_exact(torch_cuda):
    """Hot NVE jobs of different lengths in one batch: a job whose atom moved more than skin/2
    has its own neighbour lists rebuilt while the other jobs keep their atom order and lists.
    Every job's final state equals the oracle's velocity Verlet run of that job alone."""
    from paper_2205_10046_gb300 import nep
    model = W.mixed_model(0)
    jobs = []
    for k, (n, steps) in enumerate([(40, 30), (64, 12), (100, 25), (150, 8), (200, 30), (300, 18)]):
        pos, types, box = W.random_structure(60 + k, n)
        vel = W.maxwell_boltzmann(model.mass[types], 1000.0, 900 + k)
        jobs.append(dict(kind=2, pos=pos, types=types, box=box, n_steps=steps, dt_fs=1.0, fmax=0.0, vel=vel))
    s = nep.Server(model, memory_budget=8 << 30, workers=8, skin=0.2)
    out = _run(s, jobs)
    st = s.stats()
    s.close()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["builds"] >= 1
    for (r, a), j in zip(out, jobs):
        assert r["status"] == 0, r["message"]
        xo, vo, thermo, fo = oracle.md(model, j["pos"], j["vel"], j["types"], j["box"], j["n_steps"], 1.0)
        n = j["pos"].shape[0]
        assert np.abs(_min_image(a[0] - xo, j["box"])).max() <= 1e-5
        assert np.abs(a[2] - vo).max() <= 1e-6
        assert np.linalg.norm(a[1] - fo) <= 1e-5 * np.linalg.norm(fo)
        assert abs(r["energy"] - thermo[-1, 0]) / n <= 1e-6
