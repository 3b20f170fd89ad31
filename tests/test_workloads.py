"""The seeded synthetic inputs follow the stated workload recipes: lattices, sizes, species,
displacement width, shear, velocities at the target temperature with 3N - 3 degrees of freedom,
and random weights U(-1, 1)/sqrt(fan_in) (the random draws the method consumes are inputs, made
here and handed identically to the oracle and to the CUDA path).
"""
import math

import numpy as np
import pytest

from paper_2205_10046_gb300 import workloads as W


def _kinetic_temperature(m, v):
    ke = 0.5 * W.AMU_A2_PER_FS2_IN_EV * float((m[:, None] * v * v).sum())
    return 2.0 * ke / ((3 * m.shape[0] - 3) * W.KB_EV)


def test_si_tiny_and_pbte_boxes():
    si = W.si_diamond(3, seed=0)
    assert si.n_atoms == 216 and np.allclose(si.box, np.eye(3) * 3 * 5.43)
    assert np.all(si.types == 0) and si.model.n_types == 1 and si.dt_fs == 1.0
    ideal, _, _ = W.lattice("diamond", 5.43, (3, 3, 3))
    d = si.pos - ideal
    assert abs(d.std() - 0.05) < 0.006 and abs(d.mean()) < 0.01  # sigma = 0.05 A
    pb = W.pbte_rocksalt(4, seed=1)
    assert pb.n_atoms == 512 and np.allclose(pb.box, np.eye(3) * 4 * 6.46)
    assert np.bincount(pb.types).tolist() == [256, 256] and pb.dt_fs == 2.0
    ideal, _, _ = W.lattice("rocksalt", 6.46, (4, 4, 4))
    assert abs((pb.pos - ideal).std() - 0.1) < 0.008  # sigma = 0.1 A
    # every Pb has its six Te neighbours at a/2 in the ideal rocksalt lattice
    frac = ideal / 6.46
    pb_sites, te_sites = frac[pb.types == 0], frac[pb.types == 1]
    dd = (te_sites[None, :, :] - pb_sites[:1, None, :] + 2.0) % 4.0 - 2.0
    assert np.sum(np.isclose(np.linalg.norm(dd[0], axis=1), 0.5)) == 6


def test_velocities_are_at_the_temperature_with_no_drift():
    for w in (W.si_diamond(3, seed=0), W.pbte_rocksalt(4, seed=1)):
        m = w.masses()
        assert abs(_kinetic_temperature(m, w.vel) - 300.0) < 1e-9
        assert np.abs((m[:, None] * w.vel).sum(0)).max() < 1e-12
    pos, types, box = W.random_structure(5, 100)
    v = W.maxwell_boltzmann(W.mixed_model(0).mass[types], 1000.0, 9)
    assert abs(_kinetic_temperature(W.mixed_model(0).mass[types], v) - 1000.0) < 1e-9


@pytest.mark.parametrize("hyper", [W.SI_MODEL, W.PBTE_MODEL, W.MIXED_MODEL])
def test_random_weights_are_bounded_by_one_over_sqrt_fan_in(hyper):
    m = W.random_model(hyper, 3, [1.0] * hyper["n_types"])
    D, H = m.n_des, m.n_neuron
    for arr, fan in ((m.c_radial, m.basis_radial + 1), (m.c_angular, m.basis_angular + 1),
                     (m.w0, D), (m.b0, D), (m.w1, H), (np.array([m.b1]), H)):
        bound = 1.0 / math.sqrt(fan)
        assert np.abs(arr).max() <= bound
        if arr.size >= 50:  # uniform over the whole interval, not a narrower one
            assert np.abs(arr).max() > 0.8 * bound
    assert D == (m.n_max_radial + 1) + 6 * (m.n_max_angular + 1)  # l = 1..4, 4-body, 5-body
    # one PCG64 stream: the same seed gives the same model, another seed another one
    assert np.array_equal(W.random_model(hyper, 3, [1.0] * hyper["n_types"]).w0, m.w0)
    assert not np.array_equal(W.random_model(hyper, 4, [1.0] * hyper["n_types"]).w0, m.w0)


def test_structure_batch_recipe():
    b = W.batch_structures(96, seed=3)
    sizes = np.diff(b.offsets)
    assert b.n_struct == 96 and sizes.min() >= 8 and sizes.max() <= 512
    assert np.all(b.types >= 0) and np.all(b.types < 3)
    kinds = set()
    for s in range(b.n_struct):
        pos, types, box = b.structure(s)
        assert len(set(types.tolist())) <= 3
        # +-10% off-diagonal shear of a cubic supercell: box = diag(L) (I + E), |E_ab| <= 0.1
        lengths = np.diag(box)
        e = box / lengths[:, None] - np.eye(3)
        assert np.abs(e).max() <= 0.1 + 1e-12
        # the lattice kind is the structure stream's first draw; the unsheared volume
        # (the product of the box diagonal) per atom is at least the volume per site of that
        # kind at the smallest lattice constant (0.95 a; sites >= atoms after the deletions)
        kind = int(np.random.Generator(np.random.PCG64(int(b.seeds[s]))).integers(0, 3))
        kinds.add(kind)
        a, nb = ((4.05, 4), (3.30, 2), (5.43, 8))[kind]
        assert (0.95 * a) ** 3 / nb * (1 - 1e-9) <= float(np.prod(lengths)) / pos.shape[0]
    assert kinds == {0, 1, 2}
    # structure s is random_structure(1000003 * seed + s, size): reproducible one by one
    p, t, bx = W.random_structure(int(b.seeds[7]), int(sizes[7]))
    assert np.array_equal(p, b.structure(7)[0]) and np.array_equal(bx, b.structure(7)[2])


def test_serving_pool_sizes_are_log_uniform():
    """The serving pool: 32-20,000 atoms, log-uniform (median at the geometric mean of the
    bounds, within three standard errors for 256 draws), 300 K velocities for every structure."""
    import bench
    pool = bench.serve_pool(256, 4)
    n = np.array([p[0].shape[0] for p in pool])
    assert n.min() >= 32 and n.max() <= 20000
    assert abs(np.log(np.median(n)) - 0.5 * (np.log(32) + np.log(20000))) < 0.5
    m = W.mixed_model(0).mass
    for pos, types, box, vel in pool[:8]:
        assert vel.shape == pos.shape and abs(_kinetic_temperature(m[types], vel) - 300.0) < 1e-9
