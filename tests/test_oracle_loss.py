"""Pins of the oracle's Eq. loss (Sec. III) against closed forms."""
import math

import numpy as np

import oracle
from paper_2205_10046_gb300 import workloads as W


def _targets(rng, ns=5, n=17):
    return rng.normal(size=ns), rng.normal(size=(n, 3)), rng.normal(size=(ns, 6))


def test_zero_error_leaves_only_the_regularisers():
    rng = np.random.default_rng(0)
    e, f, w = _targets(rng)
    z = np.array([3.0, -4.0])
    L, re, rf, rw, l1, l2 = oracle.eq_loss(e, e, f, f, z, (1, 1, 1, 0.5, 0.25), w, w)
    assert re == rf == rw == 0.0
    assert l1 == 3.5 and abs(l2 - math.sqrt(12.5)) < 1e-15
    assert abs(L - (0.5 * 3.5 + 0.25 * math.sqrt(12.5))) < 1e-15


def test_constant_offsets_give_their_magnitude():
    rng = np.random.default_rng(1)
    e, f, w = _targets(rng)
    z = np.ones(4)
    L, re, rf, rw, l1, l2 = oracle.eq_loss(e + 0.3, e, f + 0.2, f, z, (2.0, 3.0, 5.0, 0, 0), w - 0.1, w)
    assert abs(re - 0.3) < 1e-14 and abs(rf - 0.2) < 1e-14 and abs(rw - 0.1) < 1e-14
    assert abs(L - (2 * 0.3 + 3 * 0.2 + 5 * 0.1)) < 1e-13
    assert l1 == 1.0 and l2 == 1.0


def test_single_component_errors_are_normalised_by_their_counts():
    # one wrong force component among 3N, one wrong virial component among 6 S
    e, f, w = np.zeros(2), np.zeros((4, 3)), np.zeros((2, 6))
    f2 = f.copy()
    f2[3, 1] = 1.2
    w2 = w.copy()
    w2[1, 4] = -0.6
    _, re, rf, rw, _, _ = oracle.eq_loss(e, e, f2, f, np.ones(1), (1, 1, 1, 0, 0), w2, w)
    assert re == 0.0
    assert abs(rf - 1.2 / math.sqrt(12)) < 1e-15
    assert abs(rw - 0.6 / math.sqrt(12)) < 1e-15


def test_virial6_is_the_symmetric_part():
    a = np.arange(9, dtype=np.float64).reshape(3, 3)
    order = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2), (1, 0), (2, 0), (2, 1)]
    w9 = np.array([a[i, j] for i, j in order])
    s = 0.5 * (a + a.T)
    np.testing.assert_array_equal(oracle.virial6(w9)[0], [s[0, 0], s[1, 1], s[2, 2], s[0, 1], s[1, 2], s[2, 0]])


def test_model_vector_round_trip():
    m = W.mixed_model(3)
    z = m.to_vector()
    assert z.shape[0] == m.n_par
    m2 = m.with_vector(z)
    np.testing.assert_array_equal(m2.to_vector(), z)
    np.testing.assert_array_equal(m2.w0, m.w0)
    assert m2.b1 == m.b1


def test_batch_predictions_match_single_structures():
    m = W.mixed_model(0)
    b = W.concat_structures([W.random_structure(1, 8), (np.zeros((0, 3)), np.zeros(0, np.int32), np.eye(3) * 9),
                             W.random_structure(2, 12)])
    e, F, w = oracle.batch_predictions(m, b.offsets, b.pos, b.types, b.boxes)
    U, F2, W2 = oracle.compute(m, *b.structure(2))
    assert abs(e[2] - U.sum() / 12) < 1e-15
    np.testing.assert_array_equal(F[8:], F2)
    assert e[1] == 0.0 and np.all(w[1] == 0.0)
    np.testing.assert_allclose(w[2], oracle.virial6(W2.sum(0))[0] / 12, rtol=0, atol=1e-15)


# ----------------------------------------------------------------------------- FIRE pins
def _quadratic(k, x0):
    def f(x):
        d = x - x0
        return 0.5 * float(np.sum(k[:, None] * d * d)), -k[:, None] * d
    return f


def test_fire_reaches_the_minimum_of_a_quadratic():
    rng = np.random.default_rng(0)
    x0 = rng.normal(size=(6, 3))
    k = rng.uniform(0.5, 2.0, 6)
    start = x0 + rng.normal(0, 0.3, x0.shape)
    x, E, F, steps, energies = oracle.fire_minimize(_quadratic(k, x0), start, np.ones(6), 500, 0.1, 1e-6)
    assert np.max(np.linalg.norm(F, axis=1)) < 1e-6 and steps < 500
    np.testing.assert_allclose(x, x0, atol=1e-5)
    assert E < 1e-11


def test_fire_first_steps_follow_the_definition():
    # one particle, 1-D quadratic: the first step is plain velocity Verlet from rest, then the
    # FIRE mixing with P > 0 leaves the velocity direction (it is parallel to F)
    f = _quadratic(np.array([1.0]), np.zeros((1, 3)))
    x_start = np.array([[1.0, 0.0, 0.0]])
    x, E, F, steps, _ = oracle.fire_minimize(f, x_start, np.ones(1), 1, 0.1, 0.0)
    dt = 0.1
    v_half = 0.5 * dt * 1.0            # F(x=1) = -1 along -x
    x1 = 1.0 - dt * v_half
    assert steps == 1 and abs(x[0, 0] - x1) < 1e-15


def test_fire_overshoot_resets_velocity_and_halves_the_step():
    # worked by hand (binary fractions, exact): k = m = 1, x = 1, dt = 1.5.
    # step 1: v = -0.75, x = -0.125, F = 0.125, v = -0.65625; P < 0: v = 0, dt = 0.75.
    # step 2: v = 0.046875, x = -0.08984375, F = 0.08984375, v = 0.080566...; P > 0.
    # step 3 (alpha = 0.1, velocity parallel to F: the mixing keeps it):
    #   v = 0.0805664... + 0.375 F, x = x + 0.75 v.
    f = _quadratic(np.array([1.0]), np.zeros((1, 3)))
    x_start = np.array([[1.0, 0.0, 0.0]])
    x, _, _, steps, _ = oracle.fire_minimize(f, x_start, np.ones(1), 1, 1.5, 0.0)
    assert x[0, 0] == -0.125
    x, _, F, steps, _ = oracle.fire_minimize(f, x_start, np.ones(1), 2, 1.5, 0.0)
    assert steps == 2 and x[0, 0] == -0.08984375 and F[0, 0] == 0.08984375
    v2 = 0.046875 + 0.375 * 0.08984375
    v25 = v2 + 0.375 * 0.08984375
    x3 = -0.08984375 + 0.75 * v25
    x, _, _, _, _ = oracle.fire_minimize(f, x_start, np.ones(1), 3, 1.5, 0.0)
    assert abs(x[0, 0] - x3) < 1e-15


def test_fire_stops_on_the_starting_forces():
    f = _quadratic(np.ones(2), np.zeros((2, 3)))
    x, E, F, steps, en = oracle.fire_minimize(f, np.full((2, 3), 1e-9), np.ones(2), 10, 0.1, 1e-3)
    assert steps == 0 and en == []


# ----------------------------------------------------------------------------- heat current, BDP
def test_heat_current_forms_agree():
    """Eq. J-1 (per-atom virials contracted with each atom's own velocity) equals Eq. J-2
    (each atom's partial forces contracted with its neighbours' velocities)."""
    m = W.mixed_model(0)
    pos, types, box = W.random_structure(51, 24)
    v = np.random.default_rng(1).normal(0, 0.01, pos.shape)
    J_atoms, J1 = oracle.heat_current(m, pos, types, box, v)
    J2 = oracle.heat_current_j2(m, pos, types, box, v)
    assert np.abs(J1 - J2).max() <= 1e-10 * max(1.0, np.abs(J1).max())
    np.testing.assert_allclose(J_atoms.sum(0), J1, rtol=0, atol=1e-15)
    # J is linear in the velocities
    _, J1b = oracle.heat_current(m, pos, types, box, 2.5 * v)
    np.testing.assert_allclose(J1b, 2.5 * J1, rtol=1e-12, atol=1e-15)


def test_bdp_limits():
    # c = 1 (tau -> infinity): no rescaling
    assert oracle.bdp_alpha(3.0, 1.0, 30.0, 1.0, 0.7, 25.0) == 1.0
    # c = 0 (tau -> 0): K' = Kbar (S + R1^2) / N_f, = Kbar exactly when S + R1^2 = N_f
    K, kbar, nf = 2.0, 5.0, 30.0
    a = oracle.bdp_alpha(K, kbar, nf, 0.0, 1.0, nf - 1.0)
    assert abs(a * a * K - kbar) < 1e-14


def test_bdp_samples_the_canonical_kinetic_energy():
    """Applied alone to a kinetic energy, the BDP update leaves the canonical distribution of
    K (Gamma with shape N_f/2 and scale k_B T) stationary: mean Kbar, variance N_f (k_B T)^2 / 2."""
    rng = np.random.default_rng(7)
    nf, kT = 12.0, 0.025
    kbar = 0.5 * nf * kT
    c = np.exp(-0.1)
    K, ks = 0.3 * kbar, []
    for k in range(60000):
        R1 = rng.normal()
        S = rng.chisquare(nf - 1)
        K = oracle.bdp_alpha(K, kbar, nf, c, R1, S) ** 2 * K
        if k > 1000:
            ks.append(K)
    ks = np.array(ks)
    assert abs(ks.mean() / kbar - 1.0) < 0.03
    assert abs(ks.var() / (0.5 * nf * kT * kT) - 1.0) < 0.08


def test_md_bdp_without_thermostat_is_velocity_verlet():
    m = W.mixed_model(0)
    pos, types, box = W.random_structure(52, 16)
    v = W.maxwell_boltzmann(m.mass[types], 300.0, 3)
    x1, v1, th1, J1 = oracle.md_bdp(m, pos, v, types, box, 4, 1.0, 0.0, 100.0, None)
    x2, v2, th2, f2 = oracle.md(m, pos, v, types, box, 4, 1.0)
    d = (x1 - x2) @ np.linalg.inv(box)
    d -= np.round(d)
    assert np.abs(d @ box).max() < 1e-12 and np.abs(v1 - v2).max() < 1e-13
    np.testing.assert_allclose(th1[:, 0], th2[1:, 0], rtol=1e-12)
