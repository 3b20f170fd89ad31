"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks one part of the oracle against an independent route: crystallographic
neighbour shells, a minimum-image search written here, numpy's Chebyshev series, the
Legendre double sum of Eq. qinl_legendre, scipy's spherical harmonics (Eqs.
qinl_spherical, Ainlm), the generic Wigner-3j forms of Eqs. q_4body and q_5body (sympy),
finite differences of the total energy (Eqs. F_ij, F_i), the strain derivative of the
energy (Eq. virial), symmetry invariances (Sec. II B) and properties of velocity Verlet.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2205_10046_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _shells():
    rows = []
    with open(os.path.join(GOLDEN, "neighbor_shells.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, a, rc, n = line.split()
                rows.append((k, float(a), float(rc), int(n)))
    return rows


def _model(hyper_over=None, seed=7, T=None, mass=None):
    h = dict(W.MIXED_MODEL)
    h.update(dict(n_max_radial=4, basis_radial=5, n_max_angular=3, basis_angular=4, n_neuron=6))
    if hyper_over:
        h.update(hyper_over)
    if T is not None:
        h["n_types"] = T
    return W.random_model(h, seed, mass if mass is not None else np.linspace(10.0, 30.0, h["n_types"]))


# ----------------------------------------------------------------------------- neighbours
@pytest.mark.parametrize("kind,a,rc,expect", _shells())
def test_shell_counts_multi_image(kind, a, rc, expect):
    """A 2x2x2 supercell is thinner than 2 rc, so many periodic images of each atom lie
    inside the cutoff; every atom must still see exactly the crystallographic count."""
    pos, box, _ = W.lattice(kind, a, (2, 2, 2))
    counts = oracle.neighbor_counts(pos, box, rc)
    assert set(counts.tolist()) == {expect}


def test_triclinic_descriptions_of_one_lattice():
    """The diamond lattice described by its 2-atom primitive (triclinic) cell, by a heavily
    skewed but equivalent cell, and by a conventional supercell gives identical counts."""
    a = 5.43
    prim = np.array([[0, .5, .5], [.5, 0, .5], [.5, .5, 0]]) * a
    skew = np.array([prim[0], prim[1], prim[0] + prim[1] + prim[2]])
    basis = np.array([[0, 0, 0], [.25, .25, .25]]) * a
    conv_pos, conv_box, _ = W.lattice("diamond", a, (3, 3, 3))
    for rc in (4.0, 5.0, 5.5, 6.0):
        c_prim = oracle.neighbor_counts(basis, prim, rc)
        c_skew = oracle.neighbor_counts(basis, skew, rc)
        c_conv = oracle.neighbor_counts(conv_pos, conv_box, rc)
        assert len(set(c_conv.tolist())) == 1
        assert set(c_prim.tolist()) == set(c_skew.tolist()) == set(c_conv.tolist())


def test_neighbors_match_minimum_image_in_large_box():
    """With every face distance above 2 rc, the all-image search reduces to minimum image."""
    rng = np.random.default_rng(11)
    L = 15.0
    pos = rng.uniform(0, L, (40, 3))
    box = np.eye(3) * L
    rc = 5.0
    for i in (0, 7, 39):
        j, n, d = oracle.neighbors(pos, box, rc, i)
        dd = pos - pos[i]
        dd -= L * np.round(dd / L)
        r = np.linalg.norm(dd, axis=1)
        want = sorted((int(k), tuple(np.round(dd[k], 9))) for k in np.nonzero((r < rc) & (np.arange(40) != i))[0])
        got = sorted((int(jj), tuple(np.round(x, 9))) for jj, x in zip(j, d))
        assert got == want


# ----------------------------------------------------------------------------- radial
def _f_numpy(r, rc, K):
    """f_k(r) of Eq. f_n via numpy's Chebyshev series and the cosine cutoff."""
    x = 2.0 * (r / rc - 1.0) ** 2 - 1.0
    fc = 0.5 * (1.0 + math.cos(math.pi * r / rc)) if r < rc else 0.0
    return np.array([0.5 * (np.polynomial.chebyshev.chebval(x, np.eye(K + 1)[k]) + 1.0) * fc
                     for k in range(K + 1)])


def test_radial_basis_is_chebyshev_times_cutoff():
    rng = np.random.default_rng(3)
    for rc, K in ((5.0, 8), (6.0, 10), (4.0, 12)):
        for r in rng.uniform(0.3, rc, 12):
            np.testing.assert_allclose(oracle.radial_basis(rc, K, r), _f_numpy(r, rc, K), rtol=1e-12, atol=1e-14)
        # T_k(x) = cos(k arccos x) and the cutoff makes every f_k vanish at rc
        assert np.all(np.abs(oracle.radial_basis(rc, K, rc * (1 - 1e-7))) < 1e-12)
        assert np.all(oracle.radial_basis(rc, K, rc) == 0.0)
        r = 0.37 * rc
        x = 2.0 * (r / rc - 1.0) ** 2 - 1.0
        fc = 0.5 * (1.0 + math.cos(math.pi * r / rc))
        tk = np.array([math.cos(k * math.acos(x)) for k in range(K + 1)])
        np.testing.assert_allclose(oracle.radial_basis(rc, K, r), 0.5 * (tk + 1.0) * fc, rtol=1e-12)


def test_radial_descriptor_dimer_uses_ordered_type_pair():
    """Two atoms of different types: q_n of atom i is sum_k c^{t_i t_j}_{nk} f_k(r) (Eqs. qin,
    g_n); atom j uses the transposed type pair, which differs for random weights."""
    m = _model(T=2, seed=21)
    nR = m.n_max_radial
    rng = np.random.default_rng(2)
    for r in (2.2, 3.9, 5.3):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        pos = np.array([[20.0, 20.0, 20.0], 20.0 + r * u])
        types = np.array([0, 1], np.int32)
        q = oracle.descriptors(m, pos, types, np.eye(3) * 40.0)
        f = _f_numpy(r, m.rc_radial, m.basis_radial)
        np.testing.assert_allclose(q[0, :nR + 1], m.c_radial[0, 1] @ f, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(q[1, :nR + 1], m.c_radial[1, 0] @ f, rtol=1e-12, atol=1e-14)
        assert not np.allclose(q[0, :nR + 1], q[1, :nR + 1])
        if r >= m.rc_angular:
            assert np.all(q[:, nR + 1:] == 0.0)


# ----------------------------------------------------------------------------- angular
def _cluster(seed, n_nb=7, T=2):
    """A central atom with n_nb neighbours inside r_c^A, alone in a large box, and a model
    whose angular radial functions equal its radial ones (so dimers give g^A_n)."""
    rng = np.random.default_rng(seed)
    m = _model(dict(rc_radial=4.0, rc_angular=4.0, n_max_radial=3, n_max_angular=3,
                    basis_radial=4, basis_angular=4), seed=seed, T=T)
    m.c_angular = m.c_radial.copy()
    d = rng.normal(size=(n_nb, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    d *= rng.uniform(1.2, 3.9, (n_nb, 1))
    pos = np.vstack([[0, 0, 0], d]) + 30.0
    box = np.eye(3) * 80.0
    types = rng.integers(0, T, n_nb + 1).astype(np.int32)
    q = oracle.descriptors(m, pos, types, box, sel=[0])[0]
    G = []
    for k in range(n_nb):  # g^{t_0 t_j}_n(r_j) from a dimer of the same two types
        dim = np.array([[30.0, 30.0, 30.0], [30.0 + np.linalg.norm(d[k]), 30.0, 30.0]])
        G.append(oracle.descriptors(m, dim, np.array([types[0], types[k + 1]], np.int32), box, sel=[0])[0][:4])
    G = np.array(G)
    r = np.linalg.norm(d, axis=1)
    u = d / r[:, None]
    return m, q, G, u


def _A(G, u, n, l, mm):
    """A_nlm of Eq. Ainlm with scipy's complex spherical harmonics."""
    from scipy.special import sph_harm_y
    th = np.arccos(np.clip(u[:, 2], -1, 1))
    ph = np.arctan2(u[:, 1], u[:, 0])
    return np.sum(G[:, n] * sph_harm_y(l, mm, th, ph))


def test_three_body_equals_legendre_and_spherical_harmonic_forms():
    """q_nl (l = 1..4) built from S_nk and C3b equals the Legendre double sum of Eq.
    qinl_legendre and the spherical-harmonic sum of Eq. qinl_spherical."""
    from scipy.special import eval_legendre
    for seed in (1, 2):
        m, q, G, u = _cluster(seed)
        nA, off = 3, 4
        for l in range(1, 5):
            for n in range(nA + 1):
                cos_t = u @ u.T
                leg = (2 * l + 1) / (4 * math.pi) * np.sum(np.outer(G[:, n], G[:, n]) * eval_legendre(l, cos_t))
                sph = sum((-1) ** mm * _A(G, u, n, l, mm) * _A(G, u, n, l, -mm) for mm in range(-l, l + 1))
                got = q[off + (l - 1) * (nA + 1) + n]
                assert got == pytest.approx(leg, rel=1e-11, abs=1e-14)
                assert got == pytest.approx(sph.real, rel=1e-11, abs=1e-14)


def _w3j(*a):
    from sympy.physics.wigner import wigner_3j
    return float(wigner_3j(*a))


def test_four_body_equals_wigner_3j_contraction():
    """q_n222 from C4b equals the generic Eq. q_4body with l1 = l2 = l3 = 2, and the same
    generic form vanishes for l = 1 and l = 3 (the paper's q_n111 = q_n333 = 0)."""
    m, q, G, u = _cluster(4)
    nA, off = 3, 4 + 4 * 4

    def generic(n, l):
        s = 0.0
        for m1 in range(-l, l + 1):
            for m2 in range(-l, l + 1):
                m3 = -m1 - m2
                if abs(m3) <= l:
                    s += _w3j(l, l, l, m1, m2, m3) * _A(G, u, n, l, m1) * _A(G, u, n, l, m2) * _A(G, u, n, l, m3)
        return s

    for n in range(nA + 1):
        g2 = generic(n, 2)
        assert abs(g2.imag) < 1e-13
        assert q[off + n] == pytest.approx(g2.real, rel=1e-10, abs=1e-15)
        assert abs(generic(n, 1)) < 1e-13 and abs(generic(n, 3)) < 1e-13


def test_five_body_equals_generalised_coupling():
    """q_n1111 from C5b equals Eq. q_5body with the coupling symbol of the paper (sum over
    L, M of two 3j symbols), and equals (7/15) q_n1^2."""
    m, q, G, u = _cluster(5)
    nA, off5, off1 = 3, 4 + 5 * 4, 4
    coup = {}
    for m1 in (-1, 0, 1):
        for m2 in (-1, 0, 1):
            for m3 in (-1, 0, 1):
                for m4 in (-1, 0, 1):
                    c = 0.0
                    for L in range(0, 3):
                        for M in range(-L, L + 1):
                            c += (-1) ** M * _w3j(L, 1, 1, -M, m1, m2) * _w3j(L, 1, 1, M, m3, m4)
                    coup[(m1, m2, m3, m4)] = c
    for n in range(nA + 1):
        A = {mm: _A(G, u, n, 1, mm) for mm in (-1, 0, 1)}
        s = sum(c * A[a] * A[b] * A[cc] * A[d] for (a, b, cc, d), c in coup.items())
        assert q[off5 + n] == pytest.approx(s.real, rel=1e-10, abs=1e-16)
        assert q[off5 + n] == pytest.approx(7.0 / 15.0 * q[off1 + n] ** 2, rel=1e-12, abs=1e-16)


def test_descriptor_length_and_parameter_count():
    """N_des = (n_R+1) + (n_A+1)(l_max^3b + 2) and N_par of NEP3 (Sec. II D, II E)."""
    m = W.random_model(W.SI_MODEL, 0, [W.MASS_SI])
    assert m.n_des == 9 + 5 * 6 == oracle.n_des(m)
    assert m.n_par == (39 + 2) * 50 + 1 + 81 + 25 == m.to_vector().size
    m = W.random_model(W.PBTE_MODEL, 1, [W.MASS_PB, W.MASS_TE])
    assert m.n_des == 11 + 7 * 6 == oracle.n_des(m)
    assert m.n_par == (53 + 2) * 30 + 1 + 4 * 121 + 4 * 49 == m.to_vector().size


# ----------------------------------------------------------------------------- network
def test_network_orientation_with_one_hot_rows():
    """With w0 rows one-hot (neuron mu reads component p(mu) with weight s_mu), Eq. Ui reduces
    to sum_mu w1_mu tanh(s_mu q_p(mu) - b0_mu) - b1: a transposed w0 would read other q's."""
    m = _model(seed=9)
    D, H = m.n_des, m.n_neuron
    rng = np.random.default_rng(1)
    pick = rng.permutation(D)[:H]
    s = rng.uniform(0.5, 2.0, H)
    m.w0 = np.zeros((H, D))
    m.w0[np.arange(H), pick] = s
    q = rng.normal(size=D)
    want = float(np.sum(m.w1 * np.tanh(s * q[pick] - m.b0)) - m.b1)
    assert oracle.site_energy(m, q) == pytest.approx(want, rel=1e-14, abs=1e-15)
    # zero descriptor: every neuron sees only its bias
    assert oracle.site_energy(m, np.zeros(D)) == pytest.approx(float(np.sum(m.w1 * np.tanh(-m.b0)) - m.b1), rel=1e-14)


# ----------------------------------------------------------------------------- forces, virial
def _small_triclinic(seed=3, n=14, T=3):
    pos, types, box = W.random_structure(seed, n, n_types_model=T)
    m = W.random_model(W.MIXED_MODEL, seed, [W.MASS_SI, W.MASS_GE, W.MASS_C])
    return m, pos, types, box


def test_forces_are_minus_energy_gradient():
    """F_i (Eqs. F_ij, F_i from the partial forces) equals -dE/dr_i by central differences,
    on a small sheared multi-species cell where many periodic images are neighbours."""
    m, pos, types, box = _small_triclinic()
    _, F, _ = oracle.compute(m, pos, types, box)
    h = 1e-5
    for i in (0, 5, 13):
        for c in range(3):
            p = pos.copy()
            p[i, c] += h
            ep = oracle.energy(m, p, types, box)
            p[i, c] -= 2 * h
            em = oracle.energy(m, p, types, box)
            assert F[i, c] == pytest.approx(-(ep - em) / (2 * h), rel=2e-6, abs=2e-9)


def test_newton_third_law_total_force_vanishes():
    for m, pos, types, box in (_small_triclinic(5), ):
        _, F, _ = oracle.compute(m, pos, types, box)
        assert np.abs(F.sum(0)).max() < 1e-12 * max(1.0, np.abs(F).max() * len(F))
    w = W.si_diamond(2, with_velocities=False)
    _, F, _ = oracle.compute(w.model, w.pos, w.types, w.box)
    assert np.abs(F.sum(0)).max() < 1e-13


def test_rotation_translation_permutation_invariance():
    m, pos, types, box = _small_triclinic(7)
    U, F, Wv = oracle.compute(m, pos, types, box)
    E = U.sum()
    # rotation of positions and cell rows together
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    U2, F2, _ = oracle.compute(m, pos @ Q, types, box @ Q)
    assert U2.sum() == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(F2, F @ Q, atol=1e-12)
    # translation
    U3, F3, _ = oracle.compute(m, pos + np.array([0.37, -1.2, 2.9]), types, box)
    assert U3.sum() == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(F3, F, atol=1e-12)
    # permutation of atoms (types move with them)
    perm = rng.permutation(len(pos))
    U4, F4, _ = oracle.compute(m, pos[perm], types[perm], box)
    np.testing.assert_allclose(U4, U[perm], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(F4, F[perm], atol=1e-12)


def test_virial_equals_strain_derivative():
    """Sum_i W_i (Eq. virial, r_ij = r_j - r_i) equals -(dE/d eps)^T for the affine strain
    r -> (I + eps) r applied to positions and cell together."""
    m, pos, types, box = _small_triclinic(9, n=12)
    _, _, Wv = oracle.compute(m, pos, types, box)
    ordr = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2), (1, 0), (2, 0), (2, 1)]
    Wt = np.zeros((3, 3))
    for c, (a, b) in enumerate(ordr):
        Wt[a, b] = Wv[:, c].sum()
    h = 1e-6
    dE = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            es = []
            for sgn in (1, -1):
                eps = np.zeros((3, 3))
                eps[a, b] = sgn * h
                T = np.eye(3) + eps  # column-vector map r -> T r, i.e. rows r -> r T^T
                es.append(oracle.energy(m, pos @ T.T, types, box @ T.T))
            dE[a, b] = (es[0] - es[1]) / (2 * h)
    np.testing.assert_allclose(Wt, -dE.T, rtol=2e-6, atol=2e-8)
    # the total is symmetric up to rounding
    np.testing.assert_allclose(Wt, Wt.T, atol=1e-10)


def test_isolated_atom_and_empty_system():
    m = _model(seed=3)
    pos = np.array([[5.0, 5.0, 5.0]])
    U, F, Wv = oracle.compute(m, pos, np.array([1], np.int32), np.eye(3) * 30.0)
    assert U[0] == pytest.approx(float(np.sum(m.w1 * np.tanh(-m.b0)) - m.b1), rel=1e-14)
    assert np.all(F == 0) and np.all(Wv == 0)
    U, F, Wv = oracle.compute(m, np.zeros((0, 3)), np.zeros(0, np.int32), np.eye(3) * 30.0)
    assert U.shape == (0,) and F.shape == (0, 3)


# ----------------------------------------------------------------------------- dynamics
def test_unit_constant():
    assert W.AMU_A2_PER_FS2_IN_EV == pytest.approx(103.6427, abs=5e-5)


def test_free_flight_with_constant_energy_model():
    """w1 = 0 makes U constant, so F = 0: positions advance by v*t (modulo the cell),
    velocities and kinetic energy stay fixed, and the kinetic energy is 1/2 m v^2 in eV."""
    w = W.si_diamond(2, with_velocities=True)
    m = w.model
    m.w1 = np.zeros_like(m.w1)
    n = 5
    pos, vel, thermo, F = oracle.md(m, w.pos, w.vel, w.types, w.box, n, 1.0)
    assert np.all(F == 0)
    np.testing.assert_allclose(vel, w.vel, rtol=0, atol=0)
    L = w.box[0, 0]
    dx = pos - (w.pos + n * 1.0 * w.vel)
    assert np.abs(dx - L * np.round(dx / L)).max() < 1e-10
    ke = 0.5 * W.AMU_A2_PER_FS2_IN_EV * np.sum(w.masses()[:, None] * w.vel ** 2)
    np.testing.assert_allclose(thermo[:, 1], ke, rtol=1e-13)
    assert thermo[0, 2] == pytest.approx(300.0, rel=1e-12)


def _md_case():
    w = W.si_diamond(2, seed=0, sigma=0.15, temperature=3000.0, with_velocities=True)
    return w


def test_energy_drift_scales_as_dt_squared():
    """Velocity Verlet is second order: halving dt over the same time cuts the energy error ~4x."""
    w = _md_case()
    errs = []
    for dt, n in ((2.0, 20), (1.0, 40)):
        _, _, th, _ = oracle.md(w.model, w.pos, w.vel, w.types, w.box, n, dt)
        e = th[:, 0] + th[:, 1]
        errs.append(np.abs(e - e[0]).max())
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.3, (errs, ratio)


def test_time_reversibility():
    w = _md_case()
    n = 15
    p1, v1, _, _ = oracle.md(w.model, w.pos, w.vel, w.types, w.box, n, 1.0)
    p2, v2, _, _ = oracle.md(w.model, p1, -v1, w.types, w.box, n, 1.0)
    L = w.box[0, 0]
    dx = p2 - w.pos
    assert np.abs(dx - L * np.round(dx / L)).max() < 1e-9
    np.testing.assert_allclose(-v2, w.vel, atol=1e-11)


def test_per_atom_virial_orientation_from_site_energy_differences():
    """W_i[a][b] = sum_j (r_ij)_a (dU_j/dr_ji)_b (Eq. virial). With one image per pair (large
    box), dU_j/dr_ji = dU_j/dr_i, which central differences of the site energies U_j give
    without any partial force; this fixes the orientation of the non-symmetric per-atom W."""
    rng = np.random.default_rng(4)
    m = W.random_model(W.MIXED_MODEL, 2, [W.MASS_SI, W.MASS_GE, W.MASS_C])
    L = 14.0
    pos = rng.uniform(0, L, (30, 3))
    types = rng.integers(0, 3, 30).astype(np.int32)
    box = np.eye(3) * L
    U0, _, Wv = oracle.compute(m, pos, types, box)
    ordr = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2), (1, 0), (2, 0), (2, 1)]
    h = 1e-5
    for i in (0, 11):
        dU = np.zeros((30, 3))  # dU_j / dr_i
        for b in range(3):
            p = pos.copy()
            p[i, b] += h
            up, _, _ = oracle.compute(m, p, types, box)
            p[i, b] -= 2 * h
            um, _, _ = oracle.compute(m, p, types, box)
            dU[:, b] = (up - um) / (2 * h)
        rij = pos - pos[i]
        rij -= L * np.round(rij / L)
        r = np.linalg.norm(rij, axis=1)
        nb = (r < m.rc_radial) & (np.arange(30) != i)
        Wi = np.einsum("ja,jb->ab", rij[nb], dU[nb])
        assert np.abs(Wi - Wi.T).max() > 5e-6  # the per-atom virial is not symmetric here
        for c, (a, b) in enumerate(ordr):
            assert Wv[i, c] == pytest.approx(Wi[a, b], rel=1e-6, abs=1e-9)


def test_subcell_cluster_reproduces_the_periodic_box():
    """The cut-out used for the 8,000,000-atom workload (inner cells plus a 2 r_c halo, as an
    open cluster) gives the inner atoms exactly the energies, forces and virials they have in
    the periodic box; a halo of only r_c does not (their neighbours' environments are cut)."""
    w = W.si_diamond(8, seed=0, with_velocities=False)  # 43.4 A box, 4096 atoms
    cpos, ctypes, cbox, inner, sel = W.subcell_cluster(w, 8, 2)
    assert sel.shape[0] == 2 ** 3 * 8
    U0, F0, W0 = oracle.compute(w.model, w.pos, w.types, w.box, sel=sel)
    U1, F1, W1 = oracle.compute(w.model, cpos, ctypes, cbox, sel=inner)
    np.testing.assert_allclose(U1, U0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(F1, F0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(W1, W0, rtol=0, atol=1e-12)
    cpos2, ctypes2, cbox2, inner2, _ = W.subcell_cluster(w, 8, 2, halo=w.model.rc_radial)
    _, F2, _ = oracle.compute(w.model, cpos2, ctypes2, cbox2, sel=inner2)
    assert np.abs(F2 - F0).max() > 1e-6
