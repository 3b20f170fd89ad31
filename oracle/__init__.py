"""FP64 CPU oracle for the NEP3 energy/force/virial evaluation of arXiv:2205.10046.

TEST INFRASTRUCTURE ONLY. The test-suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only code that may import this package. The CUDA
path never imports it and shares no code with it; the two meet only in the seeded
input generators of ``paper_2205_10046_gb300.workloads``.

The arithmetic lives in ``nep_oracle.cpp`` (plain FP64 C++, see its header for the
definitions it follows and the readings of the paper it takes). This module compiles it
with g++ on first use (or via :func:`build`) and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nep_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile nep_oracle.cpp into liboracle.so (portable flags: no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


class _Model(C.Structure):
    _fields_ = [("n_types", C.c_int), ("n_max_r", C.c_int), ("n_max_a", C.c_int),
                ("basis_r", C.c_int), ("basis_a", C.c_int), ("l_max_3b", C.c_int),
                ("l_max_4b", C.c_int), ("l_max_5b", C.c_int), ("n_neuron", C.c_int),
                ("rc_r", C.c_double), ("rc_a", C.c_double),
                ("c_r", C.c_void_p), ("c_a", C.c_void_p), ("w0", C.c_void_p),
                ("b0", C.c_void_p), ("w1", C.c_void_p), ("b1", C.c_double)]


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.oracle_n_des.argtypes = [C.POINTER(_Model)]
            lib.oracle_radial_basis.argtypes = [C.c_double, C.c_int, C.c_double, _dp]
            lib.oracle_radial_basis.restype = None
            lib.oracle_angular_polynomials.argtypes = [C.c_double, C.c_double, C.c_double, _dp]
            lib.oracle_angular_polynomials.restype = None
            lib.oracle_neighbor_counts.argtypes = [C.c_int, _dp, _dp, C.c_double, _ip]
            lib.oracle_neighbors.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_int, C.c_int,
                                             _ip, _ip, _dp]
            lib.oracle_descriptors.argtypes = [C.POINTER(_Model), C.c_int, _dp, _ip, _dp, C.c_int,
                                               C.c_void_p, _dp, C.c_int]
            lib.oracle_ann.argtypes = [C.POINTER(_Model), _dp, C.POINTER(C.c_double)]
            lib.oracle_compute.argtypes = [C.POINTER(_Model), C.c_int, _dp, _ip, _dp, C.c_int,
                                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
            lib.oracle_md.argtypes = [C.POINTER(_Model), C.c_int, _dp, _dp, _ip, _dp, _dp, C.c_int,
                                      C.c_double, C.c_void_p, C.c_void_p, C.c_int]
            lib.oracle_max_threads.argtypes = []
            lib.oracle_heat_current_j2.argtypes = [C.POINTER(_Model), C.c_int, _dp, _ip, _dp, _dp, _dp, C.c_int]
            _lib = lib
    return _lib


class _Bound:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, model):
        self.arrays = [np.ascontiguousarray(a, dtype=np.float64) for a in
                       (model.c_radial, model.c_angular, model.w0, model.b0, model.w1)]
        cr, ca, w0, b0, w1 = self.arrays
        self.s = _Model(model.n_types, model.n_max_radial, model.n_max_angular, model.basis_radial,
                        model.basis_angular, model.l_max_3b, model.l_max_4b, model.l_max_5b,
                        model.n_neuron, model.rc_radial, model.rc_angular,
                        cr.ctypes.data, ca.ctypes.data, w0.ctypes.data, b0.ctypes.data,
                        w1.ctypes.data, float(model.b1))

    def ref(self):
        return C.byref(self.s)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return None if a is None else a.ctypes.data


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def n_des(model) -> int:
    b = _Bound(model)
    return int(_load().oracle_n_des(b.ref()))


def radial_basis(rc: float, K: int, r: float) -> np.ndarray:
    out = np.zeros(K + 1)
    _load().oracle_radial_basis(float(rc), int(K), float(r), out)
    return out


def angular_polynomials(d) -> np.ndarray:
    out = np.zeros(24)
    _load().oracle_angular_polynomials(float(d[0]), float(d[1]), float(d[2]), out)
    return out


def neighbor_counts(pos, box, rc) -> np.ndarray:
    pos = _f64(pos, (-1, 3))
    out = np.zeros(pos.shape[0], np.int32)
    rc_ = _load().oracle_neighbor_counts(pos.shape[0], pos, _f64(box, (3, 3)), float(rc), out)
    if rc_ != 0:
        raise ValueError("oracle_neighbor_counts failed")
    return out


def neighbors(pos, box, rc, i, cap=4096):
    """(j [M], n [M, 3], d [M, 3]) of atom i within rc, brute force over all images."""
    pos = _f64(pos, (-1, 3))
    j = np.zeros(cap, np.int32)
    n = np.zeros(cap * 3, np.int32)
    d = np.zeros(cap * 3)
    cnt = _load().oracle_neighbors(pos.shape[0], pos, _f64(box, (3, 3)), float(rc), int(i), cap, j, n, d)
    if cnt < 0 or cnt > cap:
        raise ValueError("oracle_neighbors failed")
    return j[:cnt].copy(), n[:cnt * 3].reshape(-1, 3).copy(), d[:cnt * 3].reshape(-1, 3).copy()


def descriptors(model, pos, types, box, sel=None, n_threads=0) -> np.ndarray:
    """Descriptor vectors q^i [n_sel, N_des] (all atoms when sel is None)."""
    pos = _f64(pos, (-1, 3))
    types = _i32(types)
    b = _Bound(model)
    D = model.n_des
    sel_a = None if sel is None else _i32(sel)
    ns = pos.shape[0] if sel is None else sel_a.shape[0]
    out = np.zeros((ns, D))
    rc = _load().oracle_descriptors(b.ref(), pos.shape[0], pos, types, _f64(box, (3, 3)), ns,
                                    _ptr(sel_a), out, int(n_threads))
    if rc != 0:
        raise ValueError("oracle_descriptors failed")
    return out


def site_energy(model, q) -> float:
    b = _Bound(model)
    out = C.c_double(0.0)
    if _load().oracle_ann(b.ref(), _f64(q), C.byref(out)) != 0:
        raise ValueError("oracle_ann failed")
    return float(out.value)


def compute(model, pos, types, box, sel=None, n_threads=0):
    """Site energies U [n_sel], forces F [n_sel, 3] and per-atom virials W [n_sel, 9]
    (xx, yy, zz, xy, xz, yz, yx, zx, zy) of the selected atoms (all when sel is None)."""
    pos = _f64(pos, (-1, 3))
    types = _i32(types)
    b = _Bound(model)
    sel_a = None if sel is None else _i32(sel)
    ns = pos.shape[0] if sel is None else sel_a.shape[0]
    U = np.zeros(ns)
    F = np.zeros((ns, 3))
    W = np.zeros((ns, 9))
    rc = _load().oracle_compute(b.ref(), pos.shape[0], pos, types, _f64(box, (3, 3)), ns, _ptr(sel_a),
                                U.ctypes.data, F.ctypes.data, W.ctypes.data, int(n_threads))
    if rc != 0:
        raise ValueError("oracle_compute failed")
    return U, F, W


def energy(model, pos, types, box, n_threads=0) -> float:
    U, _, _ = compute(model, pos, types, box, n_threads=n_threads)
    return float(np.sum(U))


def md(model, pos, vel, types, box, n_steps, dt, n_threads=0):
    """Velocity-Verlet NVE run. Returns (pos, vel, thermo [n_steps+1, 3] = (E_pot, E_kin, T),
    final forces [N, 3])."""
    pos = _f64(pos, (-1, 3)).copy()
    vel = _f64(vel, (-1, 3)).copy()
    types = _i32(types)
    b = _Bound(model)
    thermo = np.zeros((n_steps + 1, 3))
    F = np.zeros_like(pos)
    mass = _f64(model.mass)
    rc = _load().oracle_md(b.ref(), pos.shape[0], pos, vel, types, mass, _f64(box, (3, 3)), int(n_steps),
                           float(dt), thermo.ctypes.data, F.ctypes.data, int(n_threads))
    if rc != 0:
        raise ValueError("oracle_md failed")
    return pos, vel, thermo, F


# --------------------------------------------------------------------------- Eq. loss
def virial6(w9) -> np.ndarray:
    """The six virial components of Eq. loss (xx, yy, zz, xy, yz, zx) as the symmetric part of
    a 3x3 virial given in the order xx, yy, zz, xy, xz, yz, yx, zx, zy."""
    w = np.asarray(w9, dtype=np.float64).reshape(-1, 9)
    return np.stack([w[:, 0], w[:, 1], w[:, 2], 0.5 * (w[:, 3] + w[:, 6]), 0.5 * (w[:, 5] + w[:, 8]),
                     0.5 * (w[:, 4] + w[:, 7])], axis=1)


def eq_loss(e_pred, e_tar, f_pred, f_tar, z, lambdas, w_pred=None, w_tar=None):
    """Eq. loss of Sec. III for one candidate z, written out term by term.

    e_pred, e_tar: energy per atom of each (non-empty) structure [S]; f_pred, f_tar: forces
    of all N atoms [N, 3]; w_pred, w_tar: virial per atom [S, 6] (``virial6`` order) or None;
    lambdas = (lambda_e, lambda_f, lambda_v, lambda_1, lambda_2). The energy and virial terms
    are root mean squares over structures (the virial also over its 6 components), the force
    term over the 3N components, the regularisers the mean |z| and the root mean z^2.
    Returns (L, RMSE_E, RMSE_F, RMSE_W, l1, l2)."""
    e_pred = np.asarray(e_pred, dtype=np.float64)
    e_tar = np.asarray(e_tar, dtype=np.float64)
    n_str = e_pred.shape[0]
    rmse_e = math.sqrt(np.sum((e_pred - e_tar) ** 2) / n_str) if n_str else 0.0
    df = np.asarray(f_pred, dtype=np.float64) - np.asarray(f_tar, dtype=np.float64)
    n_atoms = df.reshape(-1, 3).shape[0]
    rmse_f = math.sqrt(np.sum(df ** 2) / (3 * n_atoms)) if n_atoms else 0.0
    rmse_w = 0.0
    if w_pred is not None and w_tar is not None and n_str:
        dw = np.asarray(w_pred, dtype=np.float64) - np.asarray(w_tar, dtype=np.float64)
        rmse_w = math.sqrt(np.sum(dw ** 2) / (6 * n_str))
    z = np.asarray(z, dtype=np.float64).reshape(-1)
    l1 = float(np.sum(np.abs(z)) / z.shape[0])
    l2 = math.sqrt(float(np.sum(z ** 2)) / z.shape[0])
    le, lf, lv, c1, c2 = (float(x) for x in lambdas)
    total = le * rmse_e + lf * rmse_f + lv * rmse_w + c1 * l1 + c2 * l2
    return total, rmse_e, rmse_f, rmse_w, l1, l2


def batch_predictions(model, offsets, pos, types, boxes, n_threads=0):
    """Oracle energy per atom [S], forces [N, 3] and virial per atom [S, 6] of every structure
    of a batch (structure s owns atoms offsets[s]..offsets[s+1]); empty structures give 0."""
    offsets = np.asarray(offsets)
    ns = offsets.shape[0] - 1
    e = np.zeros(ns)
    w = np.zeros((ns, 6))
    F = np.zeros((int(offsets[-1]), 3))
    for s in range(ns):
        a, b = int(offsets[s]), int(offsets[s + 1])
        if b == a:
            continue
        U, Fs, Ws = compute(model, pos[a:b], types[a:b], boxes[s], n_threads=n_threads)
        e[s] = U.sum() / (b - a)
        F[a:b] = Fs
        w[s] = virial6(Ws.sum(0))[0] / (b - a)
    return e, F, w


# --------------------------------------------------------------------------- FIRE
# Constants of the FIRE minimiser (Bitzek et al., Phys. Rev. Lett. 97, 170201 (2006)).
FIRE_NMIN, FIRE_FINC, FIRE_FDEC, FIRE_ALPHA_START, FIRE_FALPHA, FIRE_DTMAX_FACTOR = 5, 1.1, 0.5, 0.1, 0.99, 10.0
KAPPA = 1.66053906660e-27 * 1e-20 / 1e-30 / 1.602176634e-19  # 1 u A^2 / fs^2 in eV


def fire_minimize(force_fn, x0, inv_mass, n_steps, dt0, fmax):
    """FIRE from rest, written out step by step: a velocity-Verlet step of length dt
    (a = F * inv_mass), then with P = F . v: for P > 0, v <- (1 - alpha) v + alpha |v| F/|F|
    and, once more than N_min steps in a row had P > 0, dt <- min(f_inc dt, dt_max) and
    alpha <- f_alpha alpha; for P <= 0, v <- 0, dt <- f_dec dt, alpha <- alpha_start. Stops
    when max_i |F_i| < fmax (tested on the starting forces and after every step).

    force_fn(x) -> (E, F). Returns (x, E, F, steps, energies) with energies after each step."""
    x = np.array(x0, dtype=np.float64)
    im = np.asarray(inv_mass, dtype=np.float64).reshape(-1, 1)
    v = np.zeros_like(x)
    E, F = force_fn(x)
    dt, alpha, npos, steps = float(dt0), FIRE_ALPHA_START, 0, 0
    dt_max = FIRE_DTMAX_FACTOR * dt0
    energies = []
    if np.max(np.sum(F * F, axis=1)) < fmax * fmax:
        return x, E, F, 0, energies
    for _ in range(n_steps):
        v = v + 0.5 * dt * F * im
        x = x + dt * v
        E, F = force_fn(x)
        v = v + 0.5 * dt * F * im
        steps += 1
        energies.append(E)
        if np.max(np.sum(F * F, axis=1)) < fmax * fmax:
            break
        P = float(np.sum(F * v))
        if P > 0.0:
            fn = math.sqrt(float(np.sum(F * F)))
            vn = math.sqrt(float(np.sum(v * v)))
            v = (1.0 - alpha) * v + (alpha * vn / fn if fn > 0 else 0.0) * F
            if npos > FIRE_NMIN:
                dt = min(dt * FIRE_FINC, dt_max)
                alpha *= FIRE_FALPHA
            npos += 1
        else:
            v = np.zeros_like(v)
            dt *= FIRE_FDEC
            alpha = FIRE_ALPHA_START
            npos = 0
    return x, E, F, steps, energies


def fire(model, pos, types, box, n_steps, dt0, fmax, n_threads=0):
    """FIRE relaxation of one structure with the oracle's energy and forces."""
    types = _i32(types)
    inv_mass = 1.0 / (np.asarray(model.mass, dtype=np.float64)[types] * KAPPA)

    def force_fn(x):
        U, F, _ = compute(model, x, types, box, n_threads=n_threads)
        return float(np.sum(U)), F

    return fire_minimize(force_fn, pos, inv_mass, n_steps, dt0, fmax)


# --------------------------------------------------------------------------- heat current
def heat_current(model, pos, types, box, vel, n_threads=0):
    """Per-atom heat current J_i = W_i . v_i (Eq. Ji) from the oracle's per-atom virials, and
    the total J = sum_i J_i (Eq. J-1). Velocities in A/fs; J in eV A/fs."""
    _, _, Wv = compute(model, pos, types, box, n_threads=n_threads)
    v = _f64(vel, (-1, 3))
    order = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2), (1, 0), (2, 0), (2, 1)]
    Wm = np.zeros((Wv.shape[0], 3, 3))
    for c, (a, b) in enumerate(order):
        Wm[:, a, b] = Wv[:, c]
    J = np.einsum("iab,ib->ia", Wm, v)
    return J, J.sum(axis=0)


def heat_current_j2(model, pos, types, box, vel, n_threads=0):
    """Total heat current by Eq. J-2, from every atom's own partial forces and its neighbours'
    velocities (a different data path from Eq. J-1)."""
    b = _Bound(model)
    pos = _f64(pos, (-1, 3))
    J = np.zeros(3)
    rc = _load().oracle_heat_current_j2(b.ref(), pos.shape[0], pos, _i32(types), _f64(box, (3, 3)),
                                        _f64(vel, (-1, 3)), J, int(n_threads))
    if rc != 0:
        raise ValueError("oracle_heat_current_j2 failed")
    return J


# --------------------------------------------------------------------------- BDP thermostat
KB = 8.617333262e-5  # eV/K


def bdp_alpha(K, kbar, nf, c, R1, S):
    """Velocity factor of the Bussi-Donadio-Parrinello thermostat (J. Chem. Phys. 126,
    014101 (2007)) for kinetic energy K, target Kbar, N_f degrees of freedom, c = exp(-dt/tau)
    and the step's random numbers R1 ~ N(0,1), S ~ chi^2(N_f - 1): the new kinetic energy is
    alpha^2 K with alpha^2 = c + (1 - c)(S + R1^2) Kbar/(N_f K) + 2 R1 sqrt(c (1-c) Kbar/(N_f K)),
    alpha taking the sign of R1 + sqrt(c N_f K / ((1 - c) Kbar))."""
    if K <= 0.0:
        return 1.0
    q = kbar / (nf * K)
    a2 = c + (1.0 - c) * (S + R1 * R1) * q + 2.0 * R1 * math.sqrt(c * (1.0 - c) * q)
    alpha = math.sqrt(max(a2, 0.0))
    if c < 1.0 and R1 + math.sqrt(c / ((1.0 - c) * q)) < 0.0:
        alpha = -alpha
    return alpha


def md_bdp(model, pos, vel, types, box, n_steps, dt, temperature, tau, rand, n_threads=0):
    """Velocity-Verlet steps, each followed by the BDP rescaling with rand[k] = (R1, S)
    (temperature <= 0: plain NVE). Returns (pos, vel, thermo [n_steps, 3] = (E_pot, E_kin, T)
    after each step, heat current [n_steps, 3] = sum_i W_i . v_i after each step)."""
    types = _i32(types)
    x = _f64(pos, (-1, 3)).copy()
    v = _f64(vel, (-1, 3)).copy()
    N = x.shape[0]
    m = np.asarray(model.mass, dtype=np.float64)[types]
    im = (1.0 / (m * KAPPA))[:, None]
    nf = 3.0 * N - 3.0
    c = math.exp(-dt / tau) if temperature > 0 else 1.0
    kbar = 0.5 * nf * KB * temperature
    U, F, Wv = compute(model, x, types, box, n_threads=n_threads)
    thermo, heat = [], []
    order = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2), (1, 0), (2, 0), (2, 1)]
    for k in range(n_steps):
        v = v + 0.5 * dt * F * im
        x = x + dt * v
        U, F, Wv = compute(model, x, types, box, n_threads=n_threads)
        v = v + 0.5 * dt * F * im
        if temperature > 0:
            K = 0.5 * KAPPA * float(np.sum(m[:, None] * v * v))
            v = v * bdp_alpha(K, kbar, nf, c, float(rand[k][0]), float(rand[k][1]))
        ke = 0.5 * KAPPA * float(np.sum(m[:, None] * v * v))
        thermo.append((float(U.sum()), ke, 2.0 * ke / (nf * KB)))
        Wm = np.zeros((N, 3, 3))
        for cc, (a, b) in enumerate(order):
            Wm[:, a, b] = Wv[:, cc]
        heat.append(np.einsum("iab,ib->ia", Wm, v).sum(axis=0))
    return x, v, np.array(thermo), np.array(heat)
