"""Thin ctypes binding of libnep (include/nep.h).

Argument marshalling only: every step of the NEP evaluation runs in the library's CUDA
kernels. Functions keep the C names (nep_create, nep_compute, md_init, md_run, ...);
device arrays are torch CUDA tensors, passed by data pointer on torch's current stream.
There is no CPU fallback: if libnep.so is missing or cannot load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnep.so")

NEP_OK = 0
ERRORS = {-1: "NEP_ERR_ARG", -2: "NEP_ERR_OOM", -3: "NEP_ERR_CUDA", -4: "NEP_ERR_NEIGHBOR_OVERFLOW",
          -5: "NEP_ERR_NONFINITE", -6: "NEP_ERR_UNSUPPORTED", -7: "NEP_ERR_STATE", -8: "NEP_ERR_TIMEOUT"}


class NepError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class nep_params(C.Structure):
    _fields_ = [("version", C.c_int), ("n_types", C.c_int), ("rc_radial", C.c_double),
                ("rc_angular", C.c_double), ("n_max_radial", C.c_int), ("n_max_angular", C.c_int),
                ("basis_radial", C.c_int), ("basis_angular", C.c_int), ("l_max_3b", C.c_int),
                ("l_max_4b", C.c_int), ("l_max_5b", C.c_int), ("n_neuron", C.c_int),
                ("c_radial", C.c_void_p), ("c_angular", C.c_void_p), ("w0", C.c_void_p),
                ("b0", C.c_void_p), ("w1", C.c_void_p), ("b1", C.c_double), ("mass", C.c_void_p),
                ("skin", C.c_double)]


class nep_stats(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("cap_radial", C.c_int), ("cap_angular", C.c_int),
                ("max_radial", C.c_int), ("max_angular", C.c_int), ("mean_radial", C.c_double),
                ("mean_angular", C.c_double), ("mean_radial_in_rc", C.c_double),
                ("mean_angular_in_rc", C.c_double), ("n_rebuilds", C.c_longlong),
                ("md_steps", C.c_longlong), ("cells", C.c_int * 3), ("graph_kernels", C.c_int),
                ("rebuild_kernels", C.c_int), ("batch_graph_kernels", C.c_int)]


class nep_tuning(C.Structure):
    _fields_ = [("members_per_launch", C.c_int), ("atom_block", C.c_int), ("gather_block", C.c_int),
                ("last_members", C.c_int), ("n_tried", C.c_int), ("best_ms", C.c_float),
                ("default_ms", C.c_float), ("atom_form", C.c_int)]


class md_options(C.Structure):
    _fields_ = [("thermo_every", C.c_int), ("thermo", C.c_void_p), ("heat_current", C.c_void_p),
                ("temperature", C.c_double), ("tau_fs", C.c_double), ("bdp_random", C.c_void_p)]


class nep_server_config(C.Structure):
    _fields_ = [("memory_budget", C.c_size_t), ("workers", C.c_int), ("precision", C.c_int),
                ("compact_every", C.c_int), ("min_chunk", C.c_int)]


class nep_job(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_atoms", C.c_int), ("pos", C.c_void_p), ("types", C.c_void_p),
                ("vel", C.c_void_p), ("box", C.c_double * 9), ("n_steps", C.c_int), ("dt_fs", C.c_double),
                ("fmax", C.c_double)]


class nep_result(C.Structure):
    _fields_ = [("id", C.c_longlong), ("status", C.c_int), ("kind", C.c_int), ("n_atoms", C.c_int),
                ("steps", C.c_int), ("energy", C.c_double), ("virial", C.c_double * 9), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_done", C.c_double), ("workspace_est", C.c_size_t),
                ("workspace_used", C.c_size_t), ("message", C.c_char * 160)]


class nep_server_stats(C.Structure):
    _fields_ = [("queued", C.c_int), ("running", C.c_int), ("completed", C.c_longlong), ("failed", C.c_longlong),
                ("bytes_reserved", C.c_size_t), ("peak_bytes_reserved", C.c_size_t),
                ("peak_workspace_bytes", C.c_size_t), ("atom_evaluations", C.c_double),
                ("iterations", C.c_longlong), ("relayouts", C.c_longlong), ("relayout_seconds", C.c_double),
                ("step_seconds", C.c_double), ("fetch_seconds", C.c_double), ("builds", C.c_longlong)]


JOB_SINGLE, JOB_FIRE, JOB_NVE = 0, 1, 2

_lib = None

# exported symbol -> (restype, argtypes)
_P = C.c_void_p
_SIGS = {
    "nep_create": (C.c_int, [C.POINTER(nep_params), C.POINTER(_P)]),
    "nep_destroy": (C.c_int, [_P]),
    "nep_last_error": (C.c_char_p, [_P]),
    "nep_compute": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "nep_compute_host": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, _P, _P, _P]),
    "nep_compute_batch": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "nep_n_par": (C.c_int, [_P]),
    "nep_eval_population": (C.c_int, [_P, C.c_int, _P, C.c_int, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "nep_set_tuning": (C.c_int, [_P, C.POINTER(nep_tuning)]),
    "nep_get_tuning": (C.c_int, [_P, C.POINTER(nep_tuning)]),
    "nep_autotune": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, C.c_int, C.POINTER(nep_tuning), _P]),
    "nep_descriptors": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P]),
    "nep_n_des": (C.c_int, [_P]),
    "md_init": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P]),
    "md_init_host": (C.c_int, [_P, C.c_int, _P, _P, _P, _P]),
    "md_run": (C.c_int, [_P, C.c_int, C.c_double, C.c_int, _P, _P]),
    "md_run_async": (C.c_int, [_P, C.c_int, C.c_double, C.c_int, _P, _P]),
    "fire_run": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, _P, C.POINTER(C.c_int), _P]),
    "md_run_ex": (C.c_int, [_P, C.c_int, C.c_double, C.POINTER(md_options), _P]),
    "nep_heat_current": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, _P, _P]),
    "md_status": (C.c_int, [_P, _P]),
    "md_get_state": (C.c_int, [_P, _P, _P, _P, _P]),
    "md_get_state_host": (C.c_int, [_P, _P, _P, _P]),
    "nep_get_stats": (C.c_int, [_P, C.POINTER(nep_stats)]),
    "nep_set_profiling": (C.c_int, [_P, C.c_int]),
    "nep_set_graph_conditional": (C.c_int, [_P, C.c_int]),
    "nep_set_precision": (C.c_int, [_P, C.c_int]),
    "nep_kernel_slots": (C.c_int, []),
    "nep_kernel_name": (C.c_char_p, [C.c_int]),
    "nep_kernel_times": (C.c_int, [_P, C.POINTER(C.c_float), C.c_int]),
    "nep_supported": (C.c_int, [C.POINTER(C.c_int), C.c_int]),
    "nep_export_lists": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, _P]),
    "nep_descriptors_static": (C.c_int, [C.POINTER(nep_params), C.c_int, _P, _P, _P, _P, _P]),
    "nep_server_create": (C.c_int, [C.POINTER(nep_params), C.POINTER(nep_server_config), C.POINTER(_P)]),
    "nep_server_submit": (C.c_int, [_P, C.POINTER(nep_job), C.POINTER(C.c_longlong)]),
    "nep_server_wait": (C.c_int, [_P, C.c_double, C.POINTER(nep_result)]),
    "nep_server_arrays": (C.c_int, [_P, C.c_longlong, _P, _P, _P]),
    "nep_server_stats_get": (C.c_int, [_P, C.POINTER(nep_server_stats)]),
    "nep_server_destroy": (C.c_int, [_P]),
}
EXPORTED = tuple(_SIGS)


def load(path: str | None = None) -> C.CDLL:
    """Load libnep.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libnep.so not built ({p}); run __graft_entry__.build()")
        lib = C.CDLL(p)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int, h=None):
    if rc != NEP_OK:
        msg = load().nep_last_error(h)
        raise NepError(rc, msg.decode() if msg else "")


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _dev(t, dtype, shape=None, name="array"):
    """Data pointer of a contiguous CUDA tensor of this dtype and shape (checked in that
    order of failure: type, dtype/layout, shape, device), or None for None."""
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    return t.data_ptr()


def _shape(t, shape, name):
    """Raise ValueError unless tensor t (if given) has exactly this shape."""
    if t is not None and tuple(getattr(t, "shape", ())) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(getattr(t, 'shape', ()))}, expected {tuple(shape)}")


def _box(box) -> np.ndarray:
    b = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(3, 3))
    return b


def nep_supported():
    lib = load()
    n = lib.nep_supported(None, 0)
    buf = (C.c_int * (8 * n))()
    lib.nep_supported(buf, n)
    return [tuple(buf[8 * i:8 * i + 8]) for i in range(n)]


def _params(model, skin: float):
    """nep_params for a workloads.NepModel; returns (struct, arrays kept alive by the caller)."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in
            (model.c_radial, model.c_angular, model.w0, model.b0, model.w1)]
    mass = None if model.mass is None else np.ascontiguousarray(model.mass, dtype=np.float64)
    p = nep_params(3, model.n_types, model.rc_radial, model.rc_angular, model.n_max_radial,
                   model.n_max_angular, model.basis_radial, model.basis_angular, model.l_max_3b,
                   model.l_max_4b, model.l_max_5b, model.n_neuron,
                   *[a.ctypes.data for a in arrs], float(model.b1),
                   None if mass is None else mass.ctypes.data, float(skin))
    return p, (arrs, mass)


def nep_create(model, skin: float = 1.0):
    """Handle for a workloads.NepModel (weights are copied into the library)."""
    lib = load()
    p, _keep = _params(model, skin)
    h = C.c_void_p()
    rc = lib.nep_create(C.byref(p), C.byref(h))
    _check(rc, None)
    return h


def nep_destroy(h):
    if h:
        load().nep_destroy(h)


def nep_n_des(h) -> int:
    return int(load().nep_n_des(h))


def nep_compute(h, pos, types, box, energy=None, energy_total=None, force=None, virial=None,
                virial_total=None):
    """Device evaluation; pos [N,3] f64, types [N] i32, outputs preallocated CUDA f64 tensors."""
    import torch
    n = int(pos.shape[0])
    b = _box(box)
    rc = load().nep_compute(h, n, _dev(pos, torch.float64, (n, 3), "pos"), _dev(types, torch.int32, (n,), "types"),
                            b.ctypes.data, _dev(energy, torch.float64, (n,), "energy"),
                            _dev(energy_total, torch.float64, (1,), "energy_total"),
                            _dev(force, torch.float64, (n, 3), "force"), _dev(virial, torch.float64, (n, 9), "virial"),
                            _dev(virial_total, torch.float64, (9,), "virial_total"), _stream())
    _check(rc, h)


def nep_compute_host(h, pos, types, box):
    """Host-array evaluation: returns (U [N], E, F [N,3], W [N,9], W_total [9])."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    types = np.ascontiguousarray(types, dtype=np.int32)
    n = pos.shape[0]
    U = np.zeros(n)
    F = np.zeros((n, 3))
    Wv = np.zeros((n, 9))
    Wt = np.zeros(9)
    E = C.c_double(0.0)
    b = _box(box)
    rc = load().nep_compute_host(h, n, pos.ctypes.data, types.ctypes.data, b.ctypes.data, U.ctypes.data,
                                 C.addressof(E), F.ctypes.data, Wv.ctypes.data, Wt.ctypes.data)
    _check(rc, h)
    return U, float(E.value), F, Wv, Wt


def _offsets(offsets) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(offsets, dtype=np.int32).reshape(-1))


def _boxes(boxes, n_struct: int) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(boxes, dtype=np.float64).reshape(n_struct, 9))


def nep_compute_batch(h, offsets, pos, types, boxes, energy=None, energy_struct=None, force=None, virial=None,
                      virial_struct=None):
    """Batched evaluation of many structures: offsets [S+1] and boxes [S,3,3] on the host;
    pos [N,3] f64, types [N] i32 and the preallocated outputs are CUDA tensors."""
    import torch
    off = _offsets(offsets)
    ns = off.shape[0] - 1
    n = int(off[-1]) if ns > 0 else 0
    bx = _boxes(boxes, ns)
    rc = load().nep_compute_batch(h, ns, off.ctypes.data, _dev(pos, torch.float64, (n, 3), "pos"),
                                  _dev(types, torch.int32, (n,), "types"), bx.ctypes.data,
                                  _dev(energy, torch.float64, (n,), "energy"),
                                  _dev(energy_struct, torch.float64, (ns,), "energy_struct"),
                                  _dev(force, torch.float64, (n, 3), "force"),
                                  _dev(virial, torch.float64, (n, 9), "virial"),
                                  _dev(virial_struct, torch.float64, (ns, 9), "virial_struct"), _stream())
    _check(rc, h)


def nep_n_par(h) -> int:
    return int(load().nep_n_par(h))


def nep_eval_population(h, z, offsets, pos, types, boxes, e_tar, f_tar, w_tar=None, lambdas=(1.0, 1.0, 0.0, 0.0, 0.0),
                        loss=None):
    """Eq. loss for each candidate vector: z [P, N_par] f64 CUDA; structure set as
    nep_compute_batch; targets e_tar [S] (eV/atom), f_tar [N,3], w_tar [S,6] or None.
    Returns loss [P, 6] (CUDA): L, RMSE_E, RMSE_F, RMSE_W, l1 term, l2 term."""
    import torch
    off = _offsets(offsets)
    ns = off.shape[0] - 1
    n = int(off[-1]) if ns > 0 else 0
    bx = _boxes(boxes, ns)
    npop = int(z.shape[0])
    npar = nep_n_par(h)
    if loss is None:
        loss = torch.empty((npop, 6), dtype=torch.float64, device=z.device)
    lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64).reshape(5))
    rc = load().nep_eval_population(h, npop, _dev(z, torch.float64, (npop, npar), "z"), ns, off.ctypes.data,
                                    _dev(pos, torch.float64, (n, 3), "pos"), _dev(types, torch.int32, (n,), "types"),
                                    bx.ctypes.data, _dev(e_tar, torch.float64, (ns,), "e_tar"),
                                    _dev(f_tar, torch.float64, (n, 3), "f_tar"),
                                    _dev(w_tar, torch.float64, (ns, 6), "w_tar"), lam.ctypes.data,
                                    _dev(loss, torch.float64, (npop, 6), "loss"), _stream())
    _check(rc, h)
    return loss


def nep_set_tuning(h, members_per_launch: int = 0, atom_block: int = 0, gather_block: int = 0, atom_form: int = 0):
    t = nep_tuning(int(members_per_launch), int(atom_block), int(gather_block), 0, 0, 0.0, 0.0, int(atom_form))
    _check(load().nep_set_tuning(h, C.byref(t)), h)


def nep_autotune(h, offsets, pos, types, boxes, n_pop: int = 0) -> dict:
    """Time the batched kernels' launch shapes on this structure set; keeps and returns the best."""
    import torch
    off = _offsets(offsets)
    ns = off.shape[0] - 1
    n = int(off[-1]) if ns > 0 else 0
    bx = _boxes(boxes, ns)
    t = nep_tuning()
    rc = load().nep_autotune(h, ns, off.ctypes.data, _dev(pos, torch.float64, (n, 3), "pos"),
                             _dev(types, torch.int32, (n,), "types"), bx.ctypes.data, int(n_pop), C.byref(t),
                             _stream())
    _check(rc, h)
    return {f: getattr(t, f) for f, _ in nep_tuning._fields_}


def nep_get_tuning(h) -> dict:
    t = nep_tuning()
    _check(load().nep_get_tuning(h, C.byref(t)), h)
    return {f: getattr(t, f) for f, _ in nep_tuning._fields_}


def nep_descriptors(h, pos, types, box, q):
    """Descriptors q [n, N_des] (CUDA f64, caller atom order) of one periodic structure."""
    import torch
    n = int(pos.shape[0])
    b = _box(box)
    _shape(q, (n, nep_n_des(h)), "q")  # the kernel writes n x N_des values
    args = (_dev(pos, torch.float64, (n, 3), "pos"), _dev(types, torch.int32, (n,), "types"), b.ctypes.data,
            _dev(q, torch.float64, (n, nep_n_des(h)), "q"))
    _check(load().nep_descriptors(h, n, *args, _stream()), h)


def nep_descriptors_static(model, pos, types, box, q, skin: float = 1.0):
    """Descriptors without any device allocation (library-internal fixed scratch)."""
    import torch
    n = int(pos.shape[0])
    b = _box(box)
    _shape(q, (n, model.n_des), "q")  # the kernel writes n x N_des values
    args = (_dev(pos, torch.float64, (n, 3), "pos"), _dev(types, torch.int32, (n,), "types"), b.ctypes.data,
            _dev(q, torch.float64, (n, model.n_des), "q"))
    p, _keep = _params(model, skin)
    _check(load().nep_descriptors_static(C.byref(p), n, *args, _stream()), None)


def md_init(h, pos, types, box, vel=None):
    import torch
    n = int(pos.shape[0])
    b = _box(box)
    rc = load().md_init(h, n, _dev(pos, torch.float64, (n, 3), "pos"), _dev(types, torch.int32, (n,), "types"),
                        b.ctypes.data, _dev(vel, torch.float64, (n, 3), "vel"), _stream())
    _check(rc, h)


def md_init_host(h, pos, types, box, vel=None):
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    types = np.ascontiguousarray(types, dtype=np.int32)
    v = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64).reshape(-1, 3)
    b = _box(box)
    rc = load().md_init_host(h, pos.shape[0], pos.ctypes.data, types.ctypes.data, b.ctypes.data,
                             None if v is None else v.ctypes.data)
    _check(rc, h)


def md_run(h, n_steps: int, dt_fs: float, thermo_every: int = 1, thermo=None):
    import torch
    rc = load().md_run(h, int(n_steps), float(dt_fs), int(thermo_every), _dev(thermo, torch.float64, None, "thermo"),
                       _stream())
    _check(rc, h)


def md_run_async(h, n_steps: int, dt_fs: float, thermo_every: int = 1, thermo=None, stream=None):
    import torch
    rc = load().md_run_async(h, int(n_steps), float(dt_fs), int(thermo_every),
                             _dev(thermo, torch.float64, None, "thermo"), _stream() if stream is None else stream)
    _check(rc, h)


def fire_run(h, n_steps: int, dt0_fs: float, fmax: float, thermo=None) -> int:
    """FIRE relaxation from the md_init state; returns the steps taken before convergence."""
    import torch
    steps = C.c_int(0)
    rc = load().fire_run(h, int(n_steps), float(dt0_fs), float(fmax),
                         _dev(thermo, torch.float64, (n_steps, 4), "thermo"), C.byref(steps), _stream())
    _check(rc, h)
    return int(steps.value)


def md_run_ex(h, n_steps: int, dt_fs: float, thermo_every: int = 1, thermo=None, heat_current=None,
              temperature: float = 0.0, tau_fs: float = 100.0, bdp_random=None):
    """md_run with the total heat current per thermo row and an optional BDP thermostat
    (bdp_random [n_steps, 2] CUDA f64: R1 ~ N(0,1), S ~ chi^2(3N-4) per step)."""
    import torch
    rows = n_steps // thermo_every
    o = md_options(int(thermo_every), _dev(thermo, torch.float64, (rows, 4), "thermo"),
                   _dev(heat_current, torch.float64, (rows, 3), "heat_current"), float(temperature), float(tau_fs),
                   _dev(bdp_random, torch.float64, (n_steps, 2), "bdp_random"))
    _check(load().md_run_ex(h, int(n_steps), float(dt_fs), C.byref(o), _stream()), h)


def nep_heat_current(h, pos, types, box, vel, heat=None, heat_total=None):
    """Per-atom heat current J_i = W_i . v_i [N, 3] and its total [3] (CUDA f64 outputs)."""
    import torch
    n = int(pos.shape[0])
    b = _box(box)
    rc = load().nep_heat_current(h, n, _dev(pos, torch.float64, (n, 3), "pos"), _dev(types, torch.int32, (n,), "types"),
                                 b.ctypes.data, _dev(vel, torch.float64, (n, 3), "vel"),
                                 _dev(heat, torch.float64, (n, 3), "heat"),
                                 _dev(heat_total, torch.float64, (3,), "heat_total"), _stream())
    _check(rc, h)


def md_status(h, stream=None):
    _check(load().md_status(h, _stream() if stream is None else stream), h)


def md_get_state(h, pos=None, vel=None, force=None):
    import torch
    rc = load().md_get_state(h, _dev(pos, torch.float64, None, "pos"), _dev(vel, torch.float64, None, "vel"),
                             _dev(force, torch.float64, None, "force"), _stream())
    _check(rc, h)


def md_get_state_host(h, n: int, pos=None, vel=None, F=None):
    """(pos, vel, F) [n, 3] float64 host arrays; pass preallocated C-contiguous arrays (e.g.
    views of page-locked memory) to have them filled in place."""
    out = []
    for a in (pos, vel, F):
        if a is None:
            a = np.zeros((n, 3))
        elif a.dtype != np.float64 or a.shape != (n, 3) or not a.flags.c_contiguous:
            raise ValueError("state arrays must be C-contiguous float64 [n, 3]")
        out.append(a)
    pos, vel, F = out
    rc = load().md_get_state_host(h, pos.ctypes.data, vel.ctypes.data, F.ctypes.data)
    _check(rc, h)
    return pos, vel, F


def nep_export_lists(h, n_atoms: int, cap: int | None = None) -> dict:
    """Neighbour lists of the last build in caller order (host numpy arrays): nn_r [N],
    j_r [N, cap], d_r [N, cap, 3] (FP32 pair vectors), and the same for the angular list."""
    if cap is None:
        st = nep_get_stats(h)
        cap = max(1, int(st["max_radial"]), int(st["max_angular"]))
    n = int(n_atoms)
    out = dict(nn_r=np.zeros(n, np.int32), j_r=np.zeros((n, cap), np.int32), d_r=np.zeros((n, cap, 3), np.float32),
               nn_a=np.zeros(n, np.int32), j_a=np.zeros((n, cap), np.int32), d_a=np.zeros((n, cap, 3), np.float32))
    rc = load().nep_export_lists(h, int(cap), *(out[k].ctypes.data for k in ("nn_r", "j_r", "d_r", "nn_a", "j_a", "d_a")))
    _check(rc, h)
    return out


def nep_get_stats(h) -> dict:
    s = nep_stats()
    _check(load().nep_get_stats(h, C.byref(s)), h)
    d = {f: getattr(s, f) for f, _ in nep_stats._fields_}
    d["cells"] = tuple(s.cells)
    return d


def nep_set_profiling(h, enable: bool):
    _check(load().nep_set_profiling(h, 1 if enable else 0), h)


def nep_set_precision(h, mode: int):
    """0: FP32 network on the FMA pipes; 1: BF16 tensor-core network (tcgen05)."""
    _check(load().nep_set_precision(h, int(mode)), h)


def nep_set_graph_conditional(h, enable: bool):
    _check(load().nep_set_graph_conditional(h, 1 if enable else 0), h)


def nep_kernel_times(h) -> dict:
    lib = load()
    n = lib.nep_kernel_slots()
    buf = (C.c_float * n)()
    _check(lib.nep_kernel_times(h, buf, n), h)
    return {lib.nep_kernel_name(i).decode(): float(buf[i]) for i in range(n)}


class NEP:
    """Convenience owner of one handle (destroyed with the object)."""

    def __init__(self, model, skin: float = 1.0, precision: int = 0):
        self.model = model
        self.h = nep_create(model, skin)
        if precision:
            nep_set_precision(self.h, precision)

    def close(self):
        if self.h:
            nep_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def compute(self, pos, types, box, per_atom_virial: bool = False):
        """pos/types as CUDA tensors; returns dict of CUDA tensors (U, E, F, W?, W_total)."""
        import torch
        n = int(pos.shape[0])
        dev = pos.device
        out = dict(U=torch.empty(n, dtype=torch.float64, device=dev),
                   E=torch.empty(1, dtype=torch.float64, device=dev),
                   F=torch.empty((n, 3), dtype=torch.float64, device=dev),
                   W_total=torch.empty(9, dtype=torch.float64, device=dev))
        if per_atom_virial:
            out["W"] = torch.empty((n, 9), dtype=torch.float64, device=dev)
        nep_compute(self.h, pos, types, box, out["U"], out["E"], out["F"], out.get("W"), out["W_total"])
        return out

    def compute_batch(self, offsets, pos, types, boxes, per_atom: bool = False):
        """Batched evaluation; returns dict of CUDA tensors (E_struct [S], F [N,3],
        W_struct [S,9], and U [N], W [N,9] when per_atom)."""
        import torch
        off = _offsets(offsets)
        ns, n = off.shape[0] - 1, int(off[-1])
        dev = pos.device
        out = dict(E_struct=torch.empty(ns, dtype=torch.float64, device=dev),
                   F=torch.empty((n, 3), dtype=torch.float64, device=dev),
                   W_struct=torch.empty((ns, 9), dtype=torch.float64, device=dev))
        if per_atom:
            out["U"] = torch.empty(n, dtype=torch.float64, device=dev)
            out["W"] = torch.empty((n, 9), dtype=torch.float64, device=dev)
        nep_compute_batch(self.h, off, pos, types, boxes, out.get("U"), out["E_struct"], out["F"], out.get("W"),
                          out["W_struct"])
        return out


# ----------------------------------------------------------------------------- serving
class Server:
    """A running nep_server: submit jobs (host arrays), collect results in completion order."""

    def __init__(self, model, memory_budget: int, workers: int = 16, precision: int = 0, skin: float = 1.0,
                 compact_every: int = 0, min_chunk: int = 0):
        lib = load()
        p, self._keep = _params(model, skin)
        cfg = nep_server_config(int(memory_budget), int(workers), int(precision), int(compact_every), int(min_chunk))
        h = C.c_void_p()
        _check(lib.nep_server_create(C.byref(p), C.byref(cfg), C.byref(h)), None)
        self.h = h
        self.n = {}

    def submit(self, kind: int, pos, types, box, n_steps: int = 0, dt_fs: float = 1.0, fmax: float = 0.0,
               vel=None) -> int:
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        types = np.ascontiguousarray(types, dtype=np.int32)
        v = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64).reshape(-1, 3)
        j = nep_job(int(kind), pos.shape[0], pos.ctypes.data, types.ctypes.data, None if v is None else v.ctypes.data,
                    (C.c_double * 9)(*_box(box).ravel()), int(n_steps), float(dt_fs), float(fmax))
        jid = C.c_longlong(0)
        rc = load().nep_server_submit(self.h, C.byref(j), C.byref(jid))
        if rc != NEP_OK:
            raise NepError(rc, "nep_server_submit")
        self.n[int(jid.value)] = pos.shape[0]
        return int(jid.value)

    def wait(self, timeout_s: float = -1.0):
        """Next finished job as a dict, or None on timeout."""
        r = nep_result()
        rc = load().nep_server_wait(self.h, float(timeout_s), C.byref(r))
        if rc == -8:
            return None
        if rc != NEP_OK:
            raise NepError(rc, "nep_server_wait")
        out = {f: getattr(r, f) for f, _ in nep_result._fields_}
        out["virial"] = np.array(r.virial[:])
        out["message"] = r.message.decode(errors="replace")
        return out

    def arrays(self, job_id: int):
        """(pos, force, vel) of a finished job."""
        n = self.n.pop(job_id)
        pos, force, vel = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
        rc = load().nep_server_arrays(self.h, int(job_id), pos.ctypes.data, force.ctypes.data, vel.ctypes.data)
        if rc != NEP_OK:
            raise NepError(rc, "nep_server_arrays")
        return pos, force, vel

    def drop(self, job_id: int):
        """Discard the arrays of a finished job without copying them."""
        self.n.pop(job_id, None)
        load().nep_server_arrays(self.h, int(job_id), None, None, None)

    def stats(self) -> dict:
        st = nep_server_stats()
        _check(load().nep_server_stats_get(self.h, C.byref(st)), None)
        return {f: getattr(st, f) for f, _ in nep_server_stats._fields_}

    def close(self):
        if self.h:
            load().nep_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
