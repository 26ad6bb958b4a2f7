"""ctypes binding of libiontrap.so -- argument marshalling only.

Every function has the name of the C entry point it calls (include/iontrap.h) and does
no arithmetic of the method: all of it runs in the library's CUDA kernels.  Importing
this module loads the library and raises ``ImportError`` if it has not been built
(``python -c "import __graft_entry__ as g; g.build()"``); there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libiontrap.so")

IONTRAP_OK = 0
IONTRAP_EINVAL = 1
IONTRAP_ENOMEM = 2
IONTRAP_EUNSTABLE = 3
IONTRAP_ENONFINITE = 4
IONTRAP_ETIMEOUT = 5
IONTRAP_ECUDA = 6
IONTRAP_ETOOLARGE = 7

IONTRAP_RF_OFF = 1
IONTRAP_COULOMB_OFF = 2
IONTRAP_TRAP_OFF = 4
IONTRAP_ALLOW_UNSTABLE = 8
IONTRAP_PSEUDO = 16

IONTRAP_REC_X = 1
IONTRAP_REC_V = 2
IONTRAP_REC_VAVG = 4

IONTRAP_PREC_FP32 = 0
IONTRAP_PREC_FP64 = 1
IONTRAP_TUNE_BATCHED = 2

IONTRAP_MAX_SPECIES = 16


class iontrap_species(ctypes.Structure):
    _fields_ = [("mass_amu", ctypes.c_double), ("charge_e", ctypes.c_double)]


class iontrap_params(ctypes.Structure):
    _fields_ = [("Omega", ctypes.c_double), ("a", ctypes.c_double), ("q", ctypes.c_double),
                ("omega_z", ctypes.c_double), ("gamma", ctypes.c_double),
                ("T_bath", ctypes.c_double), ("dt", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("precision", ctypes.c_int32)]


class iontrap_cooling(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("T_bath", ctypes.c_double), ("laser", ctypes.c_double * 3)]


class iontrap_config(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("ions_per_thread", ctypes.c_int32),
                ("packed", ctypes.c_int32), ("jsplit", ctypes.c_int32), ("fused", ctypes.c_int32),
                ("pdl", ctypes.c_int32), ("graph", ctypes.c_int32)]


class iontrap_server_config(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_int64), ("max_resident", ctypes.c_int32),
                ("chunk_steps", ctypes.c_int32), ("max_parallel", ctypes.c_int32)]


class iontrap_server_counters(ctypes.Structure):
    _fields_ = [("waiting", ctypes.c_int64), ("resident", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64)]


class iontrap_tuning_entry(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("log2n", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("ions_per_thread", ctypes.c_int32), ("packed", ctypes.c_int32), ("splits", ctypes.c_int32),
                ("fused", ctypes.c_int32), ("pdl", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("us_per_step", ctypes.c_float)]


# symbol name -> (restype, argtypes)
_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p
SIGNATURES = {
    "iontrap_create": (ctypes.c_int, [ctypes.POINTER(iontrap_species), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_uint8), _dp, _dp, ctypes.c_int64,
                                      ctypes.POINTER(iontrap_params), ctypes.c_int64, _vp,
                                      ctypes.POINTER(_vp)]),
    "iontrap_step": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "iontrap_sync": (ctypes.c_int, [_vp]),
    "iontrap_set_pseudo_frequencies": (ctypes.c_int, [_vp, _dp]),
    "iontrap_minimize": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        _i64p, _dp]),
    "iontrap_hessian": (ctypes.c_int, [_vp, _dp]),
    "iontrap_step_record": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int64, _vp]),
    "iontrap_set_params": (ctypes.c_int, [_vp, ctypes.POINTER(iontrap_params), ctypes.POINTER(iontrap_cooling)]),
    "iontrap_state": (ctypes.c_int, [_vp, _dp, _dp, _i64p, _dp]),
    "iontrap_forces": (ctypes.c_int, [_vp, _dp]),
    "iontrap_checkpoint": (ctypes.c_int, [_vp, _dp, _dp, _dp, _i64p]),
    "iontrap_restore": (ctypes.c_int, [_vp, _dp, _dp, _dp, ctypes.c_int64]),
    "iontrap_step_many": (ctypes.c_int, [ctypes.POINTER(_vp), _i64p, ctypes.c_int]),
    "iontrap_destroy": (None, [_vp]),
    "iontrap_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "iontrap_stable": (ctypes.c_int, [ctypes.POINTER(iontrap_species), ctypes.c_int,
                                      ctypes.POINTER(iontrap_params), _ip]),
    "iontrap_linear_pt": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.POINTER(iontrap_species),
                                         ctypes.POINTER(iontrap_params)]),
    "iontrap_normals": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int64, _i64p, ctypes.c_int64,
                                       ctypes.c_int, _dp]),
    "iontrap_get_config": (ctypes.c_int, [_vp, ctypes.POINTER(iontrap_config)]),
    "iontrap_set_config": (ctypes.c_int, [_vp, ctypes.POINTER(iontrap_config)]),
    "iontrap_default_config": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.c_uint32, ctypes.c_int,
                                              ctypes.POINTER(iontrap_config)]),
    "iontrap_forces_noalloc": (ctypes.c_int, [ctypes.POINTER(iontrap_species), ctypes.c_int, _vp, _vp,
                                              ctypes.c_int64, _vp, _vp]),
    "iontrap_device_bytes": (ctypes.c_int, [_vp, _i64p]),
    "iontrap_autotune": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.POINTER(iontrap_config), _dp]),
    "iontrap_autotune_many": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_double]),
    "iontrap_tuning_get": (ctypes.c_int, [ctypes.POINTER(iontrap_tuning_entry), ctypes.c_int, _ip]),
    "iontrap_tuning_put": (ctypes.c_int, [ctypes.POINTER(iontrap_tuning_entry), ctypes.c_int]),
    "iontrap_estimate_bytes": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, _i64p]),
    "iontrap_server_create": (ctypes.c_int, [ctypes.POINTER(iontrap_server_config), ctypes.POINTER(_vp)]),
    "iontrap_server_submit": (ctypes.c_int, [_vp, ctypes.POINTER(iontrap_species), ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_uint8), _dp, _dp, ctypes.c_int64,
                                             ctypes.POINTER(iontrap_params), ctypes.c_int64, _i64p]),
    "iontrap_server_poll": (ctypes.c_int, [_vp, _i64p, ctypes.c_int64, _i64p]),
    "iontrap_server_result": (ctypes.c_int, [_vp, ctypes.c_int64, _dp, _dp, _i64p, _ip]),
    "iontrap_server_stats": (ctypes.c_int, [_vp, ctypes.POINTER(iontrap_server_counters)]),
    "iontrap_server_destroy": (None, [_vp]),
    "iontrap_trace_step": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int64, _i64p, _i64p]),
    "iontrap_test_stall": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64]),
    "iontrap_alu_probe": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_longlong, _dp, _dp]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libiontrap.so is not built ({LIB_PATH}); run "
                          "`python -c \"import __graft_entry__ as g; g.build()\"`")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


class IonTrapError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = int(code)
        super().__init__(f"{where}: status {code} ({iontrap_strerror(code)})")


def _check(code: int, where: str) -> None:
    if code != IONTRAP_OK:
        raise IonTrapError(code, where)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _species_array(species: Sequence) -> ctypes.Array:
    arr = (iontrap_species * len(species))()
    for k, s in enumerate(species):
        if isinstance(s, (tuple, list)):
            arr[k].mass_amu, arr[k].charge_e = float(s[0]), float(s[1])
        else:
            arr[k].mass_amu, arr[k].charge_e = float(s.mass_amu), float(s.charge_e)
    return arr


def make_params(trap=None, precision: int = IONTRAP_PREC_FP32, flags: Optional[int] = None,
                **kw) -> iontrap_params:
    """Build an ``iontrap_params`` from an object with Omega, a, q, omega_z, gamma,
    T_bath, dt, seed (and optionally flags) attributes, overridden by keywords."""
    p = iontrap_params()
    src = {}
    if trap is not None:
        for f in ("Omega", "a", "q", "omega_z", "gamma", "T_bath", "dt", "seed", "flags"):
            if hasattr(trap, f):
                src[f] = getattr(trap, f)
    src.update(kw)
    for f in ("Omega", "a", "q", "omega_z", "gamma", "T_bath", "dt"):
        setattr(p, f, float(src.get(f, 0.0)))
    p.seed = int(src.get("seed", 0)) & (2**64 - 1)
    p.flags = int(src.get("flags", 0) if flags is None else flags)
    p.precision = int(precision)
    return p


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream) or None
    return int(stream) or None


# ------------------------------------------------------------------ entry points

def iontrap_strerror(code: int) -> str:
    return _lib.iontrap_strerror(int(code)).decode()


def iontrap_create(species: Sequence, species_of_ion, x0, v0=None,
                   params: Optional[iontrap_params] = None, step0: int = 0, stream=None):
    """Returns an opaque handle (ctypes.c_void_p)."""
    sp = np.ascontiguousarray(species_of_ion, dtype=np.uint8)
    n = sp.shape[0]
    x = _f64(x0).reshape(3, n)
    v = None if v0 is None else _f64(v0).reshape(3, n)
    spa = _species_array(species)
    h = ctypes.c_void_p()
    st = _lib.iontrap_create(spa, len(species), sp.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                             _ptr(x), None if v is None else _ptr(v), n,
                             ctypes.byref(params if params is not None else iontrap_params()),
                             int(step0), _stream_ptr(stream), ctypes.byref(h))
    _check(st, "iontrap_create")
    return h


def iontrap_step(h, n_steps: int) -> None:
    _check(_lib.iontrap_step(h, int(n_steps)), "iontrap_step")


def _cooling_array(cooling) -> Optional[ctypes.Array]:
    """One iontrap_cooling per species from objects with gamma, T_bath and laser
    attributes (or (gamma, T_bath, laser) tuples); None passes NULL."""
    if cooling is None:
        return None
    arr = (iontrap_cooling * len(cooling))()
    for k, c in enumerate(cooling):
        g, T, L = (c.gamma, c.T_bath, c.laser) if hasattr(c, "gamma") else c
        arr[k].gamma, arr[k].T_bath = float(g), float(T)
        for d in range(3):
            arr[k].laser[d] = float(L[d])
    return arr


def iontrap_set_params(h, params: iontrap_params, cooling=None) -> None:
    """Change the trap and the per-species cooling between evolve calls."""
    _check(_lib.iontrap_set_params(h, ctypes.byref(params), _cooling_array(cooling)), "iontrap_set_params")


def iontrap_set_pseudo_frequencies(h, omega=None) -> None:
    """Per-species secular angular frequencies (n_species x 3, rad/s) of the
    pseudopotential trap, or None for Eq. 2."""
    w = None if omega is None else _f64(omega).reshape(-1)
    _check(_lib.iontrap_set_pseudo_frequencies(h, None if w is None else _ptr(w)),
           "iontrap_set_pseudo_frequencies")


def iontrap_minimize(h, max_iters: int, dmax: float, ftol: float, dt: float = 0.0):
    """Damped minimisation of the static potential; returns (iterations, |F|)."""
    it_ = ctypes.c_int64()
    fn = ctypes.c_double()
    _check(_lib.iontrap_minimize(h, int(max_iters), float(dt), float(dmax), float(ftol), ctypes.byref(it_),
                                 ctypes.byref(fn)), "iontrap_minimize")
    return it_.value, fn.value


def iontrap_hessian(h, n: int) -> np.ndarray:
    """Mass-weighted Hessian (3n x 3n) of the static potential at the current state."""
    H = np.empty((3 * n, 3 * n))
    _check(_lib.iontrap_hessian(h, _ptr(H)), "iontrap_hessian")
    return H


def iontrap_step_record(h, n_steps: int, every: int, fields: int, avg_steps: int, d_out: int) -> None:
    """Enqueue n_steps steps with a record every ``every`` steps written to the device
    array at address d_out ((n_steps // every) x fields x 3 x n doubles)."""
    _check(_lib.iontrap_step_record(h, int(n_steps), int(every), int(fields), int(avg_steps), ctypes.c_void_p(d_out)),
           "iontrap_step_record")


def iontrap_sync(h) -> None:
    _check(_lib.iontrap_sync(h), "iontrap_sync")


def iontrap_state(h, n: int, x_out: Optional[np.ndarray] = None, v_out: Optional[np.ndarray] = None,
                  accept=()):
    """Returns (x, v, step, t); x and v are (3, n) float64 arrays.  Statuses listed in
    ``accept`` (e.g. IONTRAP_ETIMEOUT after a failed launch) do not raise."""
    x = np.empty((3, n)) if x_out is None else x_out
    v = np.empty((3, n)) if v_out is None else v_out
    step = ctypes.c_int64()
    t = ctypes.c_double()
    code = _lib.iontrap_state(h, _ptr(x), _ptr(v), ctypes.byref(step), ctypes.byref(t))
    if code not in accept:
        _check(code, "iontrap_state")
    return x, v, int(step.value), float(t.value)


def iontrap_test_stall(h, wait_limit_ns: int, cta: int, step: int) -> None:
    _check(_lib.iontrap_test_stall(h, int(wait_limit_ns), int(cta), int(step)), "iontrap_test_stall")


def iontrap_forces(h, n: int) -> np.ndarray:
    acc = np.empty((3, n))
    _check(_lib.iontrap_forces(h, _ptr(acc)), "iontrap_forces")
    return acc


def iontrap_checkpoint(h, n: int):
    """Returns (x, v, a, step) of the current state."""
    x, v, a = np.empty((3, n)), np.empty((3, n)), np.empty((3, n))
    step = ctypes.c_int64()
    _check(_lib.iontrap_checkpoint(h, _ptr(x), _ptr(v), _ptr(a), ctypes.byref(step)), "iontrap_checkpoint")
    return x, v, a, int(step.value)


def iontrap_restore(h, x, v, a, step: int) -> None:
    x, v, a = _f64(x), _f64(v), _f64(a)
    _check(_lib.iontrap_restore(h, _ptr(x), _ptr(v), _ptr(a), int(step)), "iontrap_restore")


def iontrap_step_many(handles: Sequence, n_steps: Sequence[int]) -> None:
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h
                                             for h in handles])
    ns = np.ascontiguousarray(n_steps, dtype=np.int64)
    _check(_lib.iontrap_step_many(arr, ns.ctypes.data_as(_i64p), len(handles)), "iontrap_step_many")


def iontrap_destroy(h) -> None:
    _lib.iontrap_destroy(h)


def iontrap_stable(species: Sequence, params: iontrap_params) -> bool:
    ok = ctypes.c_int()
    _check(_lib.iontrap_stable(_species_array(species), len(species), ctypes.byref(params),
                               ctypes.byref(ok)), "iontrap_stable")
    return bool(ok.value)


def iontrap_linear_pt(V0: float, U0: float, R0: float, Z0: float, kappa: float, Omega: float, species0,
                      params: Optional[iontrap_params] = None) -> iontrap_params:
    """Fill Omega, a, q, omega_z of ``params`` (a new one if None) from the voltages
    and geometry of a linear Paul trap; returns the params."""
    p = params if params is not None else iontrap_params()
    _check(_lib.iontrap_linear_pt(float(V0), float(U0), float(R0), float(Z0), float(kappa), float(Omega),
                                  _species_array([species0]), ctypes.byref(p)), "iontrap_linear_pt")
    return p


def iontrap_normals(seed: int, counter: int, ids, precision: int = IONTRAP_PREC_FP32) -> np.ndarray:
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    z = np.empty((3, len(ids)))
    _check(_lib.iontrap_normals(int(seed) & (2**64 - 1), int(counter), ids.ctypes.data_as(_i64p),
                                len(ids), int(precision), _ptr(z)), "iontrap_normals")
    return z


def iontrap_get_config(h):
    """Returns (threads, ions_per_thread, packed, jsplit, fused, pdl, graph)."""
    c = iontrap_config()
    _check(_lib.iontrap_get_config(h, ctypes.byref(c)), "iontrap_get_config")
    return c.threads, c.ions_per_thread, c.packed, c.jsplit, c.fused, c.pdl, c.graph


def iontrap_default_config(n: int, precision: int = IONTRAP_PREC_FP32, flags: int = 0,
                           allow_persistent: int = 1):
    """Returns (threads, ions_per_thread, packed, jsplit, fused, pdl, graph)."""
    c = iontrap_config()
    _check(_lib.iontrap_default_config(int(n), int(precision), int(flags), int(allow_persistent), ctypes.byref(c)),
           "iontrap_default_config")
    return c.threads, c.ions_per_thread, c.packed, c.jsplit, c.fused, c.pdl, c.graph


def iontrap_set_config(h, threads: int, ions_per_thread: int, packed: int, jsplit: int, fused: int = 1,
                       pdl: int = 1, graph: int = 1) -> None:
    c = iontrap_config(int(threads), int(ions_per_thread), int(packed), int(jsplit), int(fused), int(pdl),
                       int(graph))
    _check(_lib.iontrap_set_config(h, ctypes.byref(c)), "iontrap_set_config")


def iontrap_forces_noalloc(species: Sequence, d_species_of_ion: int, d_x: int, n: int, d_acc: int,
                           stream=None) -> None:
    """Device-pointer, allocation-free Coulomb accelerations (see include/iontrap.h).
    d_species_of_ion, d_x and d_acc are device addresses (e.g. tensor.data_ptr())."""
    _check(_lib.iontrap_forces_noalloc(_species_array(species), len(species), int(d_species_of_ion), int(d_x),
                                       int(n), int(d_acc), _stream_ptr(stream)), "iontrap_forces_noalloc")


def iontrap_device_bytes(h) -> int:
    b = ctypes.c_int64()
    _check(_lib.iontrap_device_bytes(h, ctypes.byref(b)), "iontrap_device_bytes")
    return b.value


def iontrap_autotune(h, trial_us: float = 3000.0):
    """Returns ((threads, ions_per_thread, packed, jsplit, fused, pdl, graph), us_per_step)."""
    c = iontrap_config()
    us = ctypes.c_double()
    _check(_lib.iontrap_autotune(h, float(trial_us), ctypes.byref(c), ctypes.byref(us)), "iontrap_autotune")
    return (c.threads, c.ions_per_thread, c.packed, c.jsplit, c.fused, c.pdl, c.graph), us.value


def iontrap_autotune_many(handles: Sequence, trial_us: float = 3000.0) -> None:
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h
                                             for h in handles])
    _check(_lib.iontrap_autotune_many(arr, len(handles), float(trial_us)), "iontrap_autotune_many")


_TUNE_FIELDS = [f for f, _ in iontrap_tuning_entry._fields_]


def iontrap_tuning_get():
    """The current device's tuning table as a list of dicts."""
    cnt = ctypes.c_int()
    _check(_lib.iontrap_tuning_get(None, 0, ctypes.byref(cnt)), "iontrap_tuning_get")
    arr = (iontrap_tuning_entry * max(1, cnt.value))()
    _check(_lib.iontrap_tuning_get(arr, cnt.value, ctypes.byref(cnt)), "iontrap_tuning_get")
    return [{f: getattr(arr[k], f) for f in _TUNE_FIELDS} for k in range(cnt.value)]


def iontrap_tuning_put(entries) -> None:
    arr = (iontrap_tuning_entry * max(1, len(entries)))()
    for k, e in enumerate(entries):
        for f in _TUNE_FIELDS:
            setattr(arr[k], f, e[f])
    _check(_lib.iontrap_tuning_put(arr, len(entries)), "iontrap_tuning_put")


def iontrap_estimate_bytes(n: int, precision: int = IONTRAP_PREC_FP32) -> int:
    b = ctypes.c_int64()
    _check(_lib.iontrap_estimate_bytes(int(n), int(precision), ctypes.byref(b)), "iontrap_estimate_bytes")
    return b.value


def iontrap_server_create(mem_budget_bytes: int = 0, max_resident: int = 0, chunk_steps: int = 0,
                          max_parallel: int = 0):
    cfg = iontrap_server_config(int(mem_budget_bytes), int(max_resident), int(chunk_steps), int(max_parallel))
    s = ctypes.c_void_p()
    _check(_lib.iontrap_server_create(ctypes.byref(cfg), ctypes.byref(s)), "iontrap_server_create")
    return s


def iontrap_server_submit(s, species, species_of_ion, x0, v0, params: iontrap_params, n_steps: int) -> int:
    sp = np.ascontiguousarray(species_of_ion, dtype=np.uint8)
    n = sp.shape[0]
    x = _f64(x0).reshape(3, n)
    v = None if v0 is None else _f64(v0).reshape(3, n)
    rid = ctypes.c_int64()
    _check(_lib.iontrap_server_submit(s, _species_array(species), len(species),
                                      sp.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _ptr(x),
                                      None if v is None else _ptr(v), n, ctypes.byref(params), int(n_steps),
                                      ctypes.byref(rid)), "iontrap_server_submit")
    return rid.value


def iontrap_server_poll(s, cap: int = 4096):
    ids = np.empty(cap, dtype=np.int64)
    k = ctypes.c_int64()
    _check(_lib.iontrap_server_poll(s, ids.ctypes.data_as(_i64p), cap, ctypes.byref(k)), "iontrap_server_poll")
    return ids[:min(k.value, cap)].tolist()


def iontrap_server_result(s, rid: int, n: int):
    """Returns (x, v, step, status) of a completed request and releases it."""
    x, v = np.empty((3, n)), np.empty((3, n))
    step, status = ctypes.c_int64(), ctypes.c_int()
    _check(_lib.iontrap_server_result(s, int(rid), _ptr(x), _ptr(v), ctypes.byref(step), ctypes.byref(status)),
           "iontrap_server_result")
    return x, v, step.value, status.value


def iontrap_server_stats(s):
    st = iontrap_server_counters()
    _check(_lib.iontrap_server_stats(s, ctypes.byref(st)), "iontrap_server_stats")
    return {"waiting": st.waiting, "resident": st.resident, "completed": st.completed,
            "device_bytes": st.device_bytes}


def iontrap_server_destroy(s) -> None:
    _lib.iontrap_server_destroy(s)


def iontrap_trace_step(h, cap: int = 1 << 22):
    """One traced step: returns (force_marks (k, 4), epilogue_marks (m, 2)) in ns."""
    buf = np.zeros(cap, dtype=np.uint64)
    nf, ne = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.iontrap_trace_step(h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_ulonglong)), cap,
                                   ctypes.byref(nf), ctypes.byref(ne)), "iontrap_trace_step")
    return buf[:nf.value].reshape(-1, 4), buf[nf.value:nf.value + ne.value].reshape(-1, 2)


def iontrap_alu_probe(kind: int, iters: int = 20000):
    """Returns (lane operations per SM clock, SM MHz) for one instruction kind."""
    ops, mhz = ctypes.c_double(), ctypes.c_double()
    _check(_lib.iontrap_alu_probe(int(kind), int(iters), ctypes.byref(ops), ctypes.byref(mhz)),
           "iontrap_alu_probe")
    return ops.value, mhz.value


class Simulation:
    """Owning wrapper of a handle (closes it on ``close()`` / context exit)."""

    def __init__(self, species, species_of_ion, x0, v0=None, params=None, step0=0, stream=None):
        self.n = int(np.asarray(species_of_ion).shape[0])
        self.handle = iontrap_create(species, species_of_ion, x0, v0, params, step0, stream)

    def step(self, n_steps: int) -> "Simulation":
        iontrap_step(self.handle, n_steps)
        return self

    def sync(self) -> None:
        iontrap_sync(self.handle)

    def set_params(self, params, cooling=None) -> None:
        iontrap_set_params(self.handle, params, cooling)

    def set_pseudo_frequencies(self, omega=None) -> None:
        iontrap_set_pseudo_frequencies(self.handle, omega)

    def minimize(self, max_iters: int, dmax: float, ftol: float, dt: float = 0.0):
        return iontrap_minimize(self.handle, max_iters, dmax, ftol, dt)

    def hessian(self) -> np.ndarray:
        return iontrap_hessian(self.handle, self.n)

    def step_record(self, n_steps: int, every: int, fields: int, avg_steps: int, d_out: int) -> "Simulation":
        iontrap_step_record(self.handle, n_steps, every, fields, avg_steps, d_out)
        return self

    def state(self):
        return iontrap_state(self.handle, self.n)

    def forces(self) -> np.ndarray:
        return iontrap_forces(self.handle, self.n)

    def checkpoint(self):
        return iontrap_checkpoint(self.handle, self.n)

    def restore(self, x, v, a, step: int) -> None:
        iontrap_restore(self.handle, x, v, a, step)

    def config(self):
        return iontrap_get_config(self.handle)

    def autotune(self, trial_us: float = 3000.0):
        return iontrap_autotune(self.handle, trial_us)

    def set_config(self, threads, ions_per_thread, packed, jsplit, fused=1, pdl=1, graph=1) -> None:
        iontrap_set_config(self.handle, threads, ions_per_thread, packed, jsplit, fused, pdl, graph)

    def close(self) -> None:
        if self.handle is not None:
            iontrap_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
