"""FP64 CPU oracle of the trapped-ion timestep -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import this package.  The product library never calls it and shares
no code with it: the arithmetic lives in ``iontrap_oracle.c`` (plain C, FP64, OpenMP
over ions), this module only compiles it with gcc and marshals numpy arrays.

Functions follow the paper:
  * ``coulomb_accel``  -- direct-sum Coulomb acceleration, Eq. 4 / Sec. 6 "Interactions"
  * ``trap_accel``     -- linear Paul trap field, Eq. 1 in the Mathieu form of Eq. 3
  * ``normals``        -- Langevin kicks (Sec. 3, "Cooling the motion of ions") from
                          Philox-4x64-10 + Box-Muller
  * ``cooling_arrays`` -- per-species baths and laser cooling (Sec. 3, langevinBath
                          on a group, laserCool) as per-ion arrays for ``accel``/``run``
  * ``linear_pt``      -- Mathieu parameters of a trap given by voltages (Eq. 3)
  * ``pseudo_springs`` -- the pseudopotential of the trap (Eq. 2); ``springs_arrays``
                          a pseudopotential trap given by per-species frequencies
  * ``record``         -- dump and timeAvg (Sec. 3 "Writing/reading data"): strided
                          states and windowed velocity averages, summed step by step
  * ``minimize``       -- damped minimisation of the static potential (Sec. 3)
  * ``hessian``        -- mass-weighted Hessian whose eigenvalues are the squared
                          normal-mode frequencies (Sec. 5 "Normal modes of motion")
  * ``run``            -- velocity-Verlet time evolution (Sec. 6 "Integration", "nve")
  * ``energy``         -- Eq. 4 energy for a static trap
  * ``stable``         -- discrete-Verlet Floquet stability of a single ion (|tr M| < 2)

Every one of these is pinned by ``tests/test_oracle_pins.py`` against closed forms,
invariants or a library routine (numpy's Philox).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "iontrap_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

RF_OFF = 1
COULOMB_OFF = 2
TRAP_OFF = 4
PSEUDO = 16  # the trap is its Eq. 2 pseudopotential (static springs)


class _Params(ctypes.Structure):
    _fields_ = [("Omega", ctypes.c_double), ("a", ctypes.c_double), ("q", ctypes.c_double),
                ("omega_z", ctypes.c_double), ("gamma", ctypes.c_double),
                ("T_bath", ctypes.c_double), ("dt", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("pad_", ctypes.c_uint32), ("qm_ref", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) into oracle/_build."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _SO + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-std=c11",
                                   "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        pp = ctypes.POINTER(_Params)
        L.oracle_const.restype = ctypes.c_double
        L.oracle_const.argtypes = [ctypes.c_int]
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_threads.restype = ctypes.c_int
        L.oracle_philox4x64_10.argtypes = [u64p, u64p, u64p]
        L.oracle_normals_many.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, i64p, dp]
        L.oracle_coulomb_accel.argtypes = [ctypes.c_int64, dp, dp, dp, i64p, ctypes.c_int64, dp]
        L.oracle_trap_accel.argtypes = [pp, ctypes.c_double, dp, ctypes.c_double, dp]
        L.oracle_accel.argtypes = [ctypes.c_int64, dp, dp, dp, dp, pp, ctypes.c_int64,
                                   ctypes.c_double, dp]
        L.oracle_run.argtypes = [ctypes.c_int64, dp, dp, dp, dp, dp, pp, ctypes.c_int64,
                                 ctypes.c_int64, ctypes.c_int, dp]
        L.oracle_accel_ex.argtypes = [ctypes.c_int64, dp, dp, dp, dp, pp, ctypes.c_int64,
                                      ctypes.c_double, dp, dp, dp, dp, dp]
        L.oracle_run_ex.argtypes = [ctypes.c_int64, dp, dp, dp, dp, dp, pp, ctypes.c_int64,
                                    ctypes.c_int64, ctypes.c_int, dp, dp, dp, dp, dp]
        L.oracle_energy.restype = ctypes.c_double
        L.oracle_energy.argtypes = [ctypes.c_int64, dp, dp, dp, dp, pp]
        L.oracle_energy_ex.restype = ctypes.c_double
        L.oracle_energy_ex.argtypes = [ctypes.c_int64, dp, dp, dp, dp, pp, dp]
        L.oracle_pseudo_springs.argtypes = [pp, ctypes.c_double, dp]
        L.oracle_hessian.argtypes = [ctypes.c_int64, dp, dp, dp, pp, dp, dp]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def const(name: str) -> float:
    return lib().oracle_const({"e": 0, "kB": 1, "eps0": 2, "amu": 3, "ke": 4}[name])


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def threads() -> int:
    return int(lib().oracle_threads())


# ------------------------------------------------------------------ per-ion inputs

def ion_arrays(species: Sequence, species_of_ion: np.ndarray):
    """Charge (C) and mass (kg) per ion, and the reference charge/mass (species 0)."""
    e, amu = const("e"), const("amu")
    q_s = np.array([s.charge_e * e for s in species])
    m_s = np.array([s.mass_amu * amu for s in species])
    sp = np.asarray(species_of_ion, dtype=np.int64)
    return _c64(q_s[sp]), _c64(m_s[sp]), float(q_s[0] / m_s[0])


def params(trap, qm_ref: float, flags: Optional[int] = None) -> _Params:
    p = _Params()
    p.Omega, p.a, p.q, p.omega_z = trap.Omega, trap.a, trap.q, trap.omega_z
    p.gamma, p.T_bath = trap.gamma, trap.T_bath
    p.dt = trap.dt if trap.dt > 0 else 2.0 * math.pi / trap.Omega / 20.0
    p.seed = int(trap.seed) & (2**64 - 1)
    p.flags = int(trap.flags if flags is None else flags)
    p.qm_ref = qm_ref
    return p


# ------------------------------------------------------------------------ wrappers

def philox4x64(ctr: np.ndarray, key: Sequence[int]) -> np.ndarray:
    """Philox-4x64-10 blocks for each row of ``ctr`` (m, 4) uint64."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint64).reshape(-1, 4)
    k = np.array(key, dtype=np.uint64)
    out = np.empty_like(ctr)
    L = lib()
    u64p = ctypes.POINTER(ctypes.c_uint64)
    for r in range(ctr.shape[0]):
        L.oracle_philox4x64_10(ctr[r].ctypes.data_as(u64p), k.ctypes.data_as(u64p),
                               out[r].ctypes.data_as(u64p))
    return out


def normals(seed: int, counter: int, ids) -> np.ndarray:
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    z = np.empty((3, len(ids)))
    lib().oracle_normals_many(ctypes.c_uint64(int(seed) & (2**64 - 1)), int(counter), len(ids),
                              ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(z))
    return z


def coulomb_accel(x: np.ndarray, charge: np.ndarray, mass: np.ndarray, idx=None) -> np.ndarray:
    x = _c64(x)
    n = x.shape[1]
    if idx is None:
        m, ip = n, None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        m, ip = len(idx), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    acc = np.empty((3, m))
    lib().oracle_coulomb_accel(n, _dp(x), _dp(_c64(charge)), _dp(_c64(mass)), ip, m, _dp(acc))
    return acc


def trap_accel(p: _Params, qm: float, r, t: float) -> np.ndarray:
    r = _c64(r)
    out = np.empty(3)
    lib().oracle_trap_accel(ctypes.byref(p), qm, _dp(r), t, _dp(out))
    return out


def cooling_arrays(species_of_ion, coolings):
    """Per-ion cooling arrays (gamma[n], T_bath[n], laser[3][n]) from one cooling
    description per species (objects with ``gamma``, ``T_bath`` and ``laser``): a bath or
    laser applied to a species applies to every ion of it (Sec. 3, langevinBath(T,
    dampingTime, group) and laserCool(species, gamma))."""
    sp = np.asarray(species_of_ion, dtype=np.int64)
    g = np.array([float(c.gamma) for c in coolings])
    T = np.array([float(c.T_bath) for c in coolings])
    L = np.array([[float(u) for u in c.laser] for c in coolings]).reshape(-1, 3)
    return _c64(g[sp]), _c64(T[sp]), _c64(L[sp].T)


def _cool_ptrs(cooling):
    if cooling is None:
        return None, None, None, ()
    g, T, L = (_c64(a) for a in cooling)
    return _dp(g), _dp(T), _dp(L), (g, T, L)


def _opt(a):
    if a is None:
        return None, None
    a = _c64(a)
    return _dp(a), a


def pseudo_springs(p: _Params, qm: float) -> np.ndarray:
    """Spring constants (1/s^2) of the Eq. 2 pseudopotential for charge/mass qm."""
    k = np.empty(3)
    lib().oracle_pseudo_springs(ctypes.byref(p), float(qm), _dp(k))
    return k


def springs_arrays(species_of_ion, omegas) -> np.ndarray:
    """Per-ion spring constants [3][n] from secular angular frequencies (wx, wy, wz)
    given per species -- a pseudopotential trap per species (linearPseudoPT, Sec. 3)."""
    w = np.asarray(omegas, dtype=np.float64).reshape(-1, 3)
    sp = np.asarray(species_of_ion, dtype=np.int64)
    return _c64((w[sp] ** 2).T)


def accel(x, udrag, charge, mass, p: _Params, counter: int, t: float, cooling=None,
          springs=None) -> np.ndarray:
    """Acceleration of every ion; ``cooling`` = (gamma[n], T_bath[n], laser[3][n]) per
    ion (see ``cooling_arrays``), or None for the bath of ``p`` and no laser; ``springs``
    = per-ion static springs [3][n] replacing the trap (see ``springs_arrays``)."""
    x, udrag = _c64(x), _c64(udrag)
    acc = np.empty_like(x)
    gp, tp, lp, keep = _cool_ptrs(cooling)
    sp_, keep2 = _opt(springs)
    lib().oracle_accel_ex(x.shape[1], _dp(x), _dp(udrag), _dp(_c64(charge)), _dp(_c64(mass)),
                          ctypes.byref(p), int(counter), float(t), gp, tp, lp, sp_, _dp(acc))
    del keep, keep2
    return acc


def run(x0, v0, charge, mass, p: _Params, nsteps: int, step0: int = 0, a0=None, cooling=None,
        springs=None):
    """Velocity-Verlet evolution.  Returns (x, v, a) after ``nsteps`` steps.  With
    ``a0`` None the initial acceleration is evaluated first (at t = step0 dt, drag on
    v0, noise counter step0) -- which is also how the forces change between two runs
    (interleaved evolve, Sec. 3 "Time evolution").  ``cooling`` and ``springs`` as for
    ``accel``."""
    x, v = _c64(x0).copy(), _c64(v0).copy()
    n = x.shape[1]
    a = np.zeros_like(x) if a0 is None else _c64(a0).copy()
    work = np.empty_like(x)
    gp, tp, lp, keep = _cool_ptrs(cooling)
    sp_, keep2 = _opt(springs)
    lib().oracle_run_ex(n, _dp(x), _dp(v), _dp(a), _dp(_c64(charge)), _dp(_c64(mass)),
                        ctypes.byref(p), int(step0), int(nsteps), int(a0 is None), gp, tp, lp, sp_,
                        _dp(work))
    del keep, keep2
    return x, v, a


def record(x0, v0, charge, mass, p: _Params, nsteps: int, every: int, avg_steps: int, step0: int = 0,
           a0=None, cooling=None, springs=None):
    """Evolve like ``run`` and record, after every ``every`` steps (dump, Sec. 3
    "Writing/reading data"), the positions, the velocities and the time average of the
    full-step velocities over the last ``avg_steps`` steps (timeAvg), summed step by step.
    Returns (X, V, VAVG), each (nsteps // every, 3, n), and the final (x, v, a)."""
    x, v = _c64(x0).copy(), _c64(v0).copy()
    a = a0
    X, V, VA = [], [], []
    step = step0
    for _ in range(int(nsteps) // int(every)):
        if every > avg_steps:
            x, v, a = run(x, v, charge, mass, p, every - avg_steps, step0=step, a0=a, cooling=cooling,
                          springs=springs)
            step += every - avg_steps
        elif a is None:
            x, v, a = run(x, v, charge, mass, p, 0, step0=step, cooling=cooling, springs=springs)
        vsum = np.zeros_like(x)
        for _k in range(int(avg_steps)):
            x, v, a = run(x, v, charge, mass, p, 1, step0=step, a0=a, cooling=cooling, springs=springs)
            step += 1
            vsum += v
        X.append(x.copy())
        V.append(v.copy())
        VA.append(vsum / avg_steps)
    return np.array(X), np.array(V), np.array(VA), (x, v, a)


def minimize(x0, charge, mass, p: _Params, dt: float, dmax: float, ftol: float, max_steps: int,
             springs=None):
    """Damped dynamics toward the minimum of the static potential (Sec. 3
    "Minimisation": the equations of motion are damped to extract energy, and the distance
    an ion may move in one step is limited).  The trap must be static (the pseudopotential
    of Eq. 2, ``springs``, or RF off); no bath acts.  Starting at rest, every step:
      1. a = acceleration at x (trap + Coulomb), F_i = M_i a_i; stop if |F| < ftol
         (2-norm over all ions and components);
      2. the velocity keeps only its component along the force, v = (v.F / F.F) F, and is
         set to zero when v.F <= 0 (moving uphill);
      3. v += dt a; the displacement d = dt v is scaled (with v) by
         min(1, dmax / max_i |d_i|), so no ion moves more than dmax; x += d.
    Returns (x, steps taken, |F| at the last evaluation)."""
    x = _c64(x0).copy()
    mass = _c64(mass)
    v = np.zeros_like(x)
    zero = np.zeros_like(x)
    fn = math.inf
    p = _Params.from_buffer_copy(p)
    p.gamma, p.T_bath = 0.0, 0.0  # no bath acts during minimisation
    for k in range(int(max_steps)):
        a = accel(x, zero, charge, mass, p, 0, 0.0, springs=springs)
        F = mass[None, :] * a
        FF = float((F * F).sum())
        fn = math.sqrt(FF)
        if fn < ftol:
            return x, k, fn
        vF = float((v * F).sum())
        v = (vF / FF) * F if vF > 0.0 else np.zeros_like(x)
        v = v + dt * a
        d = dt * v
        dm = float(np.sqrt((d * d).sum(axis=0)).max())
        s = min(1.0, dmax / dm) if dm > 0.0 else 1.0
        v = s * v
        x = x + s * d
    return x, int(max_steps), fn


def hessian(x, charge, mass, p: _Params, springs=None) -> np.ndarray:
    """Mass-weighted Hessian (3n x 3n, row/column 3i+a) of the static potential at x:
    trap springs (``springs`` or the Eq. 2 pseudopotential of ``p``) plus the Coulomb pair
    energy.  Its eigenvalues are the squared normal-mode angular frequencies (Sec. 5)."""
    x = _c64(x)
    n = x.shape[1]
    H = np.empty((3 * n, 3 * n))
    sp_, keep = _opt(springs)
    lib().oracle_hessian(n, _dp(x), _dp(_c64(charge)), _dp(_c64(mass)), ctypes.byref(p), sp_, _dp(H))
    del keep
    return H


def energy(x, v, charge, mass, p: _Params, springs=None) -> float:
    x, v = _c64(x), _c64(v)
    sp_, keep = _opt(springs)
    e = float(lib().oracle_energy_ex(x.shape[1], _dp(x), _dp(v), _dp(_c64(charge)),
                                     _dp(_c64(mass)), ctypes.byref(p), sp_))
    del keep
    return e


def linear_pt(V0: float, U0: float, R0: float, Z0: float, kappa: float, Omega: float,
              charge_c: float, mass_kg: float):
    """Trap parameters (Omega, a, q, omega_z) of the oracle's trap for a linear Paul trap
    given by voltages and geometry (linearPT, Sec. 3 "Forces and fields").  Eq. 3:
    q_x = 2 Q V0 / (M R0^2 Omega^2) and a_z = 8 Q kappa U0 / (M Z0^2 Omega^2); the static
    axial frequency follows from a_z as omega_z = (Omega/2) sqrt(a_z).  The radial a_x =
    -a_z/2 of Eq. 3 is the axial field's defocusing, which the trap of this oracle already
    contains through omega_z, so the extra a is 0."""
    q = 2.0 * charge_c * V0 / (mass_kg * R0 ** 2 * Omega ** 2)
    a_z = 8.0 * charge_c * kappa * U0 / (mass_kg * Z0 ** 2 * Omega ** 2)
    return Omega, 0.0, q, Omega / 2.0 * math.sqrt(a_z)


# ------------------------------------------------------------------- stability

def _kdk_period_matrix(k_of_t, dt: float, steps: int) -> np.ndarray:
    """Product of the kick-drift-kick step matrices of x'' = -k(t) x over ``steps``."""
    M = np.eye(2)
    for s in range(steps):
        k0, k1 = k_of_t(s * dt), k_of_t((s + 1) * dt)
        kick0 = np.array([[1.0, 0.0], [-0.5 * dt * k0, 1.0]])
        drift = np.array([[1.0, dt], [0.0, 1.0]])
        kick1 = np.array([[1.0, 0.0], [-0.5 * dt * k1, 1.0]])
        M = kick1 @ drift @ kick0 @ M
    return M


def _mathieu_monodromy(k_of_t, T: float, sub: int = 4096) -> np.ndarray:
    """RK4 monodromy of x'' = -k(t) x over one period (continuous reference)."""
    h = T / sub
    M = np.eye(2)
    for s in range(sub):
        t = s * h

        def f(tt, y):
            return np.array([y[1], -k_of_t(tt) * y[0]])

        for col in range(2):
            y = M[:, col]
            k1 = f(t, y)
            k2 = f(t + h / 2, y + h / 2 * k1)
            k3 = f(t + h / 2, y + h / 2 * k2)
            k4 = f(t + h, y + h * k3)
            M[:, col] = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return M


def radial_k(trap, rho: float, axis: int, rf: bool = True):
    """Spring constant k(t) of the trap along x (axis 0) or y (axis 1)."""
    sgn = -1.0 if axis == 0 else 1.0
    O2 = trap.Omega ** 2 / 4.0
    wz2 = rho * trap.omega_z ** 2

    def k(t):
        c = math.cos(trap.Omega * t) if rf else 0.0
        return O2 * (rho * trap.a + sgn * 2.0 * rho * trap.q * c) - 0.5 * wz2
    return k


def stable(species: Sequence, trap) -> bool:
    """True when every species' single-ion motion is bounded under the discrete
    kick-drift-kick map (|trace| < 2 of the one-RF-period monodromy along x and y,
    |2 - dt^2 omega_z^2| < 2 along z).  Commensurate steps (T_RF = K dt) use the exact
    K-step product; other steps fall back to the continuous Mathieu monodromy."""
    dt = trap.dt if trap.dt > 0 else 2.0 * math.pi / trap.Omega / 20.0
    qm0 = species[0].charge_e / species[0].mass_amu
    T = 2.0 * math.pi / trap.Omega
    K = T / dt
    for s in species:
        rho = (s.charge_e / s.mass_amu) / qm0
        wz2 = rho * trap.omega_z ** 2
        if not (wz2 > 0 and abs(2.0 - dt * dt * wz2) < 2.0):
            return False
        for axis in (0, 1):
            k = radial_k(trap, rho, axis)
            if abs(K - round(K)) < 1e-9 * K and round(K) <= 100000:
                M = _kdk_period_matrix(k, dt, int(round(K)))
            else:
                M = _mathieu_monodromy(k, T)
            if not abs(np.trace(M)) < 2.0:
                return False
    return True
