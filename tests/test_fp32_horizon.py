"""The 100-step horizon of the test clouds under FP32-sized force errors (CPU only, no
GPU).

The trajectory bar for the FP32 form is 1e-4 (relative RMS of positions) after 100
steps.  Whether FP32 pair forces can meet it on a given cloud is a property of the
cloud -- how strongly its dynamics amplify a small perturbation of the forces -- not of
any kernel.  These tests measure that on the CPU, with two instruments:

  * an FP32 emulation of the pair sum (``fp32_pairs.c``: hi/lo positions, 128-j chunks
    summed as even and odd j, Kahan across chunks, every operation correctly rounded),
    with three reciprocal square roots: correctly rounded, a model of the hardware
    approximation (relative error up to 2^-22.9, the documented bound of
    rsqrt.approx.f32, drawn per pair from a hash), and that model refined by one
    Newton-Raphson step;
  * the FP64 oracle with its Coulomb accelerations multiplied by (1 + 1e-7 xi), xi a
    standard normal per component and step: a perturbation of the size of the FP32
    form's force error, with no FP32 arithmetic at all.

In both, the rest of the step (trap, Langevin bath, kick-drift-kick in FP64) is the
oracle's, so the only difference from the oracle's own run is the pair sum.

Pinned facts (the readings the GPU parity tests rest on):
  * the harness reproduces the oracle's own run when its pair sum is the oracle's;
  * on the N = 4096 two-species cloud every FP32 variant stays below 1e-6 at step 50
    and then departs by 3e-5 .. 3e-4 at step 100 -- correctly rounded FP32 itself above
    the 1e-4 bar -- more than a hundredfold growth in 50 steps, whatever the rsqrt;
  * the oracle under 1e-7 force perturbations (somewhat larger than the FP32 form's own
    errors) does the same on that cloud, and on the 1500-ion cloud of the batched parity
    test stays below 1e-5 at step 80 and reaches ~1e-4 at step 100 (a close encounter
    between the two).
So the FP32 form is held to 1e-6 at step 50 on the first cloud and to 1e-4 at step 80
on the second, and to 5e-4 at step 100 on both (positions; 1e-3 and 5e-3 on
velocities): a factor of about two above the largest departure measured here.
"""
import math
import os
import subprocess
import threading

import ctypes
import numpy as np
import pytest

import iongen
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fp32_pairs.c")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "libfp32pairs.so")
_lock = threading.Lock()
_lib = None

MARKS = (10, 50, 75, 100)
PERTURBATION = 1e-7


def _emu():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(SO) or os.path.getmtime(SO) < os.path.getmtime(SRC):
                os.makedirs(BUILD, exist_ok=True)
                tmp = SO + f".{os.getpid()}.tmp"
                subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-std=c11", "-shared",
                                       "-fPIC", "-o", tmp, SRC, "-lm"])
                os.replace(tmp, SO)
            L = ctypes.CDLL(SO)
            dp = ctypes.POINTER(ctypes.c_double)
            L.emu_coulomb.argtypes = [ctypes.c_int64, dp, dp, ctypes.POINTER(ctypes.c_float), ctypes.c_int,
                                      ctypes.c_uint64, dp]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def emu_coulomb(x, coul, w, mode, salt):
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[1]
    acc = np.empty((3, n))
    _emu().emu_coulomb(n, _dp(x), _dp(coul), w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), int(mode),
                       ctypes.c_uint64(salt), _dp(acc))
    return acc


def run(w, steps, coulomb, marks=MARKS):
    """Kick-drift-kick as the oracle runs it, with the Coulomb term from ``coulomb(x, k)``
    (k = step index of x) and everything else from the oracle; returns {mark: (x, v)}."""
    q, m, qm0 = oracle.ion_arrays(w.species, w.species_of_ion)
    p = oracle.params(w.trap, qm0)
    ext = oracle.params(w.trap, qm0, flags=p.flags | oracle.COULOMB_OFF)
    dt = p.dt
    x, v = w.x0.copy(), w.v0.copy()
    a = coulomb(x, 0) + oracle.accel(x, v, q, m, ext, 0, 0.0)
    out = {}
    for s in range(steps):
        vh = v + 0.5 * dt * a
        x = x + dt * vh
        a = coulomb(x, s + 1) + oracle.accel(x, vh, q, m, ext, s + 1, (s + 1) * dt)
        v = vh + 0.5 * dt * a
        if s + 1 in marks:
            out[s + 1] = (x.copy(), v.copy())
    return out


def rel_rms(a, b):
    return math.sqrt(float(((a - b) ** 2).sum()) / float((b ** 2).sum()))


def _oracle_refs(w, marks):
    q, m, qm0 = oracle.ion_arrays(w.species, w.species_of_ion)
    p = oracle.params(w.trap, qm0)
    ref, x, v, a, done = {}, w.x0, w.v0, None, 0
    for mk in marks:
        x, v, a = oracle.run(x, v, q, m, p, mk - done, step0=done, a0=a)
        done = mk
        ref[mk] = (x.copy(), v.copy())
    return q, m, ref


def _errors(got, ref):
    return {mk: (rel_rms(got[mk][0], ref[mk][0]), rel_rms(got[mk][1], ref[mk][1])) for mk in got}


def _perturbed(q, m, seed):
    """The oracle's Coulomb accelerations times (1 + 1e-7 xi), xi ~ N(0, 1) per component."""
    rng = np.random.default_rng(seed)

    def coulomb(x, k):
        a = oracle.coulomb_accel(x, q, m)
        return a * (1.0 + PERTURBATION * rng.standard_normal(a.shape))
    return coulomb


def cloud1500():
    """The 1500-ion cloud of the batched parity test (same recipe and seed): Ca+, NH3+
    and a doubly charged species, Gaussian sigma 40 um, q = 0.25, a = -0.001."""
    n, seed = 1500, 1800
    species = (iongen.CA40, iongen.NH3, iongen.Species(88.0, 2.0))
    rng = np.random.default_rng(seed)
    sp = rng.integers(0, len(species), size=n).astype(np.uint8)
    sp[0] = 0
    x = iongen.gaussian_positions(n, 40e-6, seed=[seed, 7])
    trap = iongen.Trap(Omega=iongen.OMEGA_RF, a=-0.001, q=0.25, omega_z=2 * math.pi * 0.2e6,
                       gamma=1e5, T_bath=1e-3, dt=iongen.rf_period_dt(iongen.OMEGA_RF), seed=seed)
    return iongen.Workload(f"cloud{n}", list(species), sp, x,
                           np.random.default_rng(seed + 1).normal(scale=0.3, size=(3, n)), trap, 100)


@pytest.fixture(scope="module")
def cloud():
    w = iongen.mix_n4096()
    q, m, ref = _oracle_refs(w, MARKS)
    coul = np.ascontiguousarray(oracle.const("ke") * oracle.const("e") * q / m)  # k_e e^2 z_i / M_i
    wj = (q / oracle.const("e")).astype(np.float32)
    return w, q, m, ref, coul, wj


def test_harness_reproduces_the_oracle_run(cloud):
    """With the oracle's own pair sum the harness is the oracle's run, step for step."""
    w, q, m, ref, _, _ = cloud
    got = run(w, 50, lambda x, k: oracle.coulomb_accel(x, q, m), marks=(10, 50))
    for mk in (10, 50):
        assert rel_rms(got[mk][0], ref[mk][0]) < 1e-13, mk
        assert rel_rms(got[mk][1], ref[mk][1]) < 1e-12, mk


def test_emulated_forces_within_the_force_bar(cloud):
    w, q, m, _, coul, wj = cloud
    exact = oracle.coulomb_accel(w.x0, q, m)
    errs = [rel_rms(emu_coulomb(w.x0, coul, wj, mode, 7), exact) for mode in (0, 1, 2)]
    print("\n  force error (correctly rounded, approximation, refined):", ["%.2e" % e for e in errs])
    assert max(errs) < 1e-6, errs
    # the approximation model is the least accurate; the refinement recovers most of it
    assert errs[1] > errs[2] and errs[1] > errs[0], errs


def test_fp32_horizon_of_the_n4096_cloud(cloud):
    w, q, m, ref, coul, wj = cloud
    res = {}
    for name, mode, salt in (("correctly rounded", 0, 0), ("approximation, draw 1", 1, 0),
                             ("approximation, draw 2", 1, 5000), ("approximation + Newton", 2, 0)):
        got = run(w, 100, lambda x, k, mode=mode, salt=salt: emu_coulomb(x, coul, wj, mode, salt + k))
        res[name] = _errors(got, ref)
    print()
    for name, r in res.items():
        print(f"  {name:24s} " + "  ".join(f"x{mk}={r[mk][0]:.2e} v{mk}={r[mk][1]:.2e}" for mk in MARKS))
    for name, r in res.items():
        assert r[50][0] < 1e-6 and r[50][1] < 1e-5, (name, r)            # before the divergence
        assert 3e-5 < r[100][0] < 3e-4 and r[100][1] < 5e-4, (name, r)  # after it, whatever the rsqrt
        assert r[100][0] > 100 * r[50][0], (name, r)
    assert res["correctly rounded"][100][0] > 1e-4, res  # correctly rounded FP32 itself exceeds 1e-4


@pytest.mark.parametrize("which", ["mix_n4096", "cloud1500"])
def test_oracle_amplifies_fp32_sized_force_errors(which):
    w = iongen.mix_n4096() if which == "mix_n4096" else cloud1500()
    marks = (50, 80, 100)
    q, m, ref = _oracle_refs(w, marks)
    errs = [_errors(run(w, 100, _perturbed(q, m, seed), marks=marks), ref) for seed in (1, 2)]
    print()
    for r in errs:
        print(f"  {which} " + "  ".join(f"x{mk}={r[mk][0]:.2e} v{mk}={r[mk][1]:.2e}" for mk in marks))
    for r in errs:
        assert r[50][0] < 1e-5, r
        assert r[100][0] > 30 * r[50][0] and r[100][0] > 3e-5, r
        assert r[100][0] < 3e-4 and r[100][1] < 1e-3, r
        if which == "cloud1500":  # quiet until step 80, then the close encounter
            assert r[80][0] < 1e-5 and r[100][0] > 10 * r[80][0], r
