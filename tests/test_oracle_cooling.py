"""Pins of the oracle's species-selective cooling and of changing forces between runs
(CPU only).

Sec. 3 "Cooling the motion of ions": a Langevin bath may act on one group of ions
(langevinBath(T, dampingTime, group)), and laser cooling laserCool(species, g) is a
viscous force along the beam direction with no stochastic part.  Sec. 3 "Time
evolution": forces may be added or removed between evolve calls.  Sec. 5 "Cooling
mechanisms" validates both: free ions laser-cooled along a random direction decay with
the stated time constant while the perpendicular components stay untouched, and groups
of free ions coupled to distinct baths each follow Newton's law of cooling to their own
temperature.

What fixes each value here:
  laser cooling     the exact discrete decay of the kick-drift-kick map under a drag on
                    the half-step velocity (derived below), and the paper's
                    exponential-fit check of the time constant (within 1%)
  group baths       Newton's law of cooling T_j + (T_0 - T_j) exp(-2 gamma_j t) and
                    equipartition 3 k_B T_j = M <v^2> per group; a group without a bath
                    keeps its velocities bit for bit
  changing forces   a run split in two with unchanged, drag-free forces is the unsplit
                    run bit for bit; removing a bath from free ions freezes them
"""
import math

import numpy as np

import oracle
from iongen import CA40, NH3, OMEGA_RF, Cooling, Species, Trap, rf_period_dt, thermal_velocities

KB = oracle.const("kB")
DT = rf_period_dt(OMEGA_RF)


def _free_params(species, sp, seed=5, gamma=0.0, T=0.0):
    q, m, qm0 = oracle.ion_arrays(species, np.asarray(sp, np.uint8))
    tr = Trap(Omega=OMEGA_RF, a=0.0, q=0.3, omega_z=2 * math.pi * 0.2e6, gamma=gamma, T_bath=T,
              dt=DT, seed=seed)
    return q, m, oracle.params(tr, qm0, flags=oracle.TRAP_OFF | oracle.COULOMB_OFF)


def _unit(rng):
    d = rng.normal(size=3)
    return d / np.linalg.norm(d)


# ------------------------------------------------------------------ laser cooling

def test_laser_cooling_exact_discrete_decay():
    """A drag -L (k.u) k on the half-step velocity u: with p = k.v, the first half kick
    uses a_0 = -L p_0 k, so p_{1/2} = (1 - L dt/2) p_0; every later step multiplies the
    half-step projection by (1 - L dt), and the full-step value is (1 - L dt/2) times the
    preceding half-step one: p_n = (1 - L dt/2)^2 (1 - L dt)^(n-1) p_0 for n >= 1.  The
    laser vector is given unnormalised (rate times direction) along a random axis; a
    second species carries no laser and must not move at all."""
    rng = np.random.default_rng(11)
    n = 64
    sp = (np.arange(n) % 2).astype(np.uint8)
    q, m, p = _free_params([CA40, NH3], sp)
    L = 1e6  # tau = 1 us, as in the paper's check
    k = _unit(rng)
    cool = oracle.cooling_arrays(sp, [Cooling(laser=tuple(L * k)), Cooling()])
    v0 = rng.normal(size=(3, n)) * 3.0
    x0 = rng.normal(size=(3, n)) * 1e-5
    p0 = k @ v0
    for steps in (1, 2, 37, 400):
        x, v, a = oracle.run(x0, v0, q, m, p, steps, cooling=cool)
        pn = k @ v
        expect = (1 - L * DT / 2) ** 2 * (1 - L * DT) ** (steps - 1) * p0
        cooled = sp == 0
        np.testing.assert_allclose(pn[cooled], expect[cooled], rtol=1e-11, atol=1e-14 * np.abs(v0).max())
        perp = v - np.outer(k, pn)
        perp0 = v0 - np.outer(k, p0)
        np.testing.assert_allclose(perp[:, cooled], perp0[:, cooled], rtol=0, atol=1e-12 * np.abs(v0).max())
        assert np.array_equal(v[:, ~cooled], v0[:, ~cooled])


def test_laser_cooling_time_constant_fit():
    """Sec. 5 'Cooling mechanisms': project the velocities on the cooling axis, fit an
    exponential, compare the fitted time constant with tau = 1 us (the discrete map's
    rate is ln(1/(1 - dt/tau))/dt, 0.65% faster at dt = T_RF/20: within 1%)."""
    rng = np.random.default_rng(12)
    n = 32
    sp = np.zeros(n, np.uint8)
    q, m, p = _free_params([CA40], sp)
    tau = 1e-6
    k = _unit(rng)
    cool = oracle.cooling_arrays(sp, [Cooling(laser=tuple(k / tau))])
    v = rng.normal(size=(3, n)) * 5.0
    x = np.zeros((3, n))
    x, v, a = oracle.run(x, v, q, m, p, 0, cooling=cool)
    ts, ps = [], []
    step = 0
    for _ in range(40):
        x, v, a = oracle.run(x, v, q, m, p, 10, step0=step, a0=a, cooling=cool)
        step += 10
        ts.append(step * DT)
        ps.append(np.abs(k @ v))
    ps = np.array(ps)
    for i in range(n):
        slope = np.polyfit(ts, np.log(ps[:, i]), 1)[0]
        assert abs(-1.0 / slope / tau - 1) < 0.01


# ------------------------------------------------------------------ group baths

def test_species_selective_baths_follow_newton_cooling():
    """Sec. 5 'Cooling mechanisms': groups of free ions, each coupled to its own bath
    (gamma_j, T_j), relax as T_j + (T_0j - T_j) exp(-2 gamma_j t) and settle at T_j by
    3 k_B T_j = M <v^2>; a group left without a bath keeps its velocities exactly."""
    per = 4096
    species = [CA40, Species(CA40.mass_amu, 1.0), NH3, Species(NH3.mass_amu, 1.0)]
    sp = np.repeat(np.arange(4), per).astype(np.uint8)
    q, m, p = _free_params(species, sp, seed=21)
    baths = [Cooling(1e5, 1e-3), Cooling(3e5, 4e-3), Cooling(2e5, 0.5e-3), Cooling()]
    cool = oracle.cooling_arrays(sp, baths)
    v0 = thermal_velocities(species, sp, 1.0, seed=[21, 1])  # 1 K shape, rescaled per group
    scale = np.array([0.0, 0.0, math.sqrt(5e-3), math.sqrt(2e-3)])[sp]
    v0 = v0 * scale[None, :]
    x = np.zeros((3, len(sp)))

    def temps(v):
        t = m * (v ** 2).sum(axis=0) / (3 * KB)
        return np.array([t[sp == g].mean() for g in range(4)])

    T0 = temps(v0)
    x, v, a = oracle.run(x, v0, q, m, p, 0, cooling=cool)
    step = 0
    for t_mult in (0.25, 0.5, 1.0):
        target = int(round(t_mult / 1e5 / DT))
        x, v, a = oracle.run(x, v, q, m, p, target - step, step0=step, a0=a, cooling=cool)
        step = target
        T = temps(v)
        for g in range(3):
            gam, Tb = baths[g].gamma, baths[g].T_bath
            expect = Tb + (T0[g] - Tb) * math.exp(-2 * gam * step * DT)
            assert abs(T[g] / expect - 1) < 0.04, (g, T[g], expect)
        assert np.array_equal(v[:, sp == 3], v0[:, sp == 3])
    samples = []
    stride = int(round(1 / 1e5 / DT))
    for _ in range(12):
        x, v, a = oracle.run(x, v, q, m, p, stride, step0=step, a0=a, cooling=cool)
        step += stride
        samples.append(temps(v))
    mean = np.mean(samples, axis=0)
    for g in range(3):
        assert abs(mean[g] / baths[g].T_bath - 1) < 0.02, (g, mean[g])


# ------------------------------------------------------------------ changing forces

def test_split_run_without_drag_is_seamless():
    """Re-evaluating a_n at (x_n, t_n) with unchanged forces and no velocity-dependent
    term reproduces the a_n the step computed: the split run equals the unsplit one bit
    for bit (interacting ions in the RF trap)."""
    rng = np.random.default_rng(3)
    n = 24
    sp = np.zeros(n, np.uint8)
    q, m, qm0 = oracle.ion_arrays([CA40], sp)
    tr = Trap(Omega=OMEGA_RF, a=-0.001, q=0.3, omega_z=2 * math.pi * 0.2e6, gamma=0.0, T_bath=0.0,
              dt=DT, seed=1)
    p = oracle.params(tr, qm0)
    x0 = rng.normal(size=(3, n)) * 2e-5
    v0 = rng.normal(size=(3, n))
    xa, va, aa = oracle.run(x0, v0, q, m, p, 70)
    x1, v1, _ = oracle.run(x0, v0, q, m, p, 33)
    xb, vb, ab = oracle.run(x1, v1, q, m, p, 37, step0=33)
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(aa, ab)


def test_removing_the_bath_freezes_free_ions():
    """Ex. 2 removes the bath between two evolve calls: free ions then keep their
    velocities exactly, and drift in straight lines."""
    n = 256
    sp = np.zeros(n, np.uint8)
    q, m, p_on = _free_params([CA40], sp, seed=8, gamma=1e5, T=1e-3)
    _, _, p_off = _free_params([CA40], sp, seed=8)
    x, v, a = oracle.run(np.zeros((3, n)), np.zeros((3, n)), q, m, p_on, 500)
    assert np.abs(v).max() > 0
    x2, v2, a2 = oracle.run(x, v, q, m, p_off, 300, step0=500)
    assert np.array_equal(v2, v) and not np.any(a2)
    np.testing.assert_allclose(x2, x + 300 * DT * v, rtol=1e-12, atol=1e-20)
