"""Pins of the oracle's pseudopotential trap, minimiser and Hessian (CPU only).

Sec. 2 Eq. 2 (pseudopotential secular frequency), Sec. 3 "Forces and fields"
(linearPseudoPT: a static trap per species), Sec. 3 "Minimisation" (damped dynamics with a
limited step), Sec. 5 "Equilibrium separation" (James' chain) and "Normal modes of motion"
(eigenvalues of the Hessian of Eq. 4's potential; Fourier spectrum of kicked crystals).

What fixes each value here:
  pseudopotential  the exact secular frequency of the Mathieu equation at small q (Eq. 2 is
                   its small-q limit), for two charge/mass ratios; the exact discrete
                   recurrence of a single ion on a static spring
  Hessian          central differences of the oracle's own (pinned) accelerations; the
                   closed-form mode frequencies of two- and three-ion chains (axial 1, sqrt 3,
                   sqrt(29/5); radial w_r, sqrt(w_r^2 - w_z^2), sqrt(w_r^2 - 12/5 w_z^2) in
                   units of w_z, James 1998 as quoted in Sec. 5); the centre-of-mass and
                   breathing modes at w_z and sqrt(3) w_z for any chain length
  minimiser        closed-form two- and three-ion spacings; longer chains against an
                   independent root solve of the dimensionless 1D force balance; the step
                   limit itself
  spectrum         the Fourier peaks of an undamped, kicked chain at the Hessian frequencies
"""
import math

import numpy as np
import pytest

import oracle
from iongen import CA40, NH3, OMEGA_RF, Trap, rf_period_dt

E = oracle.const("e")
AMU = oracle.const("amu")
KE = oracle.const("ke")
M_CA = CA40.mass_amu * AMU
DT = rf_period_dt(OMEGA_RF)
WZ = 2 * math.pi * 0.2e6


def _p(flags, **kw):
    base = dict(Omega=OMEGA_RF, a=0.0, q=0.3, omega_z=WZ, gamma=0.0, T_bath=0.0, dt=DT, seed=1)
    base.update(kw)
    return oracle.params(Trap(**base), E / M_CA, flags=flags)


def _mathieu_omega(a, q, Omega):
    """Secular angular frequency of x'' = -(Omega^2/4)(a - 2 q cos Omega t) x from the
    monodromy over one period (RK4, fine steps): cos(pi beta) = tr/2, w = beta Omega/2."""
    def k(t):
        return Omega ** 2 / 4 * (a - 2 * q * math.cos(Omega * t))
    M = oracle._mathieu_monodromy(k, 2 * math.pi / Omega, sub=8192)
    beta = math.acos(np.trace(M) / 2) / math.pi
    return beta * Omega / 2


# ------------------------------------------------------------------ pseudopotential

@pytest.mark.parametrize("species", [CA40, NH3])
def test_pseudopotential_is_small_q_limit_of_mathieu(species):
    """At q = 0.02 the Eq. 2 frequency of each species (its q and a scaled by its
    charge/mass) matches the exact Mathieu secular frequency to 1e-3; axially the spring
    is rho w_z^2."""
    rho = (species.charge_e / species.mass_amu) / (CA40.charge_e / CA40.mass_amu)
    p = _p(oracle.PSEUDO, q=0.02, a=0.0001, omega_z=2 * math.pi * 0.02e6)
    k = oracle.pseudo_springs(p, rho * E / M_CA)
    a_x = rho * 0.0001 - 2 * rho * p.omega_z ** 2 / OMEGA_RF ** 2
    exact = _mathieu_omega(a_x, rho * 0.02, OMEGA_RF)
    assert abs(math.sqrt(k[0]) / exact - 1) < 1e-3
    assert k[0] == k[1]
    assert abs(k[2] / (rho * p.omega_z ** 2) - 1) < 1e-15


def test_single_ion_on_pseudo_springs_follows_discrete_recurrence():
    """x_{k+1} + x_{k-1} = (2 - k dt^2) x_k exactly for kick-drift-kick on a spring k, in
    each axis with its own spring (pseudopotential of Eq. 2, and explicit springs)."""
    p = _p(oracle.PSEUDO)
    q_, m_ = np.array([E]), np.array([M_CA])
    ks = oracle.pseudo_springs(p, E / M_CA)
    explicit = oracle.springs_arrays([0], [(2.1e6, 2.6e6, 1.1e6)])
    for springs, kk in ((None, ks), (explicit, explicit[:, 0])):
        x = np.array([[3e-6], [-2e-6], [5e-6]])
        v = np.array([[0.4], [0.1], [-0.3]])
        xs = []
        a = None
        for step in range(60):
            xs.append(x[:, 0].copy())
            x, v, a = oracle.run(x, v, q_, m_, p, 1, step0=step, a0=a, springs=springs)
        xs = np.array(xs)
        for c in range(3):
            lhs = xs[2:, c] + xs[:-2, c]
            rhs = (2 - kk[c] * DT ** 2) * xs[1:-1, c]
            assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(xs[:, c]).max()


# ------------------------------------------------------------------ Hessian

def test_hessian_is_derivative_of_accelerations():
    """Central differences of M_i a_i (trap springs + Coulomb, mixed charges and masses)
    give -sqrt(M_i M_j) H; the matrix is symmetric."""
    rng = np.random.default_rng(9)
    n = 7
    x = rng.normal(size=(3, n)) * 2e-5
    charge = E * np.array([1, 1, 2, 1, -1, 1, 2.0])
    mass = AMU * np.array([40, 17, 88, 40, 30, 9, 138.0])
    p = _p(oracle.PSEUDO)
    springs = rng.uniform(1e11, 5e12, size=(3, n))
    for spr in (None, springs):
        H = oracle.hessian(x, charge, mass, p, springs=spr)
        assert np.allclose(H, H.T, rtol=0, atol=1e-12 * np.abs(H).max())
        h = 1e-10
        zero = np.zeros_like(x)
        for j in range(n):
            for b in range(3):
                xp, xm = x.copy(), x.copy()
                xp[b, j] += h
                xm[b, j] -= h
                dF = (mass * oracle.accel(xp, zero, charge, mass, p, 0, 0.0, springs=spr)
                      - mass * oracle.accel(xm, zero, charge, mass, p, 0, 0.0, springs=spr)) / (2 * h)
                col = -dF.T.reshape(-1) / np.sqrt(mass[np.arange(3 * n) // 3] * mass[j])
                np.testing.assert_allclose(H[:, 3 * j + b], col, rtol=2e-6, atol=2e-6 * np.abs(H).max())


def _chain(n, wz):
    """Equilibrium of an n-ion Ca+ chain on the axis, from an independent solve of the
    dimensionless force balance u_i = sum_j sign(u_i - u_j)/(u_i - u_j)^2 (l = 1)."""
    from scipy.optimize import fsolve

    def f(u):
        d = u[:, None] - u[None, :]
        np.fill_diagonal(d, np.inf)
        return u - (np.sign(d) / d ** 2).sum(axis=1)

    u = fsolve(f, np.linspace(-1, 1, n) * n ** 0.6, xtol=1e-14)
    l = (E ** 2 / (4 * math.pi * oracle.const("eps0") * M_CA * wz ** 2)) ** (1 / 3)
    x = np.zeros((3, n))
    x[2] = np.sort(u) * l
    return x, l


def test_hessian_modes_of_two_and_three_ion_chains():
    wr, wz = 2 * math.pi * 1.0e6, 2 * math.pi * 0.2e6
    p = _p(0)
    for n, axial, radial in ((2, [1, 3], [wr ** 2 / wz ** 2, wr ** 2 / wz ** 2 - 1]),
                             (3, [1, 3, 29 / 5], [wr ** 2 / wz ** 2, wr ** 2 / wz ** 2 - 1,
                                                  wr ** 2 / wz ** 2 - 12 / 5])):
        x, _ = _chain(n, wz)
        sp = np.zeros(n, np.uint8)
        q_, m_, _ = oracle.ion_arrays([CA40], sp)
        H = oracle.hessian(x, q_, m_, p, springs=oracle.springs_arrays(sp, [(wr, wr, wz)]))
        w2 = np.linalg.eigvalsh(H) / wz ** 2
        expect = sorted(axial + radial + radial)
        np.testing.assert_allclose(np.sort(w2), expect, rtol=1e-9)


@pytest.mark.parametrize("n", [5, 8])
def test_centre_of_mass_and_breathing_modes_of_long_chains(n):
    wr, wz = 2 * math.pi * 2.0e6, 2 * math.pi * 0.2e6
    x, _ = _chain(n, wz)
    sp = np.zeros(n, np.uint8)
    q_, m_, _ = oracle.ion_arrays([CA40], sp)
    H = oracle.hessian(x, q_, m_, _p(0), springs=oracle.springs_arrays(sp, [(wr, wr, wz)]))
    axial = np.linalg.eigvalsh(H[2::3, 2::3]) / wz ** 2
    assert abs(axial[0] - 1) < 1e-9 and abs(axial[1] - 3) < 1e-9


# ------------------------------------------------------------------ minimiser

def test_minimiser_limits_each_step():
    """No ion moves more than dmax in one step; with large forces the largest move is
    exactly dmax."""
    rng = np.random.default_rng(2)
    n = 12
    x0 = rng.normal(size=(3, n)) * 5e-5
    sp = np.zeros(n, np.uint8)
    q_, m_, _ = oracle.ion_arrays([CA40], sp)
    p = _p(oracle.PSEUDO)
    prev = x0
    for k in range(1, 6):
        x, steps, _ = oracle.minimize(x0, q_, m_, p, DT * 50, 1e-7, 0.0, k)
        step_len = np.sqrt(((x - prev) ** 2).sum(axis=0))
        assert steps == k and step_len.max() <= 1e-7 * (1 + 1e-12)
        assert abs(step_len.max() / 1e-7 - 1) < 1e-12
        prev = x


@pytest.mark.parametrize("n", [2, 3, 5, 7, 10])
def test_minimiser_finds_the_chain(n):
    """From a perturbed 3D start, the minimised crystal is the linear chain of the
    independent force-balance solve (2 ions: d^3 = e^2/(2 pi eps0 M w_z^2); 3 ions:
    0, +-(5/4)^(1/3) l)."""
    wr, wz = 2 * math.pi * 3.0e6, 2 * math.pi * 0.2e6
    xe, l = _chain(n, wz)
    if n == 2:
        assert abs((xe[2, 1] - xe[2, 0]) ** 3 / (E ** 2 / (2 * math.pi * oracle.const("eps0") * M_CA * wz ** 2)) - 1) < 1e-10
    if n == 3:
        assert abs(xe[2, 2] / l - (5 / 4) ** (1 / 3)) < 1e-10
    rng = np.random.default_rng(n)
    x0 = xe * (1 + 0.2 * rng.uniform(-1, 1, size=(1, n))) + rng.normal(size=(3, n)) * 0.1 * l
    sp = np.zeros(n, np.uint8)
    q_, m_, _ = oracle.ion_arrays([CA40], sp)
    springs = oracle.springs_arrays(sp, [(wr, wr, wz)])
    fscale = M_CA * wz ** 2 * l
    x, steps, fn = oracle.minimize(x0, q_, m_, _p(0), DT, 0.05 * l, 1e-10 * fscale, 200000,
                                   springs=springs)
    assert fn < 1e-10 * fscale, (steps, fn / fscale)
    order = np.argsort(x[2])
    np.testing.assert_allclose(x[:, order], xe, rtol=0, atol=1e-8 * l)


# ------------------------------------------------------------------ spectrum

def test_kicked_chain_spectrum_peaks_at_hessian_frequencies():
    """Sec. 5 'Normal modes of motion': a minimised chain given small random velocities and
    evolved without damping in the pseudopotential; the Fourier spectrum of its axial
    positions peaks at the axial Hessian frequencies (1, sqrt 3, sqrt(29/5)) w_z."""
    n = 3
    wr, wz = 2 * math.pi * 1.0e6, 2 * math.pi * 0.2e6
    xe, l = _chain(n, wz)
    sp = np.zeros(n, np.uint8)
    q_, m_, _ = oracle.ion_arrays([CA40], sp)
    springs = oracle.springs_arrays(sp, [(wr, wr, wz)])
    rng = np.random.default_rng(4)
    v0 = rng.normal(size=(3, n)) * 0.02
    stride, samples = 10, 4096
    x, v, a = xe, v0, None
    zs = []
    p = _p(0)
    for s in range(samples):
        x, v, a = oracle.run(x, v, q_, m_, p, stride, step0=s * stride, a0=a, springs=springs)
        zs.append(x[2].copy())
    zs = np.array(zs) - xe[2]
    spec = np.abs(np.fft.rfft(zs * np.hanning(samples)[:, None], axis=0)).sum(axis=1)
    freqs = np.fft.rfftfreq(samples, d=stride * DT) * 2 * math.pi / wz
    res = freqs[1]
    peaks = [freqs[i] for i in range(1, len(spec) - 1) if spec[i] > spec[i - 1] and spec[i] > spec[i + 1]
             and spec[i] > 0.02 * spec.max()]
    for w in (1.0, math.sqrt(3), math.sqrt(29 / 5)):
        assert min(abs(f - w) for f in peaks) < 1.5 * res, (w, peaks)


# ------------------------------------------------------------------ dump / timeAvg

def test_record_time_average_of_uniform_motion_and_harmonic_motion():
    """Sec. 3 'Writing/reading data' (timeAvg): a free ion's averaged velocity is its
    velocity; on a static spring k the kick-drift-kick trajectory is x_m = A cos(m th + ph)
    with cos th = 1 - k dt^2/2 and its full-step velocity (x_{m+1} - x_{m-1})/(2 dt), whose
    window mean has a closed form (geometric sums) that the recorded average must match."""
    sp = np.zeros(1, np.uint8)
    q_, m_ = np.array([E]), np.array([M_CA])
    pfree = _p(oracle.TRAP_OFF)
    X, V, VA, _ = oracle.record(np.zeros((3, 1)), np.array([[0.3], [-0.2], [0.7]]), q_, m_, pfree, 60, 20, 20)
    np.testing.assert_allclose(VA[:, :, 0], np.tile([0.3, -0.2, 0.7], (3, 1)), rtol=1e-14)
    k = 4.0e12
    springs = np.full((3, 1), k)
    x0 = np.array([[2e-6], [-1e-6], [3e-6]])
    v0 = np.array([[0.5], [0.2], [-0.1]])
    every, W, K = 30, 20, 4
    X, V, VA, _ = oracle.record(x0, v0, q_, m_, _p(0), every * K, every, W, springs=springs)
    th = math.acos(1 - k * DT ** 2 / 2)
    # x_m = A cos(m th) + B sin(m th): x_0 given, x_1 = x_0 + dt (v_0 + dt/2 a_0), a_0 = -k x_0
    x1 = x0[:, 0] + DT * (v0[:, 0] - DT / 2 * k * x0[:, 0])
    A = x0[:, 0]
    B = (x1 - A * math.cos(th)) / math.sin(th)

    def xm(m):
        return A * math.cos(m * th) + B * math.sin(m * th)
    for r in range(K):
        s = (r + 1) * every
        expect = sum((xm(mm + 1) - xm(mm - 1)) / (2 * DT) for mm in range(s - W + 1, s + 1)) / W
        np.testing.assert_allclose(VA[r, :, 0], expect, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(X[r, :, 0], xm(s), rtol=1e-9, atol=1e-18)
