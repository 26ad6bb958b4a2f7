"""GPU parity of the pseudopotential trap, the minimiser and the normal-mode Hessian
against the FP64 oracle, through the C ABI.

Sec. 2 Eq. 2 and Sec. 3 "Forces and fields" (linearPseudoPT), Sec. 3 "Minimisation",
Sec. 5 "Equilibrium separation" and "Normal modes of motion".  Tolerances: trajectories in
the pseudopotential trap as in test_gpu_parity.py (FP32 form 1e-4 over 80 steps, FP64 form
1e-9); Hessian (FP64 on the device) within 1e-12 of the oracle's, normwise; minimised
chains within the displacement that the stopping force allows along the softest mode,
2 ftol / (M w_z^2) (ftol 1e-6 sqrt(n) of the force scale M w_z^2 l in the FP32 form, whose
forces carry ~1e-7 relative rounding, and 1e-10 in the FP64 form).
"""
import math

import numpy as np
import pytest

import iongen
import oracle

pytestmark = pytest.mark.gpu

E = oracle.const("e")
AMU = oracle.const("amu")
M_CA = iongen.CA40.mass_amu * AMU
DT = iongen.rf_period_dt(iongen.OMEGA_RF)
SR88 = iongen.Species(88.0, 2.0)


@pytest.fixture(scope="module")
def it():
    from paper_1907_10514_gb300 import build
    build.build()
    import paper_1907_10514_gb300 as mod
    return mod


def rel_rms(a, b):
    return math.sqrt(float(((a - b) ** 2).sum()) / float((b ** 2).sum()))


def _trap(**kw):
    base = dict(Omega=iongen.OMEGA_RF, a=-0.001, q=0.25, omega_z=2 * math.pi * 0.2e6, gamma=1e5, T_bath=1e-3,
                dt=DT, seed=3)
    base.update(kw)
    return iongen.Trap(**base)


def _cloud(n, seed, species=(iongen.CA40, iongen.NH3, SR88)):
    rng = np.random.default_rng(seed)
    sp = rng.integers(0, len(species), size=n).astype(np.uint8)
    sp[0] = 0
    x = iongen.gaussian_positions(n, 40e-6, seed=[seed, 7])
    v = rng.normal(scale=0.3, size=(3, n))
    return list(species), sp, x, v


def _chain(n, wz):
    """Independent solve of the dimensionless force balance of an n-ion chain (l = 1)."""
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


# per-species secular frequencies of the size of the Eq. 2 trap of _trap() (a stiffer trap
# collapses the 40 um clouds through their centre within 80 steps: close encounters that
# amplify any rounding difference chaotically)
FREQS = [(2 * math.pi * 0.32e6, 2 * math.pi * 0.35e6, 2 * math.pi * 0.2e6),
         (2 * math.pi * 0.7e6, 2 * math.pi * 0.75e6, 2 * math.pi * 0.3e6),
         (2 * math.pi * 0.28e6, 2 * math.pi * 0.3e6, 2 * math.pi * 0.19e6)]


@pytest.mark.parametrize("form", ["last_cta", "persistent", "row_persistent", "batched", "fp64"])
@pytest.mark.parametrize("given", [False, True], ids=["eq2", "frequencies"])
def test_pseudo_trap_trajectory_matches_oracle(it, form, given):
    """Mixed species in the pseudopotential trap of Eq. 2, or in per-species frequencies,
    with the bath on: 80 steps against the oracle."""
    n = 3000 if form in ("last_cta", "persistent", "row_persistent", "fp64") else 700
    species, sp, x0, v0 = _cloud(n, 12)
    tr = _trap()
    flags = it.IONTRAP_PSEUDO
    prec = 1 if form == "fp64" else 0
    q, m, qm0 = oracle.ion_arrays(species, sp)
    po = oracle.params(tr, qm0, flags=oracle.PSEUDO)
    springs = oracle.springs_arrays(sp, FREQS) if given else None
    xo, vo, _ = oracle.run(x0, v0, q, m, po, 80, springs=springs)
    with it.Simulation(species, sp, x0, v0, it.make_params(tr, precision=prec, flags=flags)) as s:
        if given:
            s.set_pseudo_frequencies(FREQS)
        if form == "last_cta":
            s.set_config(128, 2, 1, -(-n // 12), 1)
        elif form == "persistent":
            s.set_config(256, 2, 1, -(-n // 25), 4)
        elif form == "row_persistent":
            s.set_config(512, 1, 1, 20, 5)
        if form == "batched":
            it.iontrap_step_many([s.handle], [80])
        else:
            s.step(80)
        x, v, step, _ = s.state()
    tol = 1e-9 if prec else 1e-4
    assert step == 80 and rel_rms(x, xo) < tol and rel_rms(v, vo) < 10 * tol


@pytest.mark.parametrize("n", [2, 3, 5, 10])
@pytest.mark.parametrize("prec", [0, 1])
def test_minimize_finds_the_chain(it, n, prec):
    """From a perturbed 3D start the device minimiser reaches the linear chain of the
    independent force-balance solve, to the displacement its stopping force allows."""
    wr, wz = 2 * math.pi * 3.0e6, 2 * math.pi * 0.2e6
    xe, l = _chain(n, wz)
    rng = np.random.default_rng(n)
    x0 = xe * (1 + 0.2 * rng.uniform(-1, 1, size=(1, n))) + rng.normal(size=(3, n)) * 0.1 * l
    sp = np.zeros(n, np.uint8)
    fscale = M_CA * wz ** 2 * l
    ftol = (1e-6 * math.sqrt(n) if prec == 0 else 1e-10) * fscale
    with it.Simulation([iongen.CA40], sp, x0, None, it.make_params(_trap(gamma=0.0), precision=prec,
                                                                   flags=it.IONTRAP_PSEUDO)) as s:
        s.set_pseudo_frequencies([(wr, wr, wz)])
        iters, fn = s.minimize(200000, 0.05 * l, ftol)
        x, v, step, _ = s.state()
    order = np.argsort(x[2])
    dev = np.abs(x[:, order] - xe).max() / l
    print(f"n={n} prec={prec} iters={iters} |F|/fscale={fn / fscale:.3e} max dev/l={dev:.3e}")
    assert fn < ftol and step == 0 and not np.any(v)
    # a residual force |F| < ftol displaces the crystal by at most |F| / (M w_z^2) along its
    # softest mode (the centre of mass along z)
    np.testing.assert_allclose(x[:, order], xe, rtol=0, atol=2 * ftol / (M_CA * wz ** 2))


@pytest.mark.parametrize("prec", [0, 1])
def test_minimize_3d_crystal_matches_oracle(it, prec):
    """A 40-ion, two-species 3D crystal in per-species frequencies, minimised on the device
    and by the oracle from the same start.  A stopping force |F| < ftol fixes the minimum
    only to what the crystal's softest mode allows (its mass-weighted Hessian eigenvalue
    lam_min is 0.002 w0^2 here): positions within 2 ftol / (M_min lam_min), energy within
    ftol^2 / (2 M_min lam_min) of the oracle's minimum, and the FP64 residual force at the
    device's positions below 1.5 ftol."""
    n = 40
    species = [iongen.CA40, iongen.NH3]
    sp = (np.arange(n) % 4 == 0).astype(np.uint8)
    w0 = 2 * math.pi * 0.3e6
    freqs = [(w0, 1.1 * w0, 0.9 * w0), (1.6 * w0, 1.7 * w0, 1.4 * w0)]
    rng = np.random.default_rng(40)
    x0 = rng.normal(size=(3, n)) * 30e-6
    q, m, qm0 = oracle.ion_arrays(species, sp)
    springs = oracle.springs_arrays(sp, freqs)
    l = (E ** 2 / (4 * math.pi * oracle.const("eps0") * M_CA * w0 ** 2)) ** (1 / 3)
    fscale = M_CA * w0 ** 2 * l
    ftol = 1e-5 * fscale if prec == 0 else 1e-8 * fscale
    po = oracle.params(_trap(gamma=0.0, T_bath=0.0), qm0, flags=oracle.PSEUDO)
    xo, steps, fo = oracle.minimize(x0, q, m, po, 5 * DT, 0.02 * l, 1e-8 * fscale, 400000, springs=springs)
    assert fo < 1e-8 * fscale
    lam = float(np.linalg.eigvalsh(oracle.hessian(xo, q, m, po, springs=springs)).min())
    assert lam > 0
    with it.Simulation(species, sp, x0, None, it.make_params(_trap(), precision=prec,
                                                             flags=it.IONTRAP_PSEUDO)) as s:
        s.set_pseudo_frequencies(freqs)
        iters, fn = s.minimize(400000, 0.02 * l, ftol, dt=5 * DT)
        x = s.state()[0]
    assert fn < ftol
    assert np.abs(x - xo).max() < 2 * ftol / (m.min() * lam)
    zero = np.zeros_like(x)
    resid = m * oracle.accel(x, zero, q, m, po, 0, 0.0, springs=springs)
    assert math.sqrt(float((resid ** 2).sum())) < 1.5 * ftol
    e_dev, e_ref = oracle.energy(x, zero, q, m, po, springs), oracle.energy(xo, zero, q, m, po, springs)
    slack = 1e-12 * abs(e_ref)
    assert -slack - fo ** 2 / (2 * m.min() * lam) <= e_dev - e_ref <= ftol ** 2 / (2 * m.min() * lam) + slack


def test_hessian_matches_oracle(it):
    """The device Hessian (FP64) against the oracle's on a mixed-charge cloud, in the
    Eq. 2 pseudopotential, in given frequencies and in the static RF-off trap."""
    n = 300
    species, sp, x0, v0 = _cloud(n, 77)
    q, m, qm0 = oracle.ion_arrays(species, sp)
    for flags_lib, flags_or, given in ((it.IONTRAP_PSEUDO, oracle.PSEUDO, False),
                                       (it.IONTRAP_PSEUDO, oracle.PSEUDO, True),
                                       (it.IONTRAP_RF_OFF, oracle.RF_OFF, False)):
        tr = _trap(a=0.01) if flags_lib == it.IONTRAP_RF_OFF else _trap()
        po = oracle.params(tr, qm0, flags=flags_or)
        springs = oracle.springs_arrays(sp, FREQS) if given else None
        if flags_lib == it.IONTRAP_RF_OFF:
            springs = np.stack([-oracle.trap_accel(po, qi / mi, np.eye(3)[c], 0.0)[c] * np.ones(1)
                                for qi, mi in zip(q, m) for c in range(3)]).reshape(n, 3).T.copy()
        ref = oracle.hessian(x0, q, m, po, springs=springs)
        with it.Simulation(species, sp, x0, v0, it.make_params(tr, flags=flags_lib)) as s:
            if given:
                s.set_pseudo_frequencies(FREQS)
            H = s.hessian()
        assert np.abs(H - ref).max() < 1e-12 * np.abs(ref).max()


def test_normal_mode_spectrum_on_device(it):
    """Sec. 5 'Normal modes of motion': minimise a 4-ion chain on the device, read its
    Hessian, give the ions small random velocities and evolve without damping; the Fourier
    peaks of the axial motion sit at the square roots of the axial Hessian eigenvalues, the
    lowest two at w_z and sqrt(3) w_z."""
    n = 4
    wr, wz = 2 * math.pi * 1.5e6, 2 * math.pi * 0.2e6
    xe, l = _chain(n, wz)
    sp = np.zeros(n, np.uint8)
    rng = np.random.default_rng(8)
    x0 = xe + rng.normal(size=(3, n)) * 0.05 * l
    p = it.make_params(_trap(gamma=0.0, T_bath=0.0), flags=it.IONTRAP_PSEUDO)
    with it.Simulation([iongen.CA40], sp, x0, None, p) as s:
        s.set_pseudo_frequencies([(wr, wr, wz)])
        s.minimize(100000, 0.05 * l, 1e-6 * M_CA * wz ** 2 * l)
        xm = s.state()[0]
        H = s.hessian()
    w_ax = np.sqrt(np.linalg.eigvalsh(H.reshape(3 * n, 3 * n)[2::3, 2::3])) / wz
    assert abs(w_ax[0] - 1) < 1e-5 and abs(w_ax[1] - math.sqrt(3)) < 1e-5
    v0 = rng.normal(size=(3, n)) * 0.02
    stride, samples = 10, 4096
    zs = np.empty((samples, n))
    with it.Simulation([iongen.CA40], sp, xm, v0, p) as s:
        s.set_pseudo_frequencies([(wr, wr, wz)])
        for k in range(samples):
            s.step(stride)
            zs[k] = s.state()[0][2]
    zs -= zs.mean(axis=0)
    spec = np.abs(np.fft.rfft(zs * np.hanning(samples)[:, None], axis=0)).sum(axis=1)
    freqs = np.fft.rfftfreq(samples, d=stride * DT) * 2 * math.pi / wz
    peaks = [freqs[i] for i in range(1, len(spec) - 1) if spec[i] > spec[i - 1] and spec[i] > spec[i + 1]
             and spec[i] > 0.02 * spec.max()]
    for w in w_ax:
        assert min(abs(f - w) for f in peaks) < 1.5 * freqs[1], (w, peaks)


def test_minimize_and_hessian_reject_the_rf_trap(it):
    species, sp, x0, v0 = _cloud(50, 3)
    with it.Simulation(species, sp, x0, v0, it.make_params(_trap())) as s:
        for call in (lambda: s.minimize(10, 1e-6, 0.0), lambda: s.hessian(), lambda: s.set_pseudo_frequencies(FREQS)):
            with pytest.raises(it.IonTrapError) as e:
                call()
            assert e.value.code == it.IONTRAP_EINVAL
