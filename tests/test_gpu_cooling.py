"""GPU parity of species-selective cooling, laser cooling and forces changed between
evolve calls (iontrap_set_params) against the FP64 oracle, through the C ABI.

Sec. 3 "Cooling the motion of ions" (a bath on a group of ions, laserCool on a species)
and Sec. 3 "Time evolution" (forces added or removed between evolve calls, as Example 2
of Sec. 4 does).  Tolerances as in test_gpu_parity.py: FP32 form trajectories within
1e-4 relative RMS (velocities 1e-3), plain FP64 form 1e-9, over 80 steps (these clouds
amplify FP32-sized differences chaotically to ~1e-4 by step 100); the laser decay of free
ions, which involves no FP32 arithmetic, within 1e-12 of its closed form; the
sympathetic-cooling example by its temperatures (statistics of a chaotic many-ion run),
with the oracle running the same protocol beside it.
"""
import math

import numpy as np
import pytest

import iongen
import oracle
from iongen import Cooling

pytestmark = pytest.mark.gpu

FP32_TRAJ_TOL = 1e-4
FP64_TRAJ_TOL = 1e-9
SR88 = iongen.Species(88.0, 2.0)


@pytest.fixture(scope="module")
def it():
    from paper_1907_10514_gb300 import build
    build.build()
    import paper_1907_10514_gb300 as mod
    return mod


def rel_rms(a, b):
    return math.sqrt(float(((a - b) ** 2).sum()) / float((b ** 2).sum()))


def _unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


def _cloud(n, seed, species=(iongen.CA40, iongen.NH3, SR88)):
    rng = np.random.default_rng(seed)
    sp = rng.integers(0, len(species), size=n).astype(np.uint8)
    sp[0] = 0
    x = iongen.gaussian_positions(n, 40e-6, seed=[seed, 7])
    trap = iongen.Trap(Omega=iongen.OMEGA_RF, a=-0.001, q=0.25, omega_z=2 * math.pi * 0.2e6,
                       gamma=1e5, T_bath=1e-3, dt=iongen.rf_period_dt(iongen.OMEGA_RF), seed=seed)
    return iongen.Workload(f"cloud{n}", list(species), sp, x,
                           np.random.default_rng(seed + 1).normal(scale=0.3, size=(3, n)), trap, 100)


# two phases: baths and lasers per species, then a changed trap with the Ca bath removed
COOL1 = [Cooling(1e5, 1e-3, tuple(2e5 * _unit([1.0, 2.0, -0.5]))), Cooling(0.0, 0.0, (3e5, 0.0, 0.0)),
         Cooling(3e5, 5e-3)]
COOL2 = [Cooling(0.0, 0.0, tuple(2.5e5 * _unit([0.2, -1.0, 1.0]))), Cooling(2e5, 2e-3), Cooling()]


def _trap2(trap):
    t = iongen.Trap(**vars(trap))
    t.q, t.omega_z = 0.28, 2 * math.pi * 0.25e6
    return t


def _oracle_two_phase(w, k1, k2):
    q, m, qm0 = oracle.ion_arrays(w.species, w.species_of_ion)
    p1 = oracle.params(w.trap, qm0)
    p2 = oracle.params(_trap2(w.trap), qm0)
    c1 = oracle.cooling_arrays(w.species_of_ion, COOL1)
    c2 = oracle.cooling_arrays(w.species_of_ion, COOL2)
    x, v, _ = oracle.run(w.x0, w.v0, q, m, p1, k1, cooling=c1)
    return oracle.run(x, v, q, m, p2, k2, step0=k1, cooling=c2)


def _gpu_two_phase(it, sims, ws, k1, k2, batched=False, prec=0):
    for s, w in zip(sims, ws):
        s.set_params(it.make_params(w.trap, precision=prec), COOL1)
    if batched:
        it.iontrap_step_many([s.handle for s in sims], [k1] * len(sims))
    else:
        for s in sims:
            s.step(k1)
    for s, w in zip(sims, ws):
        s.set_params(it.make_params(_trap2(w.trap), precision=prec), COOL2)
    if batched:
        it.iontrap_step_many([s.handle for s in sims], [k2] * len(sims))
    else:
        for s in sims:
            s.step(k2)
    return [s.state() for s in sims]


def _gp_cfg(n, W, S):
    return (32 * W, 2, 1, -(-n // S), 4)


@pytest.mark.parametrize("form", ["last_cta", "separate_epilogue", "cluster", "cluster_warps", "persistent",
                                  "row_persistent", "row_persistent_i2", "fp64"])
def test_two_phase_cooling_matches_oracle(it, form):
    """Per-species baths and lasers, then a changed trap and cooling, in every kernel form
    of a single simulation: 40 + 40 steps against the oracle doing the same (this cloud
    amplifies FP32-sized differences chaotically to ~1e-4 by step 100)."""
    n = 3000
    w = _cloud(n, 71)
    xo, vo, _ = _oracle_two_phase(w, 40, 40)
    prec = 1 if form == "fp64" else 0
    cfg = {"last_cta": (128, 2, 1, -(-n // 12), 1), "separate_epilogue": (64, 4, 1, 256, 0),
           "cluster": (128, 1, 0, -(-n // 8), 2), "cluster_warps": (128, 2, 1, -(-n // 8), 3),
           "persistent": _gp_cfg(n, 8, 25), "row_persistent": (512, 1, 1, 20, 5),
           "row_persistent_i2": (512, 2, 1, 20, 5), "fp64": None}[form]
    with it.Simulation(w.species, w.species_of_ion, w.x0, w.v0, it.make_params(w.trap, precision=prec)) as sim:
        if cfg:
            sim.set_config(*cfg)
            assert sim.config()[:5] == cfg
        (x, v, step, _), = _gpu_two_phase(it, [sim], [w], 40, 40, prec=prec)
    tol = FP64_TRAJ_TOL if prec else FP32_TRAJ_TOL
    assert step == 80
    assert rel_rms(x, xo) < tol and rel_rms(v, vo) < 10 * tol, (rel_rms(x, xo), rel_rms(v, vo))


@pytest.mark.parametrize("n", [40, 300, 1500])
def test_two_phase_cooling_batched_matches_oracle(it, n):
    """The same two phases through the batched resident kernel (one-warp, one-CTA and
    cluster packing classes), ensembles advanced together."""
    ws = [_cloud(n, 90 + n), _cloud(max(2, n // 3), 91 + n)]
    sims = [it.Simulation(w.species, w.species_of_ion, w.x0, w.v0, it.make_params(w.trap)) for w in ws]
    try:
        out = _gpu_two_phase(it, sims, ws, 40, 40, batched=True)
    finally:
        for s in sims:
            s.close()
    for w, (x, v, step, _) in zip(ws, out):
        xo, vo, _ = _oracle_two_phase(w, 40, 40)
        assert step == 80
        assert rel_rms(x, xo) < FP32_TRAJ_TOL and rel_rms(v, vo) < 10 * FP32_TRAJ_TOL


@pytest.mark.parametrize("n,prec", [(2500, 0), (700, 0), (300, 1)])
def test_set_params_continues_like_a_fresh_handle(it, n, prec):
    """After iontrap_set_params at step k the handle continues bit for bit like a handle
    created from (x_k, v_k) at step0 = k with the new forces (default configurations:
    the row-persistent form at n = 2500)."""
    w = _cloud(n, 17)
    p1 = it.make_params(w.trap, precision=prec)
    p2 = it.make_params(_trap2(w.trap), precision=prec)
    with it.Simulation(w.species, w.species_of_ion, w.x0, w.v0, p1) as a:
        a.step(130)
        xk, vk, k, _ = a.state()
        a.set_params(p2, COOL2)
        a.step(120)
        xa, va, sa, _ = a.state()
    with it.Simulation(w.species, w.species_of_ion, xk, vk, p2, step0=k) as b:
        b.set_params(p2, COOL2)
        b.step(120)
        xb, vb, sb, _ = b.state()
    assert sa == sb == 250
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_set_params_without_cooling_is_the_default_bath(it):
    """cooling = NULL puts every species in the bath of iontrap_params, no laser: the same
    bits as a per-species table that gives each species that bath."""
    w = _cloud(900, 5)
    p = it.make_params(w.trap)
    table = [Cooling(w.trap.gamma, w.trap.T_bath)] * 3
    out = []
    for cool in (None, table):
        with it.Simulation(w.species, w.species_of_ion, w.x0, w.v0, p) as s:
            s.set_params(p, cool)
            s.step(150)
            out.append(s.state())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_laser_cooling_free_ions_closed_form(it):
    """Free ions laser-cooled along a random direction (the paper's laser-cooling check,
    Sec. 5 'Cooling mechanisms'): the projection decays as (1 - L dt/2)^2 (1 - L dt)^(k-1)
    and the perpendicular components stay put; a species without a laser does not move."""
    n = 257
    rng = np.random.default_rng(4)
    sp = (np.arange(n) % 2).astype(np.uint8)
    k = _unit(rng.normal(size=3))
    L = 1e6
    dt = iongen.rf_period_dt(iongen.OMEGA_RF)
    v0 = rng.normal(size=(3, n)) * 2.0
    x0 = iongen.gaussian_positions(n, 30e-6, seed=4)
    trap = iongen.Trap(Omega=iongen.OMEGA_RF, a=0.0, q=0.3, omega_z=2 * math.pi * 0.2e6, gamma=0.0, T_bath=0.0,
                       dt=dt, seed=1)
    flags = it.IONTRAP_TRAP_OFF | it.IONTRAP_COULOMB_OFF
    for prec in (0, 1):
        p = it.make_params(trap, precision=prec, flags=flags)
        with it.Simulation([iongen.CA40, iongen.NH3], sp, x0, v0, p) as s:
            s.set_params(p, [Cooling(laser=tuple(L * k)), Cooling()])
            done = 0
            for steps in (1, 40, 300):
                s.step(steps - done)
                done = steps
                _, v, _, _ = s.state()
                pn, p0 = k @ v, k @ v0
                c = sp == 0
                expect = (1 - L * dt / 2) ** 2 * (1 - L * dt) ** (steps - 1) * p0
                np.testing.assert_allclose(pn[c], expect[c], rtol=1e-11, atol=1e-14 * np.abs(v0).max())
                perp = v - np.outer(k, pn)
                np.testing.assert_allclose(perp[:, c], (v0 - np.outer(k, p0))[:, c], rtol=0,
                                           atol=1e-12 * np.abs(v0).max())
                assert np.array_equal(v[:, ~c], v0[:, ~c])


def test_set_params_rejects_bad_changes(it):
    """dt, seed, precision and the Coulomb switch are fixed at creation; bath values must
    be finite and non-negative; a trap that cannot hold a species is refused.  Argument
    errors leave the handle usable."""
    w = _cloud(200, 8)
    p = it.make_params(w.trap)
    with it.Simulation(w.species, w.species_of_ion, w.x0, w.v0, p) as s:
        bad = [it.make_params(w.trap, dt=w.trap.dt * 1.01), it.make_params(w.trap, seed=w.trap.seed + 1),
               it.make_params(w.trap, precision=1), it.make_params(w.trap, flags=it.IONTRAP_COULOMB_OFF)]
        for bp in bad:
            with pytest.raises(it.IonTrapError) as e:
                s.set_params(bp)
            assert e.value.code == it.IONTRAP_EINVAL
        for cool in ([Cooling(-1.0, 1e-3)] * 3, [Cooling(1e5, -1e-3)] * 3, [Cooling(laser=(math.nan, 0, 0))] * 3):
            with pytest.raises(it.IonTrapError) as e:
                s.set_params(p, cool)
            assert e.value.code == it.IONTRAP_EINVAL
        with pytest.raises(it.IonTrapError) as e:
            s.set_params(it.make_params(w.trap, q=0.95))
        assert e.value.code == it.IONTRAP_EUNSTABLE
        s.step(10)
        assert s.state()[2] == 10


def _secular_temps(x_a, x_b, dt, mass, sp):
    """Temperatures from the secular velocities: the velocity averaged over one RF period
    (Example 2 dumps timeAvg(v, 1/RF)) is the position change over that period divided by
    it; 3 k_B T = M <v_sec^2> per species."""
    vs = (x_b - x_a) / (20 * dt)
    t = mass * (vs ** 2).sum(axis=0) / (3 * oracle.const("kB"))
    return np.array([t[sp == s].mean() for s in range(int(sp.max()) + 1)])


def test_sympathetic_cooling_example(it):
    """Sec. 4 Example 2: 50 Ca+ and 20 NH3+ from a 0.5 mm cloud, both in a 1 mK bath
    (damping time 30 us) for 100 000 steps; then the bath is removed and the Ca+ ions are
    laser-cooled along x (g = (1e5, 0, 0) 1/s) for 120 000 steps.  Both species settle
    near 1 mK in the bath; afterwards the Ca+ temperature drops by more than an order of
    magnitude and the NH3+ ions, cooled only through their Coulomb coupling to Ca+, follow
    more slowly.  The example's rf (5.634 MHz), ion numbers, cloud, bath, laser and step
    counts are kept; its printed voltages leave Ca+ radially unconfined, so the trap is
    q = 0.1, a = 0, f_z = 50 kHz for Ca+ (NH3+ at q = 0.235).  The oracle runs the same
    protocol and must show the same temperatures within the statistics."""
    n_ca, n_nh3 = 50, 20
    sp = np.concatenate([np.zeros(n_ca, np.uint8), np.ones(n_nh3, np.uint8)])
    species = [iongen.CA40, iongen.NH3]
    n = n_ca + n_nh3
    rng = np.random.default_rng(5)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    x0 = np.ascontiguousarray((d * 5e-4 * rng.uniform(size=(n, 1)) ** (1 / 3)).T)
    Om = 2 * math.pi * 5.634e6
    dt = iongen.rf_period_dt(Om)
    trap = iongen.Trap(Omega=Om, a=0.0, q=0.1, omega_z=2 * math.pi * 0.05e6, gamma=1 / 30e-6, T_bath=1e-3,
                       dt=dt, seed=5)
    laser = [Cooling(0.0, 0.0, (1e5, 0.0, 0.0)), Cooling()]
    q, m, qm0 = oracle.ion_arrays(species, sp)
    K1, K2, every = 100000, 120000, 5000

    gpu = []
    p = it.make_params(trap)
    with it.Simulation(species, sp, x0, None, p) as s:
        for phase, K in enumerate((K1, K2)):
            if phase == 1:
                s.set_params(p, laser)
            for _ in range(K // every):
                s.step(every - 20)
                xa = s.state()[0]
                s.step(20)
                gpu.append(_secular_temps(xa, s.state()[0], dt, m, sp))
        assert s.state()[2] == K1 + K2
    ref = []
    po = oracle.params(trap, qm0)
    x, v, done = x0, np.zeros((3, n)), 0
    for phase, K in enumerate((K1, K2)):
        c = oracle.cooling_arrays(sp, laser) if phase == 1 else None
        a = None
        for _ in range(K // every):
            x, v, a = oracle.run(x, v, q, m, po, every - 20, step0=done, a0=a, cooling=c)
            xa = x
            x, v, a = oracle.run(x, v, q, m, po, 20, step0=done + every - 20, a0=a, cooling=c)
            done += every
            ref.append(_secular_temps(xa, x, dt, m, sp))
    for T in (np.array(gpu), np.array(ref)):
        bath = T[12:20].mean(axis=0)           # 60 000 - 100 000 steps: in the bath
        late = T[-8:].mean(axis=0)             # the last 40 000 steps of laser cooling
        early = T[20:24].mean(axis=0)          # the first 20 000 steps of laser cooling
        assert np.all(np.abs(bath / 1e-3 - 1) < 0.35), bath
        assert late[0] < 0.05 * bath[0], (late, bath)
        assert late[1] < 0.5 * bath[1], (late, bath)
        assert late[1] > 2 * late[0] and early[1] / bath[1] > early[0] / bath[0]
