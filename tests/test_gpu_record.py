"""GPU parity of strided state capture and secular time averages (dump and timeAvg of
Sec. 3 "Writing/reading data") through the C ABI.

Records of x and v are the states the handle passes through, bit for bit; the windowed
velocity average (computed on the device from four positions) matches the mean of the
velocities read back step by step within 1e-10 relative (rounding of the position
differences), and the FP64 oracle's step-by-step sums within the trajectory tolerances
(FP64 form 1e-9 for positions, 1e-8 for velocities; FP32 form 1e-4 and 1e-3).
"""
import math

import numpy as np
import pytest

import iongen
import oracle

pytestmark = pytest.mark.gpu

SR88 = iongen.Species(88.0, 2.0)
DT = iongen.rf_period_dt(iongen.OMEGA_RF)


@pytest.fixture(scope="module")
def it():
    from paper_1907_10514_gb300 import build
    build.build()
    import paper_1907_10514_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def rel_rms(a, b):
    return math.sqrt(float(((a - b) ** 2).sum()) / float((b ** 2).sum()))


def _cloud(n, seed, species=(iongen.CA40, iongen.NH3, SR88)):
    rng = np.random.default_rng(seed)
    sp = rng.integers(0, len(species), size=n).astype(np.uint8)
    sp[0] = 0
    x = iongen.gaussian_positions(n, 40e-6, seed=[seed, 7])
    trap = iongen.Trap(Omega=iongen.OMEGA_RF, a=-0.001, q=0.25, omega_z=2 * math.pi * 0.2e6, gamma=1e5,
                       T_bath=1e-3, dt=DT, seed=seed)
    return list(species), sp, x, rng.normal(scale=0.3, size=(3, n)), trap


def _record(it, torch, sim, n, n_steps, every, fields, W):
    nf = bin(fields).count("1")
    buf = torch.zeros((n_steps // every) * nf * 3 * n, dtype=torch.float64, device="cuda")
    sim.step_record(n_steps, every, fields, W, buf.data_ptr())
    sim.sync()
    return buf.cpu().numpy().reshape(n_steps // every, nf, 3, n)


@pytest.mark.parametrize("n,prec,cfg", [(500, 0, None), (2500, 0, None), (700, 0, (128, 2, 1, 100, 3)),
                                        (1500, 0, (512, 1, 1, 10, 5)), (1500, 0, (512, 2, 1, 10, 5)),
                                        (300, 1, None)])
def test_records_are_the_states_passed_through(it, torch, n, prec, cfg):
    """x and v records equal the states of a twin handle stepped to the same indices (bit
    for bit); the device time average equals the mean of the twin's velocities read after
    every step of the window."""
    species, sp, x0, v0, trap = _cloud(n, 31)
    p = it.make_params(trap, precision=prec)
    every, W, K = 7, 5, 6
    fields = it.IONTRAP_REC_X | it.IONTRAP_REC_V | it.IONTRAP_REC_VAVG
    with it.Simulation(species, sp, x0, v0, p) as a, it.Simulation(species, sp, x0, v0, p) as b:
        if cfg:
            a.set_config(*cfg)
            b.set_config(*cfg)
        rec = _record(it, torch, a, n, every * K, every, fields, W)
        for k in range(K):
            b.step(every - W)
            vs = np.zeros((3, n))
            for _ in range(W):
                b.step(1)
                x, v, step, _ = b.state()
                vs += v
            assert step == (k + 1) * every
            assert np.array_equal(rec[k, 0], x) and np.array_equal(rec[k, 1], v)
            np.testing.assert_allclose(rec[k, 2], vs / W, rtol=0, atol=1e-10 * np.abs(vs / W).max())
        assert a.state()[2] == every * K


@pytest.mark.parametrize("prec", [0, 1])
def test_records_match_oracle(it, torch, prec):
    """Records every RF period (20 steps) with the average over the period (the secular
    velocity of Example 1), against the oracle summing the velocities step by step."""
    n = 300
    species, sp, x0, v0, trap = _cloud(n, 5)
    q, m, qm0 = oracle.ion_arrays(species, sp)
    X, V, VA, _ = oracle.record(x0, v0, q, m, oracle.params(trap, qm0), 100, 20, 20)
    fields = it.IONTRAP_REC_X | it.IONTRAP_REC_V | it.IONTRAP_REC_VAVG
    with it.Simulation(species, sp, x0, v0, it.make_params(trap, precision=prec)) as s:
        rec = _record(it, torch, s, n, 100, 20, fields, 20)
    xt, vt = (1e-9, 1e-8) if prec else (1e-4, 1e-3)
    for k in range(5):
        assert rel_rms(rec[k, 0], X[k]) < xt
        assert rel_rms(rec[k, 1], V[k]) < vt
        assert rel_rms(rec[k, 2], VA[k]) < vt


def test_single_fields_and_layout(it, torch):
    """Each field alone, and x with the average only: the layout packs the requested
    fields in the order x, v, v_avg."""
    species, sp, x0, v0, trap = _cloud(200, 9)
    p = it.make_params(trap)
    outs = {}
    for fields in (it.IONTRAP_REC_X, it.IONTRAP_REC_V, it.IONTRAP_REC_VAVG,
                   it.IONTRAP_REC_X | it.IONTRAP_REC_VAVG):
        with it.Simulation(species, sp, x0, v0, p) as s:
            outs[fields] = _record(it, torch, s, 200, 60, 20, fields, 10)
    both = outs[it.IONTRAP_REC_X | it.IONTRAP_REC_VAVG]
    assert np.array_equal(both[:, 0], outs[it.IONTRAP_REC_X][:, 0])
    assert np.array_equal(both[:, 1], outs[it.IONTRAP_REC_VAVG][:, 0])


def test_record_rejects_bad_arguments(it, torch):
    species, sp, x0, v0, trap = _cloud(50, 2)
    buf = torch.zeros(10 * 3 * 3 * 50, dtype=torch.float64, device="cuda")
    with it.Simulation(species, sp, x0, v0, it.make_params(trap)) as s:
        for args in ((21, 20, 1, 1), (20, 0, 1, 1), (20, 20, 0, 1), (20, 20, 8, 1), (20, 10, 4, 11), (20, 10, 4, 0)):
            with pytest.raises(it.IonTrapError) as e:
                s.step_record(*args, buf.data_ptr())
            assert e.value.code == it.IONTRAP_EINVAL
        s.step(3)
        assert s.state()[2] == 3


def test_example1_crystal_forms(it, torch):
    """Sec. 4 Example 1: 100 Ca+ (40 amu) from a 1 mm cloud in linearPT(300 V, 7 V,
    2.75 mm, 3.5 mm, 0.3, 3.85 MHz) with a 1 mK bath of damping time 10 us, 20 000 steps,
    secular velocities (timeAvg over one RF period) dumped every period.  The secular
    temperature falls from the initial cloud's to the bath's (within a factor of 2 over
    the last 2 000 steps) and the ions settle on lattice sites: the RMS scatter of the
    once-per-period positions over the last 100 periods is below a tenth of the median
    nearest-neighbour distance (Lindemann's melting criterion), a crystal."""
    n = 100
    rng = np.random.default_rng(1)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    x0 = np.ascontiguousarray((d * 1e-3 * rng.uniform(size=(n, 1)) ** (1 / 3)).T)
    ca = iongen.Species(40.0, 1.0)
    p = it.iontrap_linear_pt(300.0, 7.0, 2.75e-3, 3.5e-3, 0.3, 2 * math.pi * 3.85e6, ca,
                             it.make_params(None, gamma=1 / 10e-6, T_bath=1e-3, seed=1))
    assert abs(p.q - 0.327) < 5e-4
    fields = it.IONTRAP_REC_X | it.IONTRAP_REC_VAVG
    with it.Simulation([ca], np.zeros(n, np.uint8), x0, None, p) as s:
        rec = _record(it, torch, s, n, 20000, 20, fields, 20)
    kb, amu = 1.380649e-23, 1.66053906660e-27
    T = 40.0 * amu * (rec[:, 1] ** 2).sum(axis=1).mean(axis=1) / (3 * kb)
    assert T[:10].mean() > 1.0  # the initial cloud: kelvins
    late = T[-100:].mean()
    assert 0.5e-3 < late < 2e-3, late
    xs = rec[-100:, 0]
    sites = xs.mean(axis=0)
    scatter = math.sqrt(float(((xs - sites) ** 2).sum(axis=1).mean()))
    d = np.sqrt(((sites[:, :, None] - sites[:, None, :]) ** 2).sum(axis=0))
    np.fill_diagonal(d, np.inf)
    assert scatter < 0.1 * float(np.median(d.min(axis=1))), (scatter, np.median(d.min(axis=1)))
