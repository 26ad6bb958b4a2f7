"""Failure detection on the GPU, tested without a fault.

Every wait of the persistent forms (a CTA's poller waiting for the other CTAs on a step
or group counter, a CTA waiting for its bulk copies) is bounded: past its limit the
kernel sets the handle's timeout flag and returns, and the host reads IONTRAP_ETIMEOUT.
Here a test makes such a wait expire on purpose: iontrap_test_stall shortens the limit to
1 ms and has one CTA withhold its arrival on the grid-wide step counter, a counter value
that then nothing reaches.  No kernel waits longer than the limit, nothing traps, and the
context stays usable: a fresh handle on the same device then runs normally.
"""
import math
import time

import numpy as np
import pytest

import iongen
import oracle

pytestmark = pytest.mark.gpu

LIMIT_NS = 1_000_000  # 1 ms: a step of these clouds takes ~10 us


@pytest.fixture(scope="module")
def it():
    from paper_1907_10514_gb300 import build
    build.build()
    import paper_1907_10514_gb300 as mod
    return mod


def _cloud(n, seed):
    rng = np.random.default_rng(seed)
    species = [iongen.CA40, iongen.NH3]
    sp = rng.integers(0, 2, size=n).astype(np.uint8)
    x = iongen.gaussian_positions(n, 60e-6, seed=[seed, 2])
    trap = iongen.Trap(Omega=iongen.OMEGA_RF, a=-0.001, q=0.25, omega_z=2 * math.pi * 0.2e6,
                       gamma=1e5, T_bath=1e-3, dt=iongen.rf_period_dt(iongen.OMEGA_RF), seed=seed)
    return species, sp, x, trap


def _rel_rms(a, b):
    return math.sqrt(float(((a - b) ** 2).sum()) / float((b ** 2).sum()))


# (threads, ions per thread, packed, jsplit, fused) of a row-persistent launch (5; also
# with two ions per thread) and a grid-persistent one (4), of 3000 ions
FORMS = {"row-persistent": (512, 1, 1, 20, 5), "row-persistent-2ipt": (512, 2, 1, 20, 5),
         "grid-persistent": (256, 2, 1, -(-3000 // 25), 4)}


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("cta,at_step", [(3, 5), (0, 0), (-1, 0)], ids=["cta3_step5", "cta0_step0", "no_stall"])
def test_bounded_wait_expires_with_a_timeout_status(it, form, cta, at_step):
    n = 3000
    species, sp, x0, trap = _cloud(n, 901)
    with it.Simulation(species, sp, x0, None, it.make_params(trap)) as sim:
        sim.set_config(*FORMS[form])
        assert sim.config()[4] == FORMS[form][4]
        ctas = -(-n // 20) if form.startswith("row-persistent") else (-(-n // 512)) * 25
        with pytest.raises(it.IonTrapError) as e:
            it.iontrap_test_stall(sim.handle, LIMIT_NS, ctas, 0)  # no such CTA
        assert e.value.code == it.IONTRAP_EINVAL
        it.iontrap_test_stall(sim.handle, LIMIT_NS, cta, at_step)
        t0 = time.perf_counter()
        sim.step(100)  # one cooperative launch of 100 steps
        if cta < 0:  # the short limit alone changes nothing
            sim.sync()
            assert sim.state()[2] == 100
            return
        with pytest.raises(it.IonTrapError) as e:
            sim.sync()
        elapsed = time.perf_counter() - t0
        assert e.value.code == it.IONTRAP_ETIMEOUT
        assert elapsed < 1.0, elapsed  # gave up after the 1 ms limit, not the default 2 s
        x, v, step, _ = it.iontrap_state(sim.handle, n, accept=(it.IONTRAP_ETIMEOUT,))
        assert step == 0  # the step index is not advanced by a failed launch
        if form.startswith("row-persistent"):  # its FP64 state is written in a launch's last step only
            assert np.array_equal(x, x0) and np.array_equal(v, np.zeros_like(v))
        with pytest.raises(it.IonTrapError) as e:  # the status is sticky
            sim.step(1)
        assert e.value.code == it.IONTRAP_ETIMEOUT

    # the device and the library are still usable: a fresh handle runs normally
    q, m, qm0 = oracle.ion_arrays(species, sp)
    xo, _, _ = oracle.run(x0, np.zeros_like(x0), q, m, oracle.params(trap, qm0), 30)
    with it.Simulation(species, sp, x0, None, it.make_params(trap)) as sim:
        sim.set_config(*FORMS[form])
        sim.step(30)
        x, _, step, _ = sim.state()
    assert step == 30 and _rel_rms(x, xo) < 1e-4
