"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports every
function include/iontrap.h declares, the binding covers them all, and the host-only
entry points (status strings, trap stability) behave -- the stability check is compared
with the oracle's own Floquet computation on random trap draws."""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "iontrap.h")


@pytest.fixture(scope="module")
def native():
    from paper_1907_10514_gb300 import build
    build.build()
    import paper_1907_10514_gb300.native as nat
    return nat


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(iontrap_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("iontrap_create", "iontrap_step", "iontrap_state", "iontrap_forces",
                 "iontrap_destroy", "iontrap_strerror", "iontrap_step_many"):
        assert must in names


def test_library_exports_every_declared_symbol(native):
    import ctypes
    lib = ctypes.CDLL(native.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(native.SIGNATURES)


def test_strerror(native):
    assert native.iontrap_strerror(0) == "ok"
    for code in range(1, 7):
        assert native.iontrap_strerror(code) not in ("", "ok", "unknown status")
    assert native.iontrap_strerror(99) == "unknown status"


def test_stability_check_agrees_with_oracle(native):
    import oracle
    import iongen
    rng = np.random.default_rng(17)
    agree = 0
    for k in range(160):
        q = rng.uniform(0.05, 0.95)
        a = rng.uniform(-0.02, 0.01)
        wz = 2 * math.pi * rng.uniform(0.05e6, 0.6e6)
        trap = iongen.Trap(Omega=iongen.OMEGA_RF, a=a, q=q, omega_z=wz, gamma=1e5, T_bath=1e-3,
                           dt=iongen.rf_period_dt(iongen.OMEGA_RF), seed=k)
        species = [iongen.CA40, iongen.NH3] if k % 2 else [iongen.CA40]
        mine = native.iontrap_stable(species, native.make_params(trap))
        ref = oracle.stable(species, trap)
        assert mine == ref, (q, a, wz, k)
        agree += 1
    assert agree == 160


def test_stability_rejects_bad_parameters(native):
    p = native.make_params(None, Omega=-1.0, q=0.3, omega_z=1e6, dt=1e-8)
    with pytest.raises(native.IonTrapError) as e:
        native.iontrap_stable([(40.0, 1.0)], p)
    assert e.value.code == native.IONTRAP_EINVAL
    p = native.make_params(None, Omega=2.4e7, q=0.3, omega_z=1e6, dt=-1.0)
    with pytest.raises(native.IonTrapError):
        native.iontrap_stable([(40.0, 1.0)], p)
    with pytest.raises(native.IonTrapError):
        native.iontrap_stable([], native.make_params(None, Omega=2.4e7))


def test_linear_pt_matches_oracle(native):
    """The voltage-form trap constructor (linearPT, Eq. 1 and Eq. 3) against the oracle's,
    which the field test of test_oracle_pins.py pins to Eq. 1 itself: random geometries
    and both signs of the charge."""
    import oracle
    rng = np.random.default_rng(5)
    e, amu = oracle.const("e"), oracle.const("amu")
    for _ in range(50):
        V0, U0 = rng.uniform(50, 1000), rng.uniform(0.5, 50)
        R0, Z0, kappa = rng.uniform(0.5e-3, 5e-3), rng.uniform(1e-3, 8e-3), rng.uniform(0.05, 0.5)
        Om = 2 * math.pi * rng.uniform(1e6, 2e7)
        mass, z = rng.uniform(1, 200), rng.choice([1.0, 2.0, -1.0])
        if z < 0:
            U0 = -U0
        p = native.iontrap_linear_pt(V0, U0, R0, Z0, kappa, Om, (mass, z))
        ref = oracle.linear_pt(V0, U0, R0, Z0, kappa, Om, z * e, mass * amu)
        got = (p.Omega, p.a, p.q, p.omega_z)
        np.testing.assert_allclose(got, ref, rtol=1e-14, atol=0)


def test_linear_pt_of_the_paper_examples(native):
    """Example 1's trap (300 V, 7 V, r0 = 2.75 mm, z0 = 3.5 mm, kappa = 0.3, 3.85 MHz,
    40 amu): q = 0.327 and f_z = 0.145 MHz by Eq. 3, a trap that holds Ca+.  Example 2's
    trap as printed (252.2 V, 5 V, 10 mm, 3.5 mm, 0.3, 5.634 MHz) gives Ca+ q = 0.0097
    against an axial defocusing of Eq. 3's a_x = -9.4e-4, a + q^2/2 < 0: radially
    unconfined, which the stability check reports."""
    ca = (40.0, 1.0)
    p = native.iontrap_linear_pt(300.0, 7.0, 2.75e-3, 3.5e-3, 0.3, 2 * math.pi * 3.85e6, ca)
    assert abs(p.q - 0.327) < 5e-4 and abs(p.omega_z / (2 * math.pi) - 0.1448e6) < 100 and p.a == 0.0
    assert native.iontrap_stable([ca], p)
    p2 = native.iontrap_linear_pt(252.2, 5.0, 10e-3, 3.5e-3, 0.3, 2 * math.pi * 5.634e6, ca)
    assert abs(p2.q - 0.0097) < 1e-4
    assert not native.iontrap_stable([ca, (17.0, 1.0)], p2)
    with pytest.raises(native.IonTrapError) as e:
        native.iontrap_linear_pt(300.0, -7.0, 2.75e-3, 3.5e-3, 0.3, 2.4e7, ca)
    assert e.value.code == native.IONTRAP_EINVAL
    with pytest.raises(native.IonTrapError):
        native.iontrap_linear_pt(300.0, 7.0, 0.0, 3.5e-3, 0.3, 2.4e7, ca)
