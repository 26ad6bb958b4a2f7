"""The allocation-free force entry point, for callers that cannot allocate device memory
(their memory pool owns the device, or they host this library as a plugin, or they
cannot take cudaMalloc's implicit synchronisation).  It must give the same Coulomb
accelerations as iontrap_forces on a handle, and the FP64 oracle's, within the FP32
force tolerance of the other tests, on consecutive calls that reuse its fixed scratch
array (at n = 8192, the size limit, on sampled ions).  This file is named to be
collected last."""
import math

import numpy as np
import pytest

import iongen
import oracle

pytestmark = pytest.mark.gpu

FP32_FORCE_TOL = 1e-5


def _rel_rms(a, b):
    return math.sqrt(float(((a - b) ** 2).sum()) / float((b ** 2).sum()))


def _cloud(n, seed):
    rng = np.random.default_rng(seed)
    species = [iongen.CA40, iongen.NH3, iongen.Species(88.0, 2.0)]
    sp = rng.integers(0, len(species), size=n).astype(np.uint8)
    sp[0] = 0
    x = iongen.gaussian_positions(n, 40e-6, seed=[seed, 3])
    trap = iongen.Trap(Omega=iongen.OMEGA_RF, a=-0.001, q=0.25, omega_z=2 * math.pi * 0.2e6,
                       gamma=1e5, T_bath=1e-3, dt=iongen.rf_period_dt(iongen.OMEGA_RF), seed=seed)
    return species, sp, x, trap


def test_forces_noalloc_matches_handle_forces_on_consecutive_calls():
    import torch
    from paper_1907_10514_gb300 import build
    build.build()
    import paper_1907_10514_gb300 as it

    stream = torch.cuda.current_stream()
    for n, seed in ((3001, 21), (1200, 22), (8192, 23)):
        species, sp, x, trap = _cloud(n, seed)
        with it.Simulation(species, sp, x, None, it.make_params(trap)) as sim:
            ref = sim.forces()
        d_x = torch.tensor(x, dtype=torch.float64, device="cuda").contiguous()
        d_sp = torch.tensor(sp, dtype=torch.uint8, device="cuda")
        d_acc = torch.full((3, n), float("nan"), dtype=torch.float64, device="cuda")
        it.iontrap_forces_noalloc(species, d_sp.data_ptr(), d_x.data_ptr(), n, d_acc.data_ptr(), stream)
        torch.cuda.synchronize()
        got = d_acc.cpu().numpy()
        assert np.isfinite(got).all()
        assert _rel_rms(got, ref) < FP32_FORCE_TOL, n
        # against the FP64 oracle (all ions, or 512 sampled ones at the size limit)
        q, m, _ = oracle.ion_arrays(species, sp)
        idx = np.arange(n) if n < 8192 else np.random.default_rng(seed).choice(n, 512, replace=False)
        exact = oracle.coulomb_accel(x, q, m, idx=idx)
        assert _rel_rms(got[:, idx], exact) < FP32_FORCE_TOL, n


def test_forces_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1907_10514_gb300 import build
    build.build()
    import paper_1907_10514_gb300 as it
    with pytest.raises(it.IonTrapError) as e:
        it.iontrap_forces_noalloc([iongen.CA40], 1, 1, 8193, 1)  # checked before any device access
    assert e.value.code == it.IONTRAP_ETOOLARGE
