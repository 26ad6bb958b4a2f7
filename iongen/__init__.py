"""Seeded synthetic ion-cloud workloads for the trapped-ion timestep.

This module only *draws inputs*: ion counts, species labels, initial positions and
velocities, and trap parameter sets.  It holds none of the method's arithmetic
(no forces, no trap fields, no integration), so that the FP64 oracle and the CUDA
library can both consume its arrays without sharing any code of the method.

The paper places ions "randomly" inside a cloud of a given radius (Sec. 3,
"Adding ions") and runs its examples on ion clouds of 20-100 ions (Sec. 4).  The
workloads below are the five synthetic configurations the library is measured on:

  plain_n64        64 Ca+ in a 50 um cube, Omega = 2 pi 3.85 MHz, q = 0.3, a = 0,
                   f_z = 0.2 MHz, Langevin 1e5 1/s to 1 mK, dt = T_RF/20, 10 000 steps
  mix_n4096        3072 Ca+ then 1024 NH3+, isotropic Gaussian sigma = 100 um,
                   thermal 10 mK, a = -0.001, 5 000 steps
  crystal_n32768   32768 Ca+ in a uniform prolate spheroid (400 um, 400 um, 1.2 mm),
                   q = 0.2, f_z = 0.05 MHz, gamma = 2e5 1/s, 1 000 steps
  batched_512      512 independent Ca+ ensembles, N log-uniform in [16, 2048],
                   q ~ U[0.1, 0.4], a ~ U[-0.005, 0], f_z ~ U[0.1, 0.5] MHz
  serve_stream     Poisson arrivals at 200 requests/s, N log-uniform in [8, 65536],
                   step budget log-uniform in [1e3, 1e5], Ca+ or an 80/20 Ca+/NH3+ mix

Positions are SoA arrays of shape (3, N) in metres, velocities (3, N) in m/s.
Every ion is at least ``min_spacing`` (1 um) from every other ion; candidates closer
than that are redrawn (the higher ion id of each offending pair is redrawn from the
same stream until no pair is left), which makes the draw a function of the seed only.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Iterator, List, Optional, Sequence

import numpy as np

# Input-side constants (CODATA 2018).  Used only to draw thermal velocities and to
# express the RF period; each consumer of these arrays defines its own constants.
AMU_KG = 1.66053906660e-27
KB_J_PER_K = 1.380649e-23

CA40_AMU = 39.96
NH3_AMU = 17.03


@dataclasses.dataclass(frozen=True)
class Species:
    mass_amu: float
    charge_e: float


CA40 = Species(CA40_AMU, 1.0)
NH3 = Species(NH3_AMU, 1.0)


@dataclasses.dataclass
class Trap:
    """Linear Paul trap + Langevin bath parameters (Mathieu a/q form, Eq. 3).

    ``a`` and ``q`` (q_x = -q_y = q) and ``omega_z`` belong to species 0; ``dt`` of 0
    means one twentieth of the RF period.
    """
    Omega: float
    a: float
    q: float
    omega_z: float
    gamma: float
    T_bath: float
    dt: float
    seed: int = 0
    flags: int = 0


@dataclasses.dataclass
class Cooling:
    """Cooling of one species (Sec. 3, "Cooling the motion of ions"): its Langevin
    bath (rate 1/dampingTime in 1/s, temperature in K; gamma 0 = no bath) and its
    laser-cooling vector in 1/s (zero vector = no laser).  Plain data."""
    gamma: float = 0.0
    T_bath: float = 0.0
    laser: tuple = (0.0, 0.0, 0.0)


@dataclasses.dataclass
class Workload:
    name: str
    species: List[Species]
    species_of_ion: np.ndarray     # uint8 (N,)
    x0: np.ndarray                 # float64 (3, N)
    v0: np.ndarray                 # float64 (3, N)
    trap: Trap
    steps: int
    redraws: int = 0               # trap draws rejected as unstable before this one

    @property
    def n(self) -> int:
        return int(self.species_of_ion.shape[0])


def rf_period_dt(Omega: float, per_period: int = 20) -> float:
    """Time step that divides one RF period into ``per_period`` steps."""
    return 2.0 * math.pi / Omega / per_period


# ----------------------------------------------------------------------------------
# position samplers (unit-free shapes scaled to metres)
# ----------------------------------------------------------------------------------

def _with_min_spacing(draw: Callable[[np.random.Generator, int], np.ndarray],
                      n: int, rng: np.random.Generator, dmin: float) -> np.ndarray:
    from scipy.spatial import cKDTree

    pts = draw(rng, n)
    for _ in range(10000):
        if n < 2:
            break
        pairs = cKDTree(pts).query_pairs(dmin, output_type="ndarray")
        if len(pairs) == 0:
            break
        bad = np.unique(pairs.max(axis=1))
        pts[bad] = draw(rng, len(bad))
    else:  # pragma: no cover - only for absurd densities
        raise RuntimeError("could not place ions with the requested minimum spacing")
    return np.ascontiguousarray(pts.T)


def cube_positions(n: int, side: float, seed, dmin: float = 1e-6) -> np.ndarray:
    """Uniform in the cube [-side/2, side/2]^3."""
    rng = np.random.default_rng(seed)
    return _with_min_spacing(lambda r, k: r.uniform(-side / 2, side / 2, size=(k, 3)),
                             n, rng, dmin)


def gaussian_positions(n: int, sigma: float, seed, dmin: float = 1e-6) -> np.ndarray:
    """Isotropic Gaussian with standard deviation ``sigma`` per axis."""
    rng = np.random.default_rng(seed)
    return _with_min_spacing(lambda r, k: r.normal(0.0, sigma, size=(k, 3)), n, rng, dmin)


def spheroid_positions(n: int, a_xy: float, c_z: float, seed, dmin: float = 1e-6) -> np.ndarray:
    """Uniform in the prolate spheroid x^2/a^2 + y^2/a^2 + z^2/c^2 <= 1 (long axis z)."""
    rng = np.random.default_rng(seed)

    def draw(r: np.random.Generator, k: int) -> np.ndarray:
        d = r.normal(size=(k, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        rad = r.uniform(size=(k, 1)) ** (1.0 / 3.0)
        return d * rad * np.array([a_xy, a_xy, c_z])

    return _with_min_spacing(draw, n, rng, dmin)


def thermal_velocities(species: Sequence[Species], species_of_ion: np.ndarray,
                       T: float, seed) -> np.ndarray:
    """Maxwell-Boltzmann velocities: each component N(0, k_B T / M)."""
    rng = np.random.default_rng(seed)
    m = np.array([species[s].mass_amu * AMU_KG for s in species_of_ion])
    sd = np.sqrt(KB_J_PER_K * T / m)
    return np.ascontiguousarray(rng.normal(size=(3, len(m))) * sd[None, :])


# ----------------------------------------------------------------------------------
# the five measured workloads
# ----------------------------------------------------------------------------------

TWO_PI = 2.0 * math.pi
OMEGA_RF = TWO_PI * 3.85e6


def plain_n64() -> Workload:
    n = 64
    trap = Trap(Omega=OMEGA_RF, a=0.0, q=0.3, omega_z=TWO_PI * 0.2e6, gamma=1e5,
                T_bath=1e-3, dt=rf_period_dt(OMEGA_RF), seed=0)
    return Workload("plain_n64", [CA40], np.zeros(n, np.uint8),
                    cube_positions(n, 50e-6, seed=0), np.zeros((3, n)), trap, 10000)


def mix_n4096() -> Workload:
    n_ca, n_nh3 = 3072, 1024
    n = n_ca + n_nh3
    sp = np.concatenate([np.zeros(n_ca, np.uint8), np.ones(n_nh3, np.uint8)])
    species = [CA40, NH3]
    trap = Trap(Omega=OMEGA_RF, a=-0.001, q=0.3, omega_z=TWO_PI * 0.2e6, gamma=1e5,
                T_bath=1e-3, dt=rf_period_dt(OMEGA_RF), seed=1)
    x0 = gaussian_positions(n, 100e-6, seed=1)
    v0 = thermal_velocities(species, sp, 10e-3, seed=[1, 1])
    return Workload("mix_n4096", species, sp, x0, v0, trap, 5000)


def crystal_n32768() -> Workload:
    n = 32768
    trap = Trap(Omega=OMEGA_RF, a=0.0, q=0.2, omega_z=TWO_PI * 0.05e6, gamma=2e5,
                T_bath=1e-3, dt=rf_period_dt(OMEGA_RF), seed=2)
    return Workload("crystal_n32768", [CA40], np.zeros(n, np.uint8),
                    spheroid_positions(n, 400e-6, 1.2e-3, seed=2), np.zeros((3, n)),
                    trap, 1000)


def _draw_trap_params(rng: np.random.Generator):
    q = rng.uniform(0.1, 0.4)
    a = rng.uniform(-0.005, 0.0)
    wz = TWO_PI * rng.uniform(0.1e6, 0.5e6)
    return q, a, wz


StabilityPredicate = Callable[[Sequence[Species], Trap], bool]


def batched_512(stable: Optional[StabilityPredicate] = None, count: int = 512,
                steps: int = 2000) -> List[Workload]:
    """512 independent Ca+ ensembles.  If ``stable`` is given, an ensemble whose drawn
    trap is rejected by it gets new (q, a, omega_z) from the same stream; its N and
    positions are kept."""
    rng = np.random.default_rng(3)
    out = []
    for e in range(count):
        n = int(round(math.exp(rng.uniform(math.log(16), math.log(2048)))))
        redraws = -1
        while True:
            redraws += 1
            q, a, wz = _draw_trap_params(rng)
            trap = Trap(Omega=OMEGA_RF, a=a, q=q, omega_z=wz, gamma=1e5, T_bath=1e-3,
                        dt=rf_period_dt(OMEGA_RF), seed=1000 + e)
            if stable is None or stable([CA40], trap):
                break
        x0 = gaussian_positions(n, 30e-6, seed=[3, e])
        out.append(Workload(f"batched_{e}", [CA40], np.zeros(n, np.uint8), x0,
                            np.zeros((3, n)), trap, steps, redraws))
    return out


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    n: int
    steps: int
    mixed: bool
    trap: Trap
    redraws: int = 0  # trap draws rejected as unstable before this one

    @property
    def species(self) -> List[Species]:
        return [CA40, NH3] if self.mixed else [CA40]


def serve_stream(stable: Optional[StabilityPredicate] = None, count: int = 20000,
                 rate_hz: float = 200.0) -> List[Request]:
    """The request stream: Poisson arrivals, log-uniform N and step budgets, species
    mix chosen with probability 1/2, trap parameters drawn as in ``batched_512``."""
    rng = np.random.default_rng(4)
    t = 0.0
    reqs = []
    for rid in range(count):
        t += rng.exponential(1.0 / rate_hz)
        n = int(round(math.exp(rng.uniform(math.log(8), math.log(65536)))))
        steps = int(round(math.exp(rng.uniform(math.log(1e3), math.log(1e5)))))
        mixed = bool(rng.uniform() < 0.5)
        species = [CA40, NH3] if mixed else [CA40]
        redraws = -1
        while True:
            redraws += 1
            q, a, wz = _draw_trap_params(rng)
            trap = Trap(Omega=OMEGA_RF, a=a, q=q, omega_z=wz, gamma=1e5, T_bath=1e-3,
                        dt=rf_period_dt(OMEGA_RF), seed=100000 + rid)
            if stable is None or stable(species, trap):
                break
        reqs.append(Request(rid, t, n, steps, mixed, trap, redraws))
    return reqs


def request_workload(req: Request) -> Workload:
    """Initial state of one serving request (drawn on demand from seed [4, rid]).
    The cloud's sigma grows as N^(1/3) above 2048 ions so that its central density
    never exceeds the densest batched ensemble."""
    n = req.n
    sigma = 30e-6 * max(1.0, (n / 2048.0) ** (1.0 / 3.0))
    if req.mixed:
        n_nh3 = int(math.floor(0.2 * n))
        sp = np.concatenate([np.zeros(n - n_nh3, np.uint8), np.ones(n_nh3, np.uint8)])
    else:
        sp = np.zeros(n, np.uint8)
    x0 = gaussian_positions(n, sigma, seed=[4, req.rid])
    return Workload(f"req_{req.rid}", req.species, sp, x0, np.zeros((3, n)), req.trap,
                    req.steps, req.redraws)


WORKLOADS = {
    "plain_n64": plain_n64,
    "mix_n4096": mix_n4096,
    "crystal_n32768": crystal_n32768,
}
