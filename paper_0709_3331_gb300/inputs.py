"""Seeded synthetic plasma clouds (shared by the CUDA path's tests, the oracle
tests and the benchmark).  This module draws random numbers only: it holds none
of the TREE method's arithmetic.

Recipe (reduced units, k_B = 1, Coulomb constant 1): N/2 ions (species 0,
indices [0, N/2)) and N/2 electrons (species 1, indices [N/2, N)).  With
``numpy.random.default_rng(seed)`` (PCG64) the generator draws, in this order,
ion positions, electron positions (each i.i.d. isotropic Gaussian N(0, sigma^2 I)),
ion velocities N(0, T_i/m_i) and electron velocities N(0, T_e/m_e) per
component; each species' mean velocity is then subtracted (zero net momentum).
Sec. 5 of the paper starts its plasmas from given electron and ion temperatures
in a roughly spherical cloud; the Gaussian cloud stands in for that shape.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

ION, ELECTRON = 0, 1


@dataclass(frozen=True)
class Cloud:
    pos: np.ndarray      # (N, 3) float64
    vel: np.ndarray      # (N, 3) float64
    species: np.ndarray  # (N,) int8: 0 = ion, 1 = electron
    q: np.ndarray        # (2,) charge per species
    m: np.ndarray        # (2,) mass per species

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def gaussian_cloud(n: int, sigma: float, seed: int, t_e: float = 1.0, t_i: float = 0.01,
                   m_i: float = 1000.0, m_e: float = 1.0, q_i: float = 1.0,
                   q_e: float = -1.0) -> Cloud:
    if n < 0 or n % 2:
        raise ValueError("n must be a non-negative even number")
    h = n // 2
    rng = np.random.default_rng(seed)
    pos = np.empty((n, 3))
    pos[:h] = rng.normal(0.0, sigma, size=(h, 3))
    pos[h:] = rng.normal(0.0, sigma, size=(h, 3))
    vel = np.empty((n, 3))
    vel[:h] = rng.normal(0.0, math.sqrt(t_i / m_i), size=(h, 3))
    vel[h:] = rng.normal(0.0, math.sqrt(t_e / m_e), size=(h, 3))
    if h:
        vel[:h] -= vel[:h].mean(axis=0)
        vel[h:] -= vel[h:].mean(axis=0)
    species = np.empty(n, dtype=np.int8)
    species[:h] = ION
    species[h:] = ELECTRON
    return Cloud(pos, vel, species, np.array([q_i, q_e]), np.array([m_i, m_e]))


# Named workloads (sizes, spreads and seeds of the five standard configurations).
WORKLOADS = {
    "plain_n2048": dict(n=2048, sigma=1.0, seed=1),
    "plain_n131072": dict(n=131072, sigma=4.0, seed=2),
    "precision_n524288": dict(n=524288, sigma=8.0, seed=3),
    "adjoint_n262144": dict(n=262144, sigma=6.0, seed=5),
}


def workload(name: str) -> Cloud:
    return gaussian_cloud(**WORKLOADS[name])


def batched_sizes(n_clouds: int = 64, seed: int = 4):
    """Per-cloud N, log-uniform in [4096, 65536], even; sigma_c = (N_c/2048)^(1/3)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(4096), math.log(65536), size=n_clouds)
    ns = [int(2 * round(math.exp(v) / 2)) for v in u]
    return ns, [(nc / 2048.0) ** (1.0 / 3.0) for nc in ns]


# Physical constants (CODATA 2018) for the Sec. 5 set-up.
_E = 1.602176634e-19
_EPS0 = 8.8541878128e-12
_KB = 1.380649e-23
_ME = 9.1093837015e-31
_AMU = 1.66053906660e-27


def sec5_units(density_per_cm3, lambda_ei_angstrom, t_e_kelvin, t_i_kelvin, ion_mass_amu,
               dt_fs):
    """Reduced units for a physical set-up: length = Wigner-Seitz radius a of the
    density, energy = e^2 / (4 pi eps0 a), mass = electron mass, time =
    sqrt(m_e a^3 4 pi eps0 / e^2).  Returns lambda, temperatures (k_B T in energy
    units), ion mass and time step in those units, and the units themselves."""
    n = density_per_cm3 * 1e6
    a = (3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    energy = _E * _E / (4.0 * math.pi * _EPS0 * a)
    tau = math.sqrt(_ME * a ** 3 * 4.0 * math.pi * _EPS0 / (_E * _E))
    return {"length_m": a, "energy_j": energy, "time_s": tau,
            "lambda": lambda_ei_angstrom * 1e-10 / a,
            "t_e": _KB * t_e_kelvin / energy, "t_i": _KB * t_i_kelvin / energy,
            "m_i": ion_mass_amu * _AMU / _ME, "dt": dt_fs * 1e-15 / tau}


def uniform_sphere(n, radius, seed, t_e, t_i, m_i, m_e=1.0):
    """N/2 ions then N/2 electrons uniformly in a sphere (the Sec. 5 cloud shape),
    Maxwellian velocities with each species' mean removed."""
    if n < 0 or n % 2:
        raise ValueError("n must be a non-negative even number")
    h = n // 2
    rng = np.random.default_rng(seed)
    pos = np.empty((n, 3))
    for lo, hi in ((0, h), (h, n)):
        d = rng.normal(size=(hi - lo, 3))
        d /= np.linalg.norm(d, axis=1)[:, None]
        pos[lo:hi] = d * (radius * rng.uniform(size=(hi - lo, 1)) ** (1.0 / 3.0))
    vel = np.empty((n, 3))
    vel[:h] = rng.normal(0.0, math.sqrt(t_i / m_i), size=(h, 3))
    vel[h:] = rng.normal(0.0, math.sqrt(t_e / m_e), size=(h, 3))
    if h:
        vel[:h] -= vel[:h].mean(axis=0)
        vel[h:] -= vel[h:].mean(axis=0)
    species = np.empty(n, dtype=np.int8)
    species[:h] = ION
    species[h:] = ELECTRON
    return Cloud(pos, vel, species, np.array([1.0, -1.0]), np.array([m_i, m_e]))
