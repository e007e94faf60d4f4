"""Seeded density fields, source lists and the named workloads.

Everything here is random-number drawing and array layout only.  Arrays use
CGS units: lengths in cm, hydrogen number density n_H in cm^-3, photon rates
in s^-1.  A density cube of N^3 cells is a float64 array of shape (N, N, N)
indexed [iz, iy, ix] (x fastest), with the box's low corner at the origin.

Workload recipes (the paper's static test setups, Sec. 3.1 and Sec. 5.2,
re-created synthetically; no dataset is read):

* ``stromgren32``: uniform 32^3 grid, box 8 pc, n_H = 100 cm^-3, one point
  source with Q = 1e49 s^-1 at the box centre (Sec. 3.1 Strömgren set-up).
* ``turbulent128``: 128^3 grid, box 10 pc, log-normal density drawn from a
  Gaussian random field with power spectrum P(k) ~ k^-4, sigma_ln = 1.5,
  mean n_H = 100 cm^-3; 10 point sources at uniform random positions with
  log10 Q uniform in [47, 50].
* ``sourcecount256``: 256^3 grid, box 30 pc (the source-count test of
  Sec. 5.2), same field recipe; S point sources sharing a total of 1e51 s^-1,
  or the diffuse case where every cell emits in proportion to n_H^2.
* ``turbulent32`` / ``turbulent64``: smaller fields of the same recipe, used
  as parity cases that the CPU oracle finishes in seconds.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PC_CM = 3.0856775814913673e18      # parsec in cm
ALPHA_B = 2.7e-13                  # case-B recombination coefficient, cm^3 s^-1 (Sec. 3.1)
HNU_EUV = 13.6 * 1.602176634e-12   # mean EUV photon energy, erg (13.6 eV; the paper gives no value)
SEED_BASE = 2105_09644


@dataclasses.dataclass
class Workload:
    """One synthetic problem: grid, density, sources and solver parameters."""
    name: str
    N: int                         # cells per axis
    box_cm: float                  # edge length of the cubic box, cm
    n_H: np.ndarray                # (N, N, N) float64, cm^-3, [iz, iy, ix]
    src_xyz: np.ndarray            # (S, 3) float64, cm
    src_Q: np.ndarray              # (S,) float64, photons s^-1
    ndot_cell: np.ndarray | None = None   # (N, N, N) float64 diffuse emission s^-1, or None
    nside: int = 2
    theta_lim: float = 0.5
    theta_if: float = math.inf
    theta_src: float = math.inf
    eta_r: int = 2
    alpha_B: float = ALPHA_B
    hnu: float = HNU_EUV
    seed: int = 0

    @property
    def dx(self) -> float:
        return self.box_cm / self.N

    @property
    def n_cells(self) -> int:
        return self.N ** 3

    @property
    def npix(self) -> int:
        return 12 * self.nside * self.nside


def uniform_density(N: int, n_H: float) -> np.ndarray:
    return np.full((N, N, N), float(n_H), dtype=np.float64)


def lognormal_density(N: int, seed: int, sigma_ln: float = 1.5,
                      mean_nH: float = 100.0, slope: float = -4.0) -> np.ndarray:
    """Log-normal field n = mean * exp(g - sigma^2/2).

    g is a zero-mean Gaussian random field with power spectrum |g_k|^2 ~ k^slope
    (zero mode removed), rescaled to standard deviation sigma_ln.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    white = rng.standard_normal((N, N, N))
    wk = np.fft.rfftn(white)
    kz = np.fft.fftfreq(N) * N
    ky = np.fft.fftfreq(N) * N
    kx = np.fft.rfftfreq(N) * N
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (slope / 4.0)           # |g_k| ~ k^(slope/2)
    g = np.fft.irfftn(wk * amp, s=(N, N, N), axes=(0, 1, 2))
    g -= g.mean()
    g *= sigma_ln / g.std()
    return mean_nH * np.exp(g - 0.5 * sigma_ln * sigma_ln)


def uniform_sources(S: int, box_cm: float, seed: int, log10_q_lo: float,
                    log10_q_hi: float) -> tuple[np.ndarray, np.ndarray]:
    """S sources at uniform random positions, log10 Q uniform in [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xyz = rng.uniform(0.0, box_cm, size=(S, 3))
    q = 10.0 ** rng.uniform(log10_q_lo, log10_q_hi, size=S)
    return xyz, q


def powerlaw_sources(S: int, box_cm: float, seed: int, q_lo: float,
                     q_hi: float) -> tuple[np.ndarray, np.ndarray]:
    """S sources at uniform positions, dN/dQ ~ Q^-2 on [q_lo, q_hi] (inverse CDF)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xyz = rng.uniform(0.0, box_cm, size=(S, 3))
    u = rng.uniform(0.0, 1.0, size=S)
    q = 1.0 / (1.0 / q_lo - u * (1.0 / q_lo - 1.0 / q_hi))
    return xyz, q


def _stromgren32(**kw) -> Workload:
    N, box = 32, 8.0 * PC_CM
    return Workload("stromgren32", N, box, uniform_density(N, 100.0),
                    np.array([[0.5 * box, 0.5 * box, 0.5 * box]]),
                    np.array([1e49]), seed=SEED_BASE + 0, **kw)


def _turbulent(N: int, name: str, seed: int, n_src: int = 10, **kw) -> Workload:
    box = 10.0 * PC_CM
    rho = lognormal_density(N, seed)
    xyz, q = uniform_sources(n_src, box, seed + 7, 47.0, 50.0)
    return Workload(name, N, box, rho, xyz, q, seed=seed, **kw)


def _sourcecount(N: int = 256, n_src: int = 100, diffuse: bool = False,
                 seed: int = SEED_BASE + 3, **kw) -> Workload:
    box = 30.0 * PC_CM
    rho = lognormal_density(N, seed)
    total_q = 1e51
    if diffuse:
        w = rho * rho
        ndot = total_q * w / w.sum()
        return Workload(f"diffuse{N}", N, box, rho, np.zeros((0, 3)), np.zeros(0),
                        ndot_cell=ndot, seed=seed, **kw)
    rng = np.random.Generator(np.random.PCG64(seed + 11 + n_src))
    xyz = rng.uniform(0.0, box, size=(n_src, 3))
    q = np.full(n_src, total_q / n_src)
    return Workload(f"sourcecount{N}_s{n_src}", N, box, rho, xyz, q, seed=seed, **kw)


WORKLOADS = {
    "stromgren32": lambda **kw: _stromgren32(**kw),
    "turbulent32": lambda **kw: _turbulent(32, "turbulent32", SEED_BASE + 101, **kw),
    "turbulent64": lambda **kw: _turbulent(64, "turbulent64", SEED_BASE + 102, **kw),
    "turbulent128": lambda **kw: _turbulent(128, "turbulent128", SEED_BASE + 1, **kw),
    "sourcecount256_s1": lambda **kw: _sourcecount(256, 1, **kw),
    "sourcecount256_s100": lambda **kw: _sourcecount(256, 100, **kw),
    "sourcecount256_s10000": lambda **kw: _sourcecount(256, 10000, **kw),
    "diffuse256": lambda **kw: _sourcecount(256, diffuse=True, **kw),
}


def workload(name: str, **overrides) -> Workload:
    """Build a named workload; keyword overrides replace solver parameters."""
    if name not in WORKLOADS:
        raise KeyError(f"unknown workload {name!r}; known: {sorted(WORKLOADS)}")
    return WORKLOADS[name](**overrides)
