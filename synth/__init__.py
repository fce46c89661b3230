"""Seeded synthetic inputs for the FDAS correlation path.

This module is the one piece shared by the tests, the benchmark and the
oracle.  It holds none of the method's arithmetic (no spectrum, template,
correlation, power or threshold code): it draws white Gaussian noise and adds
constant-fdot sinusoids, i.e. the signal model that the search is built to
find (constant line-of-sight acceleration -> constant frequency derivative,
Section 2, Eqs. 21-22).

Signal model of one injection, with u = t/T in [0, 1) the fraction of the
observation and r0 the *mid-observation* frequency in Fourier bins:

    x(u) += a * cos(2 pi (r_s u + z0 u^2 / 2)),   r_s = r0 - z0/2,

so the instantaneous frequency r_s + z0 u sweeps z0 bins over the
observation (Eq. 22 defines z as the number of bins drifted).  The paper does
not define "spectral S/N"; the amplitude used here, a = 2 SNR / sqrt(n),
gives an expected coherent normalised power of about SNR^2 at (r0, z0).

Noise comes from numpy's PCG64 generator, whose output is identical on x86
and Arm, so every machine regenerates the same float32 series from a seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload",
    "WORKLOADS",
    "injection_amplitude",
    "make_series",
    "workload",
    "random_spectrum",
]


def injection_amplitude(snr: float, n: int) -> float:
    """Sinusoid amplitude whose coherent normalised power is about snr**2."""
    return 2.0 * float(snr) / math.sqrt(float(n))


def make_series(n: int, injections=(), seed: int = 0, noise: bool = True) -> np.ndarray:
    """float32[n]: sigma=1 Gaussian noise (seeded) plus constant-fdot sinusoids.

    injections: iterable of (r0, z0, snr) with r0 the mid-observation bin.
    """
    n = int(n)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n) if noise else np.zeros(n)
    if len(tuple(injections)):
        u = np.arange(n, dtype=np.float64) / n
        for r0, z0, snr in injections:
            rs = float(r0) - 0.5 * float(z0)
            cyc = rs * u + 0.5 * float(z0) * u * u
            cyc -= np.floor(cyc)  # reduce the phase before the cosine
            x += injection_amplitude(snr, n) * np.cos(2.0 * np.pi * cyc)
    return x.astype(np.float32)


def random_spectrum(nb: int, seed: int) -> np.ndarray:
    """complex64[nb] with independent unit-variance complex Gaussian entries.

    Shaped like a normalised noise spectrum (E|A|^2 = 1); used where a test
    feeds the correlator directly.
    """
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(nb)
    im = rng.standard_normal(nb)
    return ((re + 1j * im) / math.sqrt(2.0)).astype(np.complex64)


@dataclass(frozen=True)
class Workload:
    """One synthetic search: a series recipe plus the search parameters."""

    name: str
    n: int                 # time samples (power of two)
    seed: int
    injections: tuple      # ((r0, z0, snr), ...)
    zmin: int
    zmax: int
    zstep: int
    M: int                 # padded template width in taps
    L: int                 # overlap-save segment length
    median_block: int = 1024
    threshold: float = 20.0
    interbin: int = 1
    extra: dict = field(default_factory=dict)

    @property
    def nb(self) -> int:
        return self.n // 2

    @property
    def K(self) -> int:
        return (self.zmax - self.zmin) // self.zstep + 1

    def series(self) -> np.ndarray:
        return make_series(self.n, self.injections, self.seed)

    def with_(self, **kw) -> "Workload":
        d = dict(self.__dict__)
        d.update(kw)
        return Workload(**d)


def _production_injections(seed: int, count: int = 8, rmax: float = 4.0e6):
    rng = np.random.default_rng(seed + 1000)
    r = rng.uniform(1.0e4, rmax, count)
    z = rng.uniform(-200.0, 200.0, count)
    s = rng.uniform(6.0, 20.0, count)
    return tuple((float(a), float(b), float(c)) for a, b, c in zip(r, z, s))


WORKLOADS = {
    # 2^17 samples, one injection at r0=20000.3, z0=+10, S/N 15; z = -20..20
    # step 2 (21 templates), taps padded to 64, segments of 2048 points.
    "small": Workload("small", 1 << 17, 1, ((20000.3, 10.0, 15.0),),
                      -20, 20, 2, 64, 2048),
    # 2^23 samples (64 us sampling, ~537 s), 8 injections with r in
    # [1e4, 4e6], z in [-200, 200], S/N 6-20; z = -200..200 step 2
    # (201 templates), taps padded to 256; segment length swept 1024-4096.
    "production": Workload("production", 1 << 23, 2, _production_injections(2),
                           -200, 200, 2, 256, 1024),
    # The production search on a 2^20-sample series (201 x 2^20 plane, 0.84 GB):
    # same kernels and launch shapes, small enough for hardware-counter captures.
    "medium": Workload("medium", 1 << 20, 3, _production_injections(3, rmax=5.0e5),
                       -200, 200, 2, 256, 1024),
    # A few-second oracle case that still spans several segments and a
    # ragged tail: 2^14 samples, 8192 bins, 1024-point segments of 960
    # useful bins (8.53 segments).
    "tiny": Workload("tiny", 1 << 14, 7, ((1500.0, 6.0, 25.0), (4100.5, -12.0, 30.0)),
                     -20, 20, 2, 64, 1024),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]
