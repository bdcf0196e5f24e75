"""Seeded synthetic input streams for the PFB channeliser.

This module only draws random numbers and lays out sample buffers; it holds
none of the channeliser's arithmetic, so the CUDA path and the CPU oracle can
both be fed from it without sharing any of the method.

The paper measures on "randomly generated" 32-bit inputs of unstated size
(Sec. 5, experimental set-up); the recipes below stand in for that workload,
with the shapes of the five configurations the library is benchmarked on:

    c1  real fp32, N(0,1) noise + unit cosine at channel 3's centre,
        P=16, T=4, N=16*4*256, Hann prototype                       (seed 1)
    c2  complex64 CN(0,1) + 8 tones at distinct random channel centres,
        amplitudes U(0.1,1), phases U(0,2pi); N=2^24, P=1024, T=16,
        Hamming prototype                                           (seed 2)
    c3  64 streams x 2^20 complex64 CN(0,1) + 2 tones/stream,
        P=4096, T=16, Blackman prototype                            (seed 3)
    c4  256 uneven streams: P ~ U{256,512,1024,4096}, T ~ U{8,16},
        N = floor(2^U), U ~ U(14,22); CN(0,1) + 1-4 tones           (seed 4)
    c5  complex int8 (interleaved re,im), integers U[-127,127],
        scale 1, P=4096, T=16; requests of 2^20 samples in 2^16
        chunks, Poisson arrivals at 2000 req/s                      (seed 5)

A "tone at channel c's centre" is A*exp(i(2*pi*c*n/P + phi)): its period
divides P, so one length-P period is built in float64 and tiled.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# in_dtype codes (match the C ABI enum pfb_in_dtype)
IN_R32 = 0
IN_C64 = 1
IN_CI8 = 2

# window codes (match the C ABI enum pfb_window)
WIN_HANN = 0
WIN_HAMMING = 1
WIN_BLACKMAN = 2
WIN_USER = 3


@dataclass
class StreamSpec:
    """One synthetic input stream and the channeliser parameters it is run with."""

    P: int
    T: int
    window: int
    in_dtype: int
    n_samples: int
    seed: int
    tones: list = field(default_factory=list)  # (channel, amplitude, phase)
    in_scale: float = 1.0

    def generate(self) -> np.ndarray:
        """Host buffer of the stream: float32[N] (R32), complex64[N] (C64) or int8[2N] (CI8)."""
        rng = np.random.default_rng(self.seed)
        if self.in_dtype == IN_R32:
            x = rng.standard_normal(self.n_samples, dtype=np.float32)
            for (c, a, ph) in self.tones:
                period = a * np.cos(2.0 * np.pi * c * np.arange(self.P) / self.P + ph)
                x += _tile(period, self.n_samples).astype(np.float32)
            return x
        if self.in_dtype == IN_C64:
            return complex_gaussian(rng, self.n_samples, self.tones, self.P)
        if self.in_dtype == IN_CI8:
            return rng.integers(-127, 128, size=2 * self.n_samples, dtype=np.int16).astype(np.int8)
        raise ValueError(f"unknown in_dtype {self.in_dtype}")


def _tile(period: np.ndarray, n: int) -> np.ndarray:
    reps = -(-n // period.shape[0])
    return np.tile(period, reps)[:n]


def complex_gaussian(rng: np.random.Generator, n: int, tones=(), P: int = 1) -> np.ndarray:
    """CN(0,1) samples (re, im ~ N(0, 1/2)) plus tones at channel centres, as complex64."""
    xs = rng.standard_normal(2 * n, dtype=np.float32)
    xs *= np.float32(math.sqrt(0.5))
    x = xs.view(np.complex64)
    for (c, a, ph) in tones:
        period = a * np.exp(1j * (2.0 * np.pi * c * np.arange(P) / P + ph))
        x += _tile(period, n).astype(np.complex64)
    return x


def random_tones(rng: np.random.Generator, P: int, k: int):
    chans = rng.choice(P, size=k, replace=False)
    amps = rng.uniform(0.1, 1.0, size=k)
    phases = rng.uniform(0.0, 2.0 * np.pi, size=k)
    return [(int(c), float(a), float(p)) for c, a, p in zip(chans, amps, phases)]


# ----------------------------------------------------------------------------
# configuration recipes
# ----------------------------------------------------------------------------

def config_c1() -> StreamSpec:
    return StreamSpec(P=16, T=4, window=WIN_HANN, in_dtype=IN_R32, n_samples=16 * 4 * 256,
                      seed=1, tones=[(3, 1.0, 0.0)])


def config_c2(n_samples: int = 1 << 24) -> StreamSpec:
    rng = np.random.default_rng(2)
    return StreamSpec(P=1024, T=16, window=WIN_HAMMING, in_dtype=IN_C64, n_samples=n_samples,
                      seed=20002, tones=random_tones(rng, 1024, 8))


def config_c3(n_streams: int = 64, n_samples: int = 1 << 20) -> list[StreamSpec]:
    rng = np.random.default_rng(3)
    out = []
    for i in range(n_streams):
        out.append(StreamSpec(P=4096, T=16, window=WIN_BLACKMAN, in_dtype=IN_C64,
                              n_samples=n_samples, seed=30000 + i, tones=random_tones(rng, 4096, 2)))
    return out


def config_c4(n_streams: int = 256) -> list[StreamSpec]:
    rng = np.random.default_rng(4)
    out = []
    for i in range(n_streams):
        P = int(rng.choice([256, 512, 1024, 4096]))
        T = int(rng.choice([8, 16]))
        U = rng.uniform(14.0, 22.0)
        N = int(math.floor(2.0 ** U))
        win = int(rng.integers(0, 3))
        tones = random_tones(rng, P, int(rng.integers(1, 5)))
        out.append(StreamSpec(P=P, T=T, window=win, in_dtype=IN_C64, n_samples=N,
                              seed=40000 + i, tones=tones))
    return out


@dataclass
class ServingWorkload:
    """Open-loop serving workload: Poisson arrivals of channelisation requests."""

    P: int = 4096
    T: int = 16
    window: int = WIN_BLACKMAN
    request_samples: int = 1 << 20
    chunk_samples: int = 1 << 16
    rate_hz: float = 2000.0
    n_requests: int = 20000
    seed: int = 5

    def arrivals(self) -> np.ndarray:
        """Arrival times in seconds (cumulative exponential gaps)."""
        rng = np.random.default_rng(self.seed)
        return np.cumsum(rng.exponential(1.0 / self.rate_hz, size=self.n_requests))

    def request_stream(self, i: int) -> StreamSpec:
        return StreamSpec(P=self.P, T=self.T, window=self.window, in_dtype=IN_CI8,
                          n_samples=self.request_samples, seed=50000 + i)


def config_c5(**kw) -> ServingWorkload:
    return ServingWorkload(**kw)


def small_stream(P: int, T: int, n_samples: int, in_dtype: int = IN_C64, seed: int = 0,
                 window: int = WIN_HANN, ntones: int = 2) -> StreamSpec:
    """Small seeded stream for parity tests (several tiles and a ragged tail)."""
    rng = np.random.default_rng(seed + 7919)
    tones = random_tones(rng, P, min(ntones, P)) if in_dtype != IN_CI8 else []
    return StreamSpec(P=P, T=T, window=window, in_dtype=in_dtype, n_samples=n_samples,
                      seed=seed, tones=tones)
