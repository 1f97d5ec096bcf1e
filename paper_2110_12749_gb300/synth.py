"""Seeded synthetic 8-bit filterbanks with injected signals.

This module is the one input generator shared by the CUDA path's tests and
benchmark and by the CPU oracle's tests.  It holds none of the method's
arithmetic: the per-channel delays of an injected dispersed pulse are passed
in by the caller (computed by whichever side is under test), so that nothing
here can make the two sides agree by construction.

Signal model (the data of Sec. 3.1 are 8-bit FAST/CRAFTS filterbanks with
simulated pulses injected into them; those files are not available, so the
noise, RFI and bursts below stand in for them):
  X[c][t] = clip(rint(mu + sigma * N(0,1) + signal[c][t]), 0, 255)
  - narrowband RFI: chosen channels get amp * sin(2 pi t / P + phi);
  - broadband "DM 0" bursts: every channel gets +amp on [t0, t0 + w);
  - dispersed boxcar pulses: channel c gets +A on [t0 + d_c, t0 + d_c + w),
    with d_c supplied by the caller and A = snr * sigma / sqrt(nchan * w).
Every channel row has its own PCG64 stream seeded by (seed, beam, channel),
so the output does not depend on the number of threads.
"""
from __future__ import annotations

import dataclasses
import math
import os
from concurrent.futures import ThreadPoolExecutor
from typing import List, Optional, Sequence

import numpy as np

BASE_SEED = 20211025


@dataclasses.dataclass
class Pulse:
    dm: float          # DM of the pulse (informational; delays come from the caller)
    t0: int            # arrival sample at the top channel
    width: int         # boxcar width (samples)
    snr: float         # nominal matched-filter S/N at the true DM and width
    amp: float = 0.0   # per-channel amplitude (filled by pulse_amplitude)
    delays: Optional[np.ndarray] = None  # int [nchan] per-channel delay (samples)


@dataclasses.dataclass
class Rfi:
    chan: int
    period: float
    phase: float
    amp: float


@dataclasses.dataclass
class Burst:
    t0: int
    width: int
    amp: float


@dataclasses.dataclass
class Workload:
    """One synthetic workload: band, sampling, DM grid and injection recipe."""
    name: str
    nchan: int
    f_lo: float
    f_hi: float
    t_samp: float
    n_in: int
    dm_lo: float
    dm_step: float
    ndm: int
    mu: float
    sigma: float
    n_rfi: int = 0
    n_bursts: int = 0
    n_pulses: int = 0
    pulse_dm: tuple = (10.0, 1000.0)
    pulse_w: tuple = (1, 100)
    pulse_snr: tuple = (6.0, 30.0)
    fixed_pulses: tuple = ()   # (dm, width, snr) triples placed at seeded times

    @property
    def dms(self) -> np.ndarray:
        return self.dm_lo + self.dm_step * np.arange(self.ndm, dtype=np.float64)

    def sky_seconds(self, n: Optional[int] = None) -> float:
        return (self.n_in if n is None else n) * self.t_samp


# The paper's configurations of the hot path.  "tiny" is the small case the
# oracle finishes in seconds; "crafts" is one CRAFTS-like beam (4096 channels,
# 1000-1500 MHz, 49.152 us, 2^20 samples, 2000 DM trials to DM 1000); "wideband"
# is the 500-3300 MHz low-frequency variant with long dispersion sweeps.
WORKLOADS = {
    "tiny": Workload("tiny", 256, 1200.0, 1500.0, 100e-6, 32768, 0.0, 1.0, 200,
                     128.0, 16.0, fixed_pulses=((50.0, 5, 15.0),)),
    "crafts": Workload("crafts", 4096, 1000.0, 1500.0, 49.152e-6, 1 << 20, 0.0, 0.5,
                       2000, 128.0, 20.0, n_rfi=30, n_bursts=5, n_pulses=40,
                       pulse_dm=(10.0, 1000.0), pulse_w=(1, 100), pulse_snr=(6.0, 30.0)),
    "wideband": Workload("wideband", 2048, 500.0, 3300.0, 98.304e-6, 1 << 20, 0.0, 1.0,
                         3000, 128.0, 20.0, n_rfi=30, n_bursts=5, n_pulses=60,
                         pulse_dm=(0.0, 3000.0), pulse_w=(1, 150), pulse_snr=(6.0, 30.0)),
}


def beam_seed(beam: int, seed: int = BASE_SEED) -> int:
    return seed + 1000 * beam


def pulse_amplitude(snr: float, sigma: float, nchan: int, width: int) -> float:
    """Per-channel amplitude of a boxcar that reaches `snr` when all nchan
    channels and `width` samples are summed over Gaussian noise of rms sigma."""
    return snr * sigma / math.sqrt(nchan * width)


def _log_uniform_int(rng, lo, hi):
    return int(np.clip(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))), lo, hi))


def draw_recipe(wl: Workload, n_out: int, beam: int = 0, seed: int = BASE_SEED):
    """Seeded RFI channels, bursts and pulse (dm, t0, width, snr) draws for one
    beam.  Pulse delays and amplitudes are left for the caller to fill."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([beam_seed(beam, seed), 7])))
    rfi = []
    if wl.n_rfi:
        chans = rng.choice(wl.nchan, size=wl.n_rfi, replace=False)
        for c in chans:
            period = math.exp(rng.uniform(math.log(16.0), math.log(4096.0)))
            rfi.append(Rfi(int(c), period, float(rng.uniform(0, 2 * math.pi)), 10.0 * wl.sigma))
    bursts = []
    for _ in range(wl.n_bursts):
        w = _log_uniform_int(rng, 1, 100)
        bursts.append(Burst(int(rng.integers(0, wl.n_in - w)), w, 3.0 * wl.sigma))
    pulses: List[Pulse] = []
    specs = [tuple(p) for p in wl.fixed_pulses]
    for _ in range(wl.n_pulses):
        dm = float(rng.uniform(*wl.pulse_dm))
        w = _log_uniform_int(rng, *wl.pulse_w)
        specs.append((dm, w, float(rng.uniform(*wl.pulse_snr))))
    taken = []
    for dm, w, snr in specs:
        for _ in range(1000):
            t0 = int(rng.integers(0, max(n_out - w, 1)))
            if all(abs(t0 - t1) > (w + w1 + 64) for t1, w1 in taken):
                break
        taken.append((t0, w))
        pulses.append(Pulse(float(dm), t0, int(w), float(snr)))
    return rfi, bursts, pulses


def _row(c, nchan, n_in, stride, mu, sigma, rfi_by_chan, bursts, pulses, seed, beam, out):
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, beam, c])))
    v = rng.standard_normal(n_in, dtype=np.float32)
    v *= np.float32(sigma)
    v += np.float32(mu)
    for r in rfi_by_chan.get(c, ()):
        t = np.arange(n_in, dtype=np.float64)
        v += (r.amp * np.sin(2.0 * math.pi * t / r.period + r.phase)).astype(np.float32)
    for b in bursts:
        v[b.t0:b.t0 + b.width] += np.float32(b.amp)
    for p in pulses:
        s = p.t0 + int(p.delays[c])
        e = min(s + p.width, n_in)
        if s < n_in:
            v[s:e] += np.float32(p.amp)
    np.rint(v, out=v)
    np.clip(v, 0.0, 255.0, out=v)
    out[c, :n_in] = v.astype(np.uint8)
    if stride > n_in:
        out[c, n_in:] = 0


def filterbank(nchan: int, n_in: int, seed: int, mu: float, sigma: float,
               rfi: Sequence[Rfi] = (), bursts: Sequence[Burst] = (),
               pulses: Sequence[Pulse] = (), beam: int = 0,
               stride: Optional[int] = None, threads: Optional[int] = None,
               out: Optional[np.ndarray] = None) -> np.ndarray:
    """uint8 [nchan][stride] channel-major filterbank (see module docstring).
    stride defaults to n_in rounded up to 16 bytes; padding bytes are 0."""
    if stride is None:
        stride = (n_in + 15) // 16 * 16
    for p in pulses:
        if p.delays is None or len(p.delays) != nchan:
            raise ValueError("every pulse needs per-channel delays")
    if out is None:
        out = np.empty((nchan, stride), dtype=np.uint8)
    rfi_by_chan = {}
    for r in rfi:
        rfi_by_chan.setdefault(r.chan, []).append(r)
    if threads is None:
        threads = min(32, len(os.sched_getaffinity(0)))
    args = (nchan, n_in, stride, mu, sigma, rfi_by_chan, list(bursts), list(pulses), seed, beam, out)
    if threads <= 1 or nchan < 8:
        for c in range(nchan):
            _row(c, *args)
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda c: _row(c, *args), range(nchan)))
    return out


def workload_filterbank(wl: Workload, delays_fn, n_out: int, beam: int = 0,
                        seed: int = BASE_SEED, n_in: Optional[int] = None,
                        threads: Optional[int] = None, stride: Optional[int] = None):
    """Filterbank of a workload with its seeded RFI, bursts and pulses.
    delays_fn(dm) must return the int per-channel delays of a pulse at DM dm
    (supplied by the caller).  Returns (x, rfi, bursts, pulses)."""
    n_in = wl.n_in if n_in is None else n_in
    rfi, bursts, pulses = draw_recipe(wl, n_out, beam, seed)
    for p in pulses:
        p.delays = np.asarray(delays_fn(p.dm), dtype=np.int64).reshape(-1)
        p.amp = pulse_amplitude(p.snr, wl.sigma, wl.nchan, p.width)
    x = filterbank(wl.nchan, n_in, beam_seed(beam, seed), wl.mu, wl.sigma, rfi, bursts,
                   pulses, beam=beam, threads=threads, stride=stride)
    return x, rfi, bursts, pulses
