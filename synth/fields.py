"""Seeded synthetic stand-ins for the paper's SDRBench fields (Table II).

The SDRBench datasets (HACC, CESM, Hurricane, NYX) are not available, so
every workload is drawn here from numpy's PCG64 generator with a fixed seed,
with the shapes and value structure of the paper's data:

* 2D climate-like fields (CESM, 1800x3600): a sum of random Fourier modes
  with amplitude ~ |k|^-2 plus Gaussian noise;
* 3D fields (NYX 512^3, Hurricane 100x500x500): Gaussian random fields with
  a power-law spectrum, exponentiated for the log-normal, density-like NYX;
* 1D particle coordinates (HACC, 280,953,867 values): a wrapped random walk.

Everything is float32, C-order (dims[0] slowest).
"""
from __future__ import annotations

import math
import os

import numpy as np

try:  # scipy's FFT is multithreaded and takes float32 directly
    import scipy.fft as _fft
    _FFT_KW = {"workers": os.cpu_count() or 1}
except Exception:  # pragma: no cover - numpy fallback
    _fft = np.fft
    _FFT_KW = {}


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def fourier2d(ny: int, nx: int, seed: int, n_modes: int = 32, kmax: int = 32,
              amp_slope: float = -2.0, noise_rel: float = 1e-3,
              value_range: float | None = None, offset: float = 0.0) -> np.ndarray:
    """Sum of ``n_modes`` Fourier modes with integer wave vectors, |k| in
    [1, kmax], amplitude |k|^amp_slope and uniform phases, plus Gaussian noise
    of standard deviation noise_rel * range.  If value_range is given, the
    smooth part is rescaled to that range (and shifted by offset)."""
    rng = _rng(seed)
    ks = []
    while len(ks) < n_modes:
        kx, ky = rng.integers(-kmax, kmax + 1, size=2)
        r = math.hypot(kx, ky)
        if 1.0 <= r <= kmax:
            ks.append((int(kx), int(ky), r))
    phase = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    xs = np.arange(nx, dtype=np.float64) / nx
    ys = np.arange(ny, dtype=np.float64) / ny
    # sin(a + b) = sin a cos b + cos a sin b, summed over modes as two
    # (ny x M) @ (M x nx) products.
    A = np.array([r ** amp_slope for (_, _, r) in ks])
    alpha = 2.0 * np.pi * np.outer([k[0] for k in ks], xs) + phase[:, None]  # M x nx
    beta = 2.0 * np.pi * np.outer(ys, [k[1] for k in ks])                    # ny x M
    f = (np.cos(beta) * A) @ np.sin(alpha) + (np.sin(beta) * A) @ np.cos(alpha)
    lo, hi = float(f.min()), float(f.max())
    if value_range is not None and hi > lo:
        f = (f - lo) * (value_range / (hi - lo)) + offset
        lo, hi = offset, offset + value_range
    if noise_rel > 0:
        f = f + rng.normal(0.0, noise_rel * (hi - lo), size=f.shape)
    return f.astype(np.float32)


def grf3d(shape, seed: int, slope: float = -3.0) -> np.ndarray:
    """Gaussian random field with power spectrum ~ |k|^slope (unit variance,
    zero mean), synthesised by filtering white noise in Fourier space.
    Works for any ndim; returns float32."""
    rng = _rng(seed)
    shape = tuple(int(s) for s in shape)
    w = rng.standard_normal(size=shape, dtype=np.float32)
    W = _fft.rfftn(w, **_FFT_KW)
    del w
    # |k|^2 on the rfft grid, built axis by axis to keep memory low.
    k2 = None
    for ax, n in enumerate(shape):
        if ax == len(shape) - 1:
            k = np.fft.rfftfreq(n).astype(np.float32) * n
        else:
            k = np.fft.fftfreq(n).astype(np.float32) * n
        sh = [1] * len(shape)
        sh[ax] = k.size
        kk = (k * k).reshape(sh)
        k2 = kk if k2 is None else k2 + kk
    with np.errstate(divide="ignore"):
        filt = np.where(k2 > 0, k2 ** np.float32(slope / 4.0), np.float32(0.0))
    W *= filt.astype(np.complex64) if W.dtype == np.complex64 else filt
    del filt, k2
    g = _fft.irfftn(W, s=shape, **_FFT_KW).astype(np.float32, copy=False)
    del W
    g -= np.float32(g.mean(dtype=np.float64))
    sd = float(g.std(dtype=np.float64))
    if sd > 0:
        g *= np.float32(1.0 / sd)
    return g


def lognormal3d(n: int = 512, seed: int = 2, slope: float = -3.0) -> np.ndarray:
    """NYX-like density: exp of a unit-variance GRF with a k^-3 spectrum."""
    g = grf3d((n, n, n), seed, slope)
    np.exp(g, out=g)
    return g


def random_walk1d(n: int, seed: int, sigma: float = 1e-2, period: float = 256.0) -> np.ndarray:
    """HACC-like particle coordinates: cumulative sum of N(0, sigma^2) steps
    from a uniform start, wrapped into [0, period)."""
    rng = _rng(seed)
    out = np.empty(n, np.float32)
    start = rng.uniform(0.0, period)
    chunk = 1 << 24
    pos = start
    for i in range(0, n, chunk):
        m = min(chunk, n - i)
        steps = rng.normal(0.0, sigma, size=m)
        c = np.cumsum(steps) + pos
        pos = float(c[-1])
        out[i:i + m] = np.mod(c, period)
    return out


def tuner_field(seed: int):
    """One field of the tuner's training/evaluation distribution: rank
    uniform in {1,2,3}; 2D/3D side log-uniform in [64, 256]; 1D length
    log-uniform in [64, 2^24]; spectral slope uniform in [-4, -1]; noise
    uniform in [0, 1e-2] x range; range log-uniform in [1e-3, 1e3]; relative
    eb log-uniform in [1e-5, 1e-2].  Returns (x, rel_eb)."""
    rng = _rng(seed)
    rank = int(rng.integers(1, 4))
    if rank == 1:
        n = int(round(math.exp(rng.uniform(math.log(64), math.log(1 << 24)))))
        shape = (n,)
    else:
        shape = tuple(int(round(math.exp(rng.uniform(math.log(64), math.log(256)))))
                      for _ in range(rank))
    slope = float(rng.uniform(-4.0, -1.0))
    noise = float(rng.uniform(0.0, 1e-2))
    vrange = float(math.exp(rng.uniform(math.log(1e-3), math.log(1e3))))
    offset = float(rng.normal(0.0, vrange))
    eb = float(math.exp(rng.uniform(math.log(1e-5), math.log(1e-2))))
    # Power spectrum ~ k^(2*slope) gives amplitudes ~ k^slope.
    g = grf3d(shape, seed + 7919, 2.0 * slope).astype(np.float64)
    lo, hi = g.min(), g.max()
    if hi > lo:
        g = (g - lo) / (hi - lo)
    g = g * vrange + offset
    if noise > 0:
        g = g + rng.normal(0.0, noise * vrange, size=g.shape)
    return g.astype(np.float32), eb


# ---- named workloads --------------------------------------------------------

def cfg1_field() -> np.ndarray:
    """512x512 sum of 32 Fourier modes (|k|^-2), noise 1e-3 x range, seed 1."""
    return fourier2d(512, 512, seed=1, n_modes=32, kmax=32, amp_slope=-2.0, noise_rel=1e-3)


def cfg2_field(n: int = 512) -> np.ndarray:
    """n^3 log-normal density (exp of a k^-3 GRF), seed 2."""
    return lognormal3d(n, seed=2, slope=-3.0)


def _field_range(seed: int) -> float:
    rng = _rng(seed + 31337)
    return float(math.exp(rng.uniform(math.log(1e-3), math.log(1e3))))


def cfg3_fields():
    """The mixed batch: 79 CESM-shaped 2D fields (1800x3600, per-field range
    log-uniform in [1e-3, 1e3]), 13 Hurricane-shaped 3D fields (100x500x500)
    and 4 HACC-like 1D fields of 10M values.  Yields (name, shape, maker)
    with a zero-argument maker, so callers can generate lazily."""
    out = []
    for i in range(79):
        s = 100 + i
        out.append((f"cesm2d_{i}", (1800, 3600),
                    lambda s=s: fourier2d(1800, 3600, seed=s, value_range=_field_range(s))))
    for i in range(13):
        s = 200 + i
        out.append((f"hurricane3d_{i}", (100, 500, 500),
                    lambda s=s: (grf3d((100, 500, 500), s, -3.0) * np.float32(_field_range(s)))))
    for i in range(4):
        s = 300 + i
        out.append((f"hacc1d_{i}", (10_000_000,), lambda s=s: random_walk1d(10_000_000, s)))
    return out


def cfg5_fields():
    """The end-to-end stream: one 1D field of 280,953,867 random-walk values
    (HACC's length), 13 fields of 100x500x500 and 20 of 1800x3600."""
    out = [("hacc1d_full", (280_953_867,), lambda: random_walk1d(280_953_867, 400))]
    for i in range(13):
        s = 500 + i
        out.append((f"hurricane3d_{i}", (100, 500, 500),
                    lambda s=s: (grf3d((100, 500, 500), s, -3.0) * np.float32(_field_range(s)))))
    for i in range(20):
        s = 600 + i
        out.append((f"cesm2d_{i}", (1800, 3600),
                    lambda s=s: fourier2d(1800, 3600, seed=s, value_range=_field_range(s))))
    return out


def adversarial_values(n: int, seed: int, inv2eb: float = 0.5) -> np.ndarray:
    """Values that stress the edges of the method: exact rounding ties
    (x * inv2eb = k + 0.5), huge magnitudes that saturate int32, +-0,
    subnormals, NaN and +-Inf, mixed with ordinary values."""
    rng = _rng(seed)
    x = rng.normal(0.0, 100.0, size=n).astype(np.float32)
    kinds = rng.integers(0, 8, size=n)
    ties = ((rng.integers(-1000, 1000, size=n) + 0.5) / inv2eb).astype(np.float32)
    huge = (rng.choice([-1.0, 1.0], size=n) * 10.0 ** rng.uniform(9, 38, size=n)).astype(np.float32)
    x = np.where(kinds == 1, ties, x)
    x = np.where(kinds == 2, huge, x)
    x = np.where(kinds == 3, np.float32(0.0), x)
    x = np.where(kinds == 4, np.float32(-0.0), x)
    x = np.where(kinds == 5, np.float32(1e-40), x)
    special = np.array([np.nan, np.inf, -np.inf], np.float32)
    x = np.where(kinds == 6, special[rng.integers(0, 3, size=n)], x)
    return x.astype(np.float32)
