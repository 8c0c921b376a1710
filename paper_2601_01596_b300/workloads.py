"""Seeded synthetic inputs shaped like the paper's workloads (Sec. V, Table 1).

Shared by the CUDA path's tests/bench and by the oracle's tests.  This module
holds no arithmetic of the correction method itself: it only builds fields,
emulates a base compressor's error and picks the two bounds.

The paper's data (Nyx, HEDM, EEG; Table 1) and its base compressors (SZ3, ZFP,
SPERR) are not available, so every input is synthetic:

* ``grf``      -- Gaussian random field whose shell-summed power spectrum
                  P(k) (Sec. III) falls as k^-alpha: per-mode variance
                  |k|^-(alpha + d - 1), k = 0 mode removed, unit variance.
* ``quantization_error`` -- a uniform quantiser with bin width 2*eps stands in
                  for the base compressor; e0 = x_hat - x (Sec. IV-A sign).
* bounds      -- eps_s from the value range, eps_f from max_k |X_k| (the RFE
                  normaliser of Sec. V-A) unless stated otherwise.

Randomness is numpy PCG64 (``default_rng(seed)``); fields are generated in
float64 and cast to float32, and both sides start from the same float32 bits.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

_W = -1  # scipy.fft workers: all host cores


def _kmag(shape, real_last=True):
    """|k| in integer index units on the (r)fft grid."""
    axes = []
    for i, n in enumerate(shape):
        if real_last and i == len(shape) - 1:
            axes.append(np.arange(n // 2 + 1, dtype=np.float64))
        else:
            axes.append(np.fft.fftfreq(n) * n)
    grids = np.meshgrid(*axes, indexing="ij", sparse=True)
    k2 = sum(g * g for g in grids)
    return np.sqrt(k2)


def grf(shape, alpha: float, seed: int) -> np.ndarray:
    """Unit-variance, zero-mean Gaussian random field with P(k) ~ k^-alpha."""
    rng = np.random.default_rng(seed)
    d = len(shape)
    w = rng.standard_normal(shape)
    W = sfft.rfftn(w, workers=_W)
    k = _kmag(shape)
    with np.errstate(divide="ignore"):
        amp = np.where(k > 0, k ** (-(alpha + d - 1) / 2.0), 0.0)
    W *= amp
    del amp, k
    g = sfft.irfftn(W, s=shape, workers=_W)
    g -= g.mean()
    g /= g.std()
    return g


def quantization_error(x32: np.ndarray, eps: float) -> np.ndarray:
    """e0 = x_hat - x with x_hat = 2 eps rint(x / 2eps), computed in float64 on
    the float32 field and stored as float32."""
    x = x32.astype(np.float64)
    xh = 2.0 * eps * np.rint(x / (2.0 * eps))
    return (xh - x).astype(np.float32)


def max_abs_fft(x32: np.ndarray) -> float:
    """max_k |X_k| of the float32 field, in float64 (unnormalised DFT)."""
    X = sfft.rfftn(x32.astype(np.float64), workers=_W)
    return float(np.max(np.abs(X)))


def max_box_fft(e32: np.ndarray) -> float:
    """max_k max(|Re X_k|, |Im X_k|), used only to pick stress-test bounds."""
    X = sfft.rfftn(e32.astype(np.float64), workers=_W)
    return float(max(np.max(np.abs(X.real)), np.max(np.abs(X.imag))))


def _item(name, x32, E, D, **extra):
    out = dict(name=name, shape=tuple(x32.shape), x=x32,
               e0=quantization_error(x32, E), E=float(E), D=float(D))
    out.update(extra)
    return out


# -- single fields -----------------------------------------------------------
def grf_field(n=32, alpha=2.0, seed=0, rel_s=1e-4, rel_f=1e-3, stress=None):
    """3D n^3 GRF, P(k) ~ k^-alpha (the 32^3 parity workload at n = 32).

    ``stress``: if given, eps_f = stress * max box violation of e0 instead
    (a labelled stress variant that forces iterations)."""
    x = grf((n, n, n), alpha, seed).astype(np.float32)
    rng = float(x.max()) - float(x.min())
    E = rel_s * rng
    it = _item(f"grf{n}^3", x, E, 1.0)
    it["D"] = (stress * max_box_fft(it["e0"])) if stress else rel_f * max_abs_fft(x)
    it["stress"] = stress
    return it


def lognormal_field(n=512, alpha=2.5, seed=0, rel_s=1e-4, rel_f=1e-3, stress=None):
    """3D n^3 lognormal density, exp of a unit-variance GRF with P(k) ~ k^-alpha."""
    g = grf((n, n, n), alpha, seed)
    np.exp(g, out=g)
    x = g.astype(np.float32)
    del g
    rng = float(x.max()) - float(x.min())
    E = rel_s * rng
    it = _item(f"lognormal{n}^3", x, E, 1.0)
    it["D"] = (stress * max_box_fft(it["e0"])) if stress else rel_f * max_abs_fft(x)
    it["stress"] = stress
    return it


def lognormal_shape(shape, alpha=2.5, seed=0, rel_s=1e-4, rel_f=1e-3, stress=None):
    """The 512^3 workload's recipe on any 3D shape (smaller cases of the same
    kernels for profiling): lognormal of a GRF with P(k) ~ k^-alpha."""
    g = grf(tuple(shape), alpha, seed)
    np.exp(g, out=g)
    x = g.astype(np.float32)
    del g
    rng = float(x.max()) - float(x.min())
    E = rel_s * rng
    it = _item("lognormal" + "x".join(str(n) for n in shape), x, E, 1.0)
    it["D"] = (stress * max_box_fft(it["e0"])) if stress else rel_f * max_abs_fft(x)
    it["stress"] = stress
    return it


def turbulence_field(n=256, seed=0, rel_s=1e-4, rel_fe0=0.2):
    """3D n^3 field with E(k) ~ k^-5/3 (per-mode |k|^-11/3).

    The differentiable workload states no eps_f; eps_f = 0.2 * max box violation
    of e0 so that clips are active and the Jacobian is not the identity."""
    x = grf((n, n, n), 5.0 / 3.0, seed).astype(np.float32)
    rng = float(x.max()) - float(x.min())
    E = rel_s * rng
    it = _item(f"turbulence{n}^3", x, E, 1.0)
    it["D"] = rel_fe0 * max_box_fft(it["e0"])
    return it


# -- batched 2D diffraction-like images --------------------------------------
def diffraction_image(n: int, rng: np.random.Generator) -> np.ndarray:
    """log10 far-field intensity |FFT2(probe * exp(i phi))|^2, phi ~ U[0, pi)
    smoothed by a periodic Gaussian of 3 px, Gaussian probe sigma = n/8."""
    phi = rng.uniform(0.0, np.pi, size=(n, n))
    f = np.fft.fftfreq(n)
    sig = 3.0
    H = np.exp(-2.0 * (np.pi * sig) ** 2 * (f[:, None] ** 2 + f[None, :] ** 2))
    phi = sfft.ifft2(sfft.fft2(phi, workers=_W) * H, workers=_W).real
    c = np.arange(n) - n / 2.0
    probe = np.exp(-(c[:, None] ** 2 + c[None, :] ** 2) / (2.0 * (n / 8.0) ** 2))
    I = np.abs(sfft.fft2(probe * np.exp(1j * phi), workers=_W)) ** 2
    return np.log10(I + 1e-12 * I.max())


def _item_rng(seed: int, i: int) -> np.random.Generator:
    """Independent stream of batch item i (so items can be built in parallel)."""
    return np.random.default_rng(np.random.SeedSequence([seed, i]))


def _map(fn, args, workers):
    if workers and workers > 1 and len(args) > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            return pool.starmap(fn, args, chunksize=max(1, len(args) // (4 * workers)))
    return [fn(*a) for a in args]


def _diffraction_item(i, n, seed, rel_s, eps_f):
    x = diffraction_image(int(n), _item_rng(seed, i)).astype(np.float32)
    E = rel_s * (float(x.max()) - float(x.min()))
    return _item(f"img{i}_{n}", x, E, eps_f)


def diffraction_batch(count=512, sizes=(256, 512, 1024), seed=0, rel_s=1e-3,
                      eps_f=1e-2, workers=0):
    """Images of mixed sizes in near-equal thirds, order shuffled by rng(seed).

    eps_f is absolute (the workload gives no normaliser for it)."""
    per = [count // len(sizes) + (1 if i < count % len(sizes) else 0)
           for i in range(len(sizes))]
    ns = np.concatenate([np.full(p, s) for p, s in zip(per, sizes)])
    rng = np.random.default_rng(seed)
    rng.shuffle(ns)
    return _map(_diffraction_item, [(i, int(n), seed, rel_s, eps_f) for i, n in enumerate(ns)],
                workers)


# -- batched 1D EEG-like signals ---------------------------------------------
def eeg_signal(n: int, rng: np.random.Generator, fs=256.0) -> np.ndarray:
    """1/f noise (unit std) + A sin(2 pi 10 t + phi0) + N(0, 0.1^2)."""
    w = rng.standard_normal(n)
    W = np.fft.rfft(w)
    f = np.fft.rfftfreq(n, d=1.0 / fs)
    with np.errstate(divide="ignore"):
        W *= np.where(f > 0, f ** -0.5, 0.0)
    pink = np.fft.irfft(W, n=n)
    pink /= pink.std()
    t = np.arange(n) / fs
    A = rng.uniform(0.5, 2.0)
    ph = rng.uniform(0.0, 2 * np.pi)
    return pink + A * np.sin(2 * np.pi * 10.0 * t + ph) + rng.normal(0.0, 0.1, n)


def _eeg_item(i, n, seed, rel_s, rel_f):
    x = eeg_signal(int(n), _item_rng(seed, i)).astype(np.float32)
    E = rel_s * (float(x.max()) - float(x.min()))
    D = rel_f * float(np.max(np.abs(np.fft.rfft(x.astype(np.float64)))))
    return _item(f"eeg{i}_{n}", x, E, D)


def eeg_batch(count=4096, lo=1024, hi=65536, seed=0, rel_s=1e-3, rel_f=5e-3,
              lengths=None, workers=0):
    """1D signals of uneven length ~ U{lo..hi} (or the given ``lengths``)."""
    rng = np.random.default_rng(seed)
    ns = lengths if lengths is not None else rng.integers(lo, hi + 1, size=count)
    return _map(_eeg_item, [(i, int(n), seed, rel_s, rel_f) for i, n in enumerate(ns)], workers)


def bimodal_error(shape, seed, E=1.0, dtype=np.float64):
    """Stress error: half the points uniform in [-E, E], half near the faces
    (|e| in [0.8E, E], random sign).  Errors piled near the s-cube faces make
    the two cubes overlap partially, which takes several iterations (Sec. V-C
    discussion of Table 3)."""
    r = np.random.default_rng(seed)
    u = r.uniform(-1.0, 1.0, shape)
    s = np.sign(r.standard_normal(shape)) * r.uniform(0.8, 1.0, shape)
    return (E * np.where(r.uniform(size=shape) < 0.5, s, u)).astype(dtype)


def single_mode(shape, k0, A, dtype=np.float64):
    """e = A cos(2 pi k0 . n / N) for one wavevector k0 (a closed-form case)."""
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape],
                        indexing="ij", sparse=True)
    ph = sum(2.0 * np.pi * k * g / n for k, g, n in zip(k0, grids, shape))
    return (A * np.cos(ph)).astype(dtype)
