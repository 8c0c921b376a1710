"""FP64 CPU oracle for FFCz's alternating projection (Alg. 1, Sec. IV-B).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline
leg and its ``--impl reference`` arm) use it.  It shares no code with the CUDA
library; both sides only share the seeded input generators, which hold none of
the method's arithmetic.

Everything is float64.  The DFT step is a library primitive (``scipy.fft``,
full complex spectrum, no half-spectrum tricks); everything else is written out
in the paper's order.  Readings of passages the paper leaves open are tagged
``A1``..``A20`` and listed, with the reasons, in the design notes.

Notation: ``e`` is the spatial error vector (epsilon in the paper), ``delta``
its frequency error vector, ``E`` the spatial bound and ``D`` the frequency
bound (Delta).  Shrunk bounds ``E' = E(1-eta)``, ``D' = D(1-eta)`` with
``eta = 2**-16`` come from the bound shrink of Sec. IV-B (m = 16).
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np
import scipy.fft as sfft

ETA_DEFAULT = 2.0 ** -16
_WORKERS = int(os.environ.get("FFCZ_ORACLE_THREADS", "0")) or (os.cpu_count() or 1)

# Status codes, same meaning as the C library's (A9: iteration cap).
OK, NOT_CONVERGED, NONFINITE = 0, 4, 6


def workers() -> int:
    """Threads the oracle's FFT step uses."""
    return _WORKERS


# --------------------------------------------------------------------------
# Transforms (Eq. 1 and its 2D/nD analogue, Sec. III; Eq. frequency_err)
# --------------------------------------------------------------------------
def dft(e: np.ndarray) -> np.ndarray:
    """Unnormalised forward DFT over every axis, X_k = sum_n x_n exp(-2 pi i k.n/N).

    Eq. 1 (1D), the 2D formula below it and "additional exponential terms per
    dimension" for 3D.  Full complex spectrum of the same shape as ``e``.
    """
    return sfft.fftn(np.asarray(e, dtype=np.float64), workers=_WORKERS)


def idft(delta: np.ndarray) -> np.ndarray:
    """Inverse of :func:`dft` (scale 1/N), real part (the input is Hermitian)."""
    return sfft.ifftn(delta, workers=_WORKERS).real


# --------------------------------------------------------------------------
# The two projections and the feasibility measure (Sec. IV-A, IV-B, IV-D)
# --------------------------------------------------------------------------
def f_violation(delta: np.ndarray) -> float:
    """max over all bins of max(|Re delta_k|, |Im delta_k|) (constraints_v1, A4).

    NaN anywhere maps to +inf so that a non-finite field never looks feasible.
    """
    if delta.size == 0:
        return 0.0
    v = max(float(np.max(np.abs(delta.real))), float(np.max(np.abs(delta.imag))))
    if np.isnan(v) or not np.all(np.isfinite(delta)):
        return float("inf")
    return v


def project_f(delta: np.ndarray, D: float) -> np.ndarray:
    """ProjectOntoFCube: clip Re and Im of every bin to [-D, D] separately.

    Sec. IV-D: the f-cube faces are pairwise orthogonal, so the projection is
    the per-axis clip in the frequency basis (A6: exact Euclidean projection
    even though the basis vectors are orthogonal rather than orthonormal).
    """
    return np.clip(delta.real, -D, D) + 1j * np.clip(delta.imag, -D, D)


def project_s(e: np.ndarray, E: float) -> np.ndarray:
    """ProjectOntoSCube: clip every spatial error to [-E, E] (constraints_v2c)."""
    return np.clip(e, -E, E)


# --------------------------------------------------------------------------
# Alg. 1, the alternating projection loop
# --------------------------------------------------------------------------
@dataclass
class Result:
    e: np.ndarray                   # corrected error (float64)
    iters: int                      # number of (f-clip, s-clip) pairs run (A8)
    status: int                     # OK / NOT_CONVERGED / NONFINITE
    preclipped: bool                # A3 pre-loop s-projection applied
    f_ratio: float                  # last measured violation / D
    active_s: int = 0               # points moved by the last s-clip
    active_f: int = 0               # bins moved by the last f-clip
    trajectory: list = field(default_factory=list)   # e after every iteration
    # Alg. 1 edit accumulators (when requested): the displacement of the error
    # vector along the spatial basis (spat_edits, shape of e) and along the
    # frequency basis (freq_edits, full complex spectrum, Hermitian)
    spat_edits: np.ndarray | None = None
    freq_edits: np.ndarray | None = None


def thresholds(E: float, D: float, eta: float):
    """Shrunk bounds and the stopping threshold (Sec. IV-B shrink; A7)."""
    return E * (1.0 - eta), D * (1.0 - eta), D * (1.0 - eta / 2.0)


def correct(e0: np.ndarray, E: float, D: float, *, min_iters: int = 0,
            max_iters: int = 10000, eta: float = ETA_DEFAULT,
            record: bool = False, edits: bool = False) -> Result:
    """Alg. 1 (Sec. IV-B), the loop of FFT, CheckConvergence, ProjectOntoFCube,
    IFFT, ProjectOntoSCube, with the readings A3 (pre-loop s-projection), A7
    (shrunk projections, midpoint stopping test) and A9 (iteration cap).

    ``e0`` is the base compressor's error x_hat - x (Alg. 1, first step; A1).
    Returns the iterate at which the check passed, or the last one at the cap.

    With ``edits`` the spatial and frequency edits of Alg. 1 are accumulated:
    after each ProjectOntoFCube freq_edits += delta' - delta, after each
    ProjectOntoSCube spat_edits += eps' - eps (A18: the pre-loop s-projection
    of A3 is a spatial edit too; the check that stops the loop projects
    nothing).
    """
    e = np.asarray(e0, dtype=np.float64).copy()
    Es, Ds, thr = thresholds(E, D, eta)
    S = np.zeros_like(e) if edits else None
    F = np.zeros(e.shape, dtype=np.complex128) if edits else None
    pre = bool(e.size and np.max(np.abs(e)) > E)          # A3
    if pre:
        e_p = project_s(e, Es)
        if edits:
            S += e_p - e
        e = e_p
    t = 0
    act_s = act_f = 0
    traj = []

    def done(status, v):
        return Result(e, t, status, pre, v / D if D > 0 else v, act_s, act_f, traj, S, F)

    while True:
        delta = dft(e)                                    # FFT(eps)
        v = f_violation(delta)                            # CheckConvergence
        if not np.isfinite(v):
            return done(NONFINITE, v)
        if v <= thr and t >= min_iters:
            return done(OK, v)
        if t >= max_iters:
            return done(NOT_CONVERGED, v)
        delta_c = project_f(delta, Ds)                    # ProjectOntoFCube
        act_f = int(np.count_nonzero(delta_c != delta))
        if edits:
            F += delta_c - delta                          # freq_edits += delta' - delta
        e_i = idft(delta_c)                               # IFFT
        e = project_s(e_i, Es)                            # ProjectOntoSCube
        act_s = int(np.count_nonzero(e != e_i))
        if edits:
            S += e - e_i                                  # spat_edits += eps' - eps
        t += 1
        if record:
            traj.append(e.copy())


def certify(e: np.ndarray, E: float, D: float):
    """Check |e_n| <= E and |Re|,|Im| of every DFT bin <= D (constraints_v1).

    Returns (ok, max|e|, f_violation).  Comparisons are <= against the true,
    unshrunk bounds (A7).
    """
    e = np.asarray(e, dtype=np.float64)
    s = float(np.max(np.abs(e))) if e.size else 0.0
    v = f_violation(dft(e))
    return bool(s <= E and v <= D), s, v


# --------------------------------------------------------------------------
# Edits: storage form and application (Alg. 1 after the loop; Sec. IV-B,
# "Compaction, quantization ..." and "Applying edits ...")
# --------------------------------------------------------------------------
def half_spectrum(F: np.ndarray) -> np.ndarray:
    """The stored half of a Hermitian spectrum: last axis k = 0..N/2 (the
    layout of a real-input FFT); the other half is its conjugate (A19)."""
    return F[..., : F.shape[-1] // 2 + 1]


def compact_edits(values: np.ndarray):
    """CompactEdits: flags = 1 where the edit is nonzero (a complex edit is one
    component, nonzero if its real or imaginary part is), packed 8 per byte
    with the first component in the least significant bit (A20); compact =
    the nonzero edits in C order."""
    flat = np.asarray(values).reshape(-1)
    nz = (flat.real != 0) | (flat.imag != 0) if np.iscomplexobj(flat) else flat != 0
    return np.packbits(nz, bitorder="little"), flat[nz]


def expand_edits(flags: np.ndarray, compact: np.ndarray, n: int) -> np.ndarray:
    """Inverse of :func:`compact_edits` for n components."""
    nz = np.unpackbits(np.asarray(flags, dtype=np.uint8), count=n, bitorder="little").astype(bool)
    out = np.zeros(n, dtype=np.asarray(compact).dtype)
    out[nz] = compact
    return out


def quant_step(bound: float, m: int = 16, dtype=np.float64):
    """QuantizeEdits splits each axis [-bound, bound] of the s- or f-cube into
    2^m intervals: step q = 2 bound / 2^m (in the given precision)."""
    return dtype(dtype(bound) * dtype(2.0 ** (1 - m)))


def quantize_edits(compact: np.ndarray, bound: float, m: int = 16, dtype=np.float64) -> np.ndarray:
    """QuantizeEdits: integer codes rint(edit / q), ties to even, the division
    and the rounding in ``dtype`` (A20).  Complex edits give (Re, Im) code
    pairs."""
    q = quant_step(bound, m, dtype)
    c = np.asarray(compact)
    if np.iscomplexobj(c):
        parts = np.stack([c.real.astype(dtype), c.imag.astype(dtype)], axis=-1)
    else:
        parts = c.astype(dtype)
    return np.rint(parts / q).astype(np.int64)


def dequantize_edits(codes: np.ndarray, bound: float, m: int = 16, complex_pairs: bool = False):
    """Edits from codes: code * q (float64)."""
    q = quant_step(bound, m)
    v = np.asarray(codes, dtype=np.float64) * q
    return v[..., 0] + 1j * v[..., 1] if complex_pairs else v


def apply_edits(xhat: np.ndarray, spat: np.ndarray, freq_half: np.ndarray) -> np.ndarray:
    """Applying edits (Sec. IV-B): the complete spatial edit is the spatial
    edits plus the inverse FFT of the frequency edits; the result is the base
    reconstruction plus that complete edit.  ``freq_half`` is the stored half
    spectrum of the (Hermitian) frequency edits."""
    xhat = np.asarray(xhat, dtype=np.float64)
    full = sfft.irfftn(np.asarray(freq_half, dtype=np.complex128), s=xhat.shape, workers=_WORKERS)
    return xhat + np.asarray(spat, dtype=np.float64) + full


# --------------------------------------------------------------------------
# Adjoint of K forced iterations (derived from Alg. 1; A14)
# --------------------------------------------------------------------------
def forward_masks(e0: np.ndarray, E: float, D: float, K: int, eta: float = ETA_DEFAULT):
    """Run exactly K iterations (min_iters = max_iters = K) and keep the
    active-set masks of every clip: 1 where the clip is the identity
    (|value| <= bound, ties count as inside, A14), 0 where it clipped.

    Returns (e_K, pre_mask or None, [(mask_re, mask_im, mask_s)]*K).
    """
    e = np.asarray(e0, dtype=np.float64).copy()
    Es, Ds, _ = thresholds(E, D, eta)
    pre_mask = None
    if e.size and np.max(np.abs(e)) > E:                  # A3
        pre_mask = (np.abs(e) <= Es).astype(np.float64)
        e = project_s(e, Es)
    masks = []
    for _ in range(K):
        delta = dft(e)
        m_re = (np.abs(delta.real) <= Ds).astype(np.float64)
        m_im = (np.abs(delta.imag) <= Ds).astype(np.float64)
        e_i = idft(project_f(delta, Ds))
        m_s = (np.abs(e_i) <= Es).astype(np.float64)
        e = project_s(e_i, Es)
        masks.append((m_re, m_im, m_s))
    return e, pre_mask, masks


def correct_backward(e0: np.ndarray, g_out: np.ndarray, E: float, D: float,
                     K: int, eta: float = ETA_DEFAULT) -> np.ndarray:
    """Vector-Jacobian product of e0 -> e_K for K forced iterations.

    One step is e <- P_s(IDFT(P_f(DFT(e)))), whose Jacobian is
    M_s . IDFT . M_f . DFT.  In the real frequency basis of Sec. IV-A the map
    IDFT . M_f . DFT is symmetric (sum_j m_j a_j a_j^T / |a_j|^2), so the
    transposed step is g <- IDFT(M_f * DFT(M_s * g)), with M_f acting on Re and
    Im separately.  Steps are undone from the last to the first.
    """
    _, pre_mask, masks = forward_masks(e0, E, D, K, eta)
    g = np.asarray(g_out, dtype=np.float64).copy()
    for m_re, m_im, m_s in reversed(masks):
        g = g * m_s
        G = dft(g)
        G = G.real * m_re + 1j * (G.imag * m_im)
        g = idft(G)
    if pre_mask is not None:
        g = g * pre_mask
    return g


# --------------------------------------------------------------------------
# Batched form (A15): every item runs its own loop
# --------------------------------------------------------------------------
def correct_batch(items, Es, Ds, **kw):
    """Run :func:`correct` on every item independently (A15)."""
    return [correct(x, float(E), float(D), **kw) for x, E, D in zip(items, Es, Ds)]
