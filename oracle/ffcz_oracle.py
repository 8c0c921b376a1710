"""FP64 CPU oracle for FFCz's alternating projection (Alg. 1, Sec. IV-B).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline
leg and its ``--impl reference`` arm) use it.  It shares no code with the CUDA
library; both sides only share the seeded input generators, which hold none of
the method's arithmetic.

Everything is float64.  The DFT step is a library primitive (``scipy.fft``,
full complex spectrum, no half-spectrum tricks); everything else is written out
in the paper's order.  Where the paper leaves a passage open, the reading
taken is tagged ``A1``..``A27`` and stated in the docstring of the function
that applies it.

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


def project_s(e: np.ndarray, E) -> np.ndarray:
    """ProjectOntoSCube: clip every spatial error to [-E, E] (constraints_v2c);
    E a scalar or, for pointwise bounds E_n (footnote of Sec. IV-A), an array
    of the field's shape."""
    return np.clip(e, -E, E)


def project_f_pw(delta: np.ndarray, D_re: np.ndarray, D_im: np.ndarray) -> np.ndarray:
    """ProjectOntoFCube with pointwise bounds Delta_k^Re, Delta_k^Im (full
    spectrum arrays, even in k so that Hermitian symmetry is kept; A23)."""
    return np.clip(delta.real, -D_re, D_re) + 1j * np.clip(delta.imag, -D_im, D_im)


def f_ratio_pw(delta: np.ndarray, D_re: np.ndarray, D_im: np.ndarray) -> float:
    """Normalised violation max_k max(|Re delta_k| / D_re_k, |Im delta_k| / D_im_k)
    (NaN maps to +inf)."""
    if delta.size == 0:
        return 0.0
    r = max(float(np.max(np.abs(delta.real) / D_re)), float(np.max(np.abs(delta.imag) / D_im)))
    if np.isnan(r) or not np.all(np.isfinite(delta)):
        return float("inf")
    return r


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
    pw_f = isinstance(D, tuple)
    if pw_f:
        # pointwise frequency bounds (A23): (Delta^Re, Delta^Im) full-spectrum arrays
        D_re, D_im = (np.asarray(x, dtype=np.float64) for x in D)
        Es = np.asarray(E, dtype=np.float64) * (1.0 - eta)
        Ds_re, Ds_im = D_re * (1.0 - eta), D_im * (1.0 - eta)
        thr_r = 1.0 - eta / 2.0
        D = 1.0                                           # the ratio is normalised
    else:
        Es, Ds, thr = thresholds(E, D, eta)
    S = np.zeros_like(e) if edits else None
    F = np.zeros(e.shape, dtype=np.complex128) if edits else None
    pre = bool(e.size and np.any(np.abs(e) > E))          # A3
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
        if pw_f:
            v = f_ratio_pw(delta, D_re, D_im)             # CheckConvergence (normalised)
            stop = v <= thr_r
        else:
            v = f_violation(delta)                        # CheckConvergence
            stop = v <= thr
        if not np.isfinite(v):
            return done(NONFINITE, v)
        if stop and t >= min_iters:
            return done(OK, v)
        if t >= max_iters:
            return done(NOT_CONVERGED, v)
        delta_c = project_f_pw(delta, Ds_re, Ds_im) if pw_f else project_f(delta, Ds)   # ProjectOntoFCube
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


def certify(e: np.ndarray, E, D):
    """Check |e_n| <= E and |Re|,|Im| of every DFT bin <= D (constraints_v1).

    Returns (ok, max|e|, f_violation).  Comparisons are <= against the true,
    unshrunk bounds (A7).  With pointwise bounds (E an array, D a pair of
    full-spectrum arrays) the two maxima are the ratios max|e_n|/E_n and the
    normalised violation, each compared with 1.
    """
    e = np.asarray(e, dtype=np.float64)
    if isinstance(D, tuple) or np.ndim(E) > 0:
        s = float(np.max(np.abs(e) / E)) if e.size else 0.0
        if isinstance(D, tuple):
            v = f_ratio_pw(dft(e), *D)
        else:
            v = f_violation(dft(e)) / D
        return bool(s <= 1.0 and v <= 1.0), s, v
    s = float(np.max(np.abs(e))) if e.size else 0.0
    v = f_violation(dft(e))
    return bool(s <= E and v <= D), s, v


def shell_index(shape) -> np.ndarray:
    """Power-spectrum shell of every DFT bin: the rounded radius of its signed
    frequency vector (Sec. III, P(k) sums |X|^2 over bins at distance k from
    the centre after the zero-frequency shift; A12)."""
    grids = np.meshgrid(*[np.fft.fftfreq(n) * n for n in shape], indexing="ij")
    return np.rint(np.sqrt(sum(g * g for g in grids))).astype(np.int64)


def power_spectrum(x: np.ndarray, mean: float | None = None) -> np.ndarray:
    """P(k) of Sec. III: normalise (x - mean) / mean (the field's own mean by
    default), FFT, sum |X|^2 over each shell."""
    x = np.asarray(x, dtype=np.float64)
    m = float(np.mean(x)) if mean is None else mean
    X = dft((x - m) / m)
    return np.bincount(shell_index(x.shape).reshape(-1), weights=(np.abs(X) ** 2).reshape(-1))


def power_spectrum_bounds(x: np.ndarray, rho: float):
    """Pointwise frequency bounds from a relative bound rho on every shell of
    the power spectrum (Sec. V, power-spectrum preservation; reading A24).

    With X' = FFT((x - xbar)/xbar) and an error delta' = delta/xbar whose Re
    and Im are within d_s on shell s, |X' + delta'|^2 - |X'|^2 <= 2 sqrt(2)
    d_s |X'_k| + 2 d_s^2 per bin, so the shell total stays within rho P(s) if
    2 n_s d_s^2 + 2 sqrt(2) A_s d_s = rho P(s), A_s = sum |X'_k| over the
    shell, n_s its bin count: d_s is the positive root.  The zero-frequency
    shell (P(0) = 0 once the mean is removed, so no relative bound exists)
    takes the smallest bound of the other shells.  Returns (Delta^Re, Delta^Im) = (|xbar| d, |xbar| d), full
    spectrum, even in k.
    """
    x = np.asarray(x, dtype=np.float64)
    xbar = float(np.mean(x))
    Xp = dft((x - xbar) / xbar)
    s = shell_index(x.shape).reshape(-1)
    P = np.bincount(s, weights=(np.abs(Xp) ** 2).reshape(-1))
    A = np.bincount(s, weights=np.abs(Xp).reshape(-1))
    n = np.bincount(s).astype(np.float64)
    d = (-2.0 * np.sqrt(2.0) * A + np.sqrt(8.0 * A * A + 8.0 * n * rho * P)) / (4.0 * np.maximum(n, 1.0))
    if d.size > 1:
        d[0] = d[1:][n[1:] > 0].min()        # the zero-frequency shell
    bound = (abs(xbar) * d[s]).reshape(x.shape)
    return bound, bound.copy()


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


ESCAPE16 = -(2 ** 15)


def narrow_codes(codes: np.ndarray):
    """m-bit storage of the codes (Sec. IV-B: each axis of the cube in 2^m
    intervals, codes of m bits; m = 16).  A27: a code in [-32767, 32767] is
    stored as itself in int16; any other code (the end point 2^15 = bound / q,
    or an edit larger than the bound) is stored as the escape -32768 and its
    value appended, in order of appearance, to an int32 list.  Returns
    (int16 codes, int32 list); the codes are taken in flat order."""
    c = np.asarray(codes, dtype=np.int64).reshape(-1)
    lim = 2 ** 15 - 1
    out = np.empty(c.size, dtype=np.int16)
    wide = []
    for i in range(c.size):
        v = int(c[i])
        if -lim <= v <= lim:
            out[i] = v
        else:
            out[i] = ESCAPE16
            wide.append(v)
    return out, np.asarray(wide, dtype=np.int32)


def widen_codes(c16: np.ndarray, wide: np.ndarray) -> np.ndarray:
    """The codes back from their 16-bit storage (A27): each escape takes the
    next entry of the list."""
    c16 = np.asarray(c16, dtype=np.int16).reshape(-1)
    out = np.empty(c16.size, dtype=np.int64)
    k = 0
    for i in range(c16.size):
        if int(c16[i]) == ESCAPE16:
            out[i] = int(wide[k])
            k += 1
        else:
            out[i] = int(c16[i])
    if k != len(wide):
        raise ValueError("escape count does not match the list")
    return out


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
    return backward_from_masks(g_out, pre_mask, masks)


def backward_from_masks(g_out: np.ndarray, pre_mask, masks) -> np.ndarray:
    """The transposed steps g <- IDFT(M_f * DFT(M_s * g)), last step first,
    for given active-set masks (those of :func:`forward_masks`)."""
    g = np.asarray(g_out, dtype=np.float64).copy()
    for m_re, m_im, m_s in reversed(masks):
        g = g * m_s
        G = dft(g)
        G = G.real * m_re + 1j * (G.imag * m_im)
        g = idft(G)
    if pre_mask is not None:
        g = g * pre_mask
    return g


def near_ties(e0: np.ndarray, E: float, D: float, K: int, tau: float,
              eta: float = ETA_DEFAULT):
    """The clip decisions of K forced iterations that a small perturbation of
    the trajectory could reverse: for every step, the Re, Im and spatial
    entries whose pre-clip magnitude lies within tau * bound of the shrunk
    bound (| |v| - B | <= tau B).  The masks of :func:`forward_masks` take
    one side of each such near tie (A14); a computation of the same
    trajectory in another precision may take the other.
    Returns [(near_re, near_im, near_s)] * K (boolean arrays)."""
    e = np.asarray(e0, dtype=np.float64).copy()
    Es, Ds, _ = thresholds(E, D, eta)
    if e.size and np.max(np.abs(e)) > E:                  # A3
        e = project_s(e, Es)
    out = []
    for _ in range(K):
        delta = dft(e)
        n_re = np.abs(np.abs(delta.real) - Ds) <= tau * Ds
        n_im = np.abs(np.abs(delta.imag) - Ds) <= tau * Ds
        e_i = idft(project_f(delta, Ds))
        n_s = np.abs(np.abs(e_i) - Es) <= tau * Es
        e = project_s(e_i, Es)
        out.append((n_re, n_im, n_s))
    return out


def tie_spread(e0: np.ndarray, g_out: np.ndarray, E: float, D: float, K: int,
               tau: float, samples: int = 8, seed: int = 0,
               eta: float = ETA_DEFAULT):
    """How far the vector-Jacobian product moves, coordinate by coordinate,
    when the near ties of :func:`near_ties` are decided otherwise: the
    largest |g' - g| over g' computed with every near tie inside, every near
    tie outside, and ``samples`` random decisions (each near tie inside with
    probability 1/2).  Zero where the trajectory has no near tie.
    Returns (spread, number of near-tie entries)."""
    _, pre_mask, masks = forward_masks(e0, E, D, K, eta)
    near = near_ties(e0, E, D, K, tau, eta)
    g_ref = backward_from_masks(g_out, pre_mask, masks)
    count = int(sum(int(a.sum() + b.sum() + c.sum()) for a, b, c in near))
    spread = np.zeros_like(g_ref)
    if count == 0:
        return spread, 0
    rng = np.random.default_rng(seed)
    for trial in range(samples + 2):
        alt = []
        for (m_re, m_im, m_s), nears in zip(masks, near):
            ms = []
            for m, n in zip((m_re, m_im, m_s), nears):
                if trial == 0:
                    side = np.ones(m.shape)
                elif trial == 1:
                    side = np.zeros(m.shape)
                else:
                    side = (rng.random(m.shape) < 0.5).astype(np.float64)
                ms.append(np.where(n, side, m))
            alt.append(tuple(ms))
        g_alt = backward_from_masks(g_out, pre_mask, alt)
        spread = np.maximum(spread, np.abs(g_alt - g_ref))
    return spread, count


# --------------------------------------------------------------------------
# Projection variants named as alternatives to POCS (Sec. III, POCS
# paragraph; a direct or faster scheme is future work in Sec. VI).  A25.
# --------------------------------------------------------------------------
def project_f_spatial(z: np.ndarray, Ds) -> np.ndarray:
    """P_F' as a map of spatial vectors: IDFT(ProjectOntoFCube(DFT(z)))."""
    return idft(project_f(dft(z), Ds))


def _variant_start(e0, E, eta):
    e = np.asarray(e0, dtype=np.float64).copy()
    pre = bool(e.size and np.any(np.abs(e) > E))          # A3, as in Alg. 1
    if pre:
        e = project_s(e, E * (1.0 - eta))
    return e, pre


def correct_dykstra(e0: np.ndarray, E: float, D: float, *, min_iters: int = 0,
                    max_iters: int = 10000, eta: float = ETA_DEFAULT,
                    record: bool = False) -> Result:
    """Dykstra's alternating projection onto F' then S' (Sec. III names it).

    x_0 = e0 (after A3), p_0 = q_0 = 0, and per iteration
        y = P_F'(x + p),  p <- x + p - y,
        x' = P_S'(y + q), q <- y + q - x'.
    The iterates converge to the point of S' and F' nearest to e0 (the
    Euclidean projection of e0 onto the intersection), where POCS converges
    to some point of it.  The check of Alg. 1 runs on x (always inside S'):
    stop when its DFT violation <= D(1 - eta/2); the count is the number of
    (P_F', P_S') pairs run, as for Alg. 1 (A8).
    """
    Es, Ds, thr = thresholds(E, D, eta)
    x, pre = _variant_start(e0, E, eta)
    p = np.zeros_like(x)
    q = np.zeros_like(x)
    t = 0
    traj = []
    while True:
        v = f_violation(dft(x))
        if not np.isfinite(v):
            return Result(x, t, NONFINITE, pre, v / D, trajectory=traj)
        if v <= thr and t >= min_iters:
            return Result(x, t, OK, pre, v / D, trajectory=traj)
        if t >= max_iters:
            return Result(x, t, NOT_CONVERGED, pre, v / D, trajectory=traj)
        y = project_f_spatial(x + p, Ds)
        p = x + p - y
        x_new = project_s(y + q, Es)
        q = y + q - x_new
        x = x_new
        t += 1
        if record:
            traj.append(x.copy())


def correct_douglas_rachford(e0: np.ndarray, E: float, D: float, *, min_iters: int = 0,
                             max_iters: int = 10000, eta: float = ETA_DEFAULT,
                             record: bool = False) -> Result:
    """Douglas-Rachford splitting for the feasibility problem of F' and S'
    (Sec. III names it; its governing sequence z may end outside the
    intersection, which is why the check runs on the S'-point x).

    z_0 = e0 (after A3), and per iteration
        y = P_F'(z),  x = P_S'(2y - z),  z <- z + x - y.
    The candidate checked (as in Alg. 1) is x, e0 before the first iteration.
    """
    Es, Ds, thr = thresholds(E, D, eta)
    z, pre = _variant_start(e0, E, eta)
    x = z.copy()
    t = 0
    traj = []
    while True:
        v = f_violation(dft(x))
        if not np.isfinite(v):
            return Result(x, t, NONFINITE, pre, v / D, trajectory=traj)
        if v <= thr and t >= min_iters:
            return Result(x, t, OK, pre, v / D, trajectory=traj)
        if t >= max_iters:
            return Result(x, t, NOT_CONVERGED, pre, v / D, trajectory=traj)
        y = project_f_spatial(z, Ds)
        x = project_s(2.0 * y - z, Es)
        z = z + x - y
        t += 1
        if record:
            traj.append(x.copy())


def correct_admm(e0: np.ndarray, E: float, D: float, *, min_iters: int = 0,
                 max_iters: int = 10000, eta: float = ETA_DEFAULT,
                 record: bool = False) -> Result:
    """ADMM (scaled form) for: find a in F', b in S' with a = b (Sec. III
    names it), i.e. minimise i_F'(a) + i_S'(b) subject to a - b = 0:

        a <- P_F'(b - u),  b <- P_S'(a + u),  u <- u + a - b,

    from b_0 = e0 (after A3), u_0 = 0.  The penalty parameter drops out
    because both functions are indicators.  The candidate checked before the
    first iteration is b_0 = e0 (its DFT violation, as in Alg. 1); after
    iteration t it is a_t, which lies in F' by construction and is checked
    against the s-cube: stop when max|a_t| <= E(1 - eta/2) (the midpoint rule
    of A7 applied to the spatial bound).
    """
    Es, Ds, thr = thresholds(E, D, eta)
    thr_s = E * (1.0 - eta / 2.0)
    b, pre = _variant_start(e0, E, eta)
    u = np.zeros_like(b)
    v = f_violation(dft(b))
    if not np.isfinite(v):
        return Result(b, 0, NONFINITE, pre, v / D)
    if v <= thr and min_iters <= 0:
        return Result(b, 0, OK, pre, v / D)
    if max_iters <= 0:
        return Result(b, 0, NOT_CONVERGED, pre, v / D)
    t = 0
    traj = []
    while True:
        a = project_f_spatial(b - u, Ds)
        t += 1
        if record:
            traj.append(a.copy())
        sv = float(np.max(np.abs(a))) if a.size else 0.0
        if not np.isfinite(sv):
            return Result(a, t, NONFINITE, pre, sv / E, trajectory=traj)
        if sv <= thr_s and t >= min_iters:
            return Result(a, t, OK, pre, sv / E, trajectory=traj)
        if t >= max_iters:
            return Result(a, t, NOT_CONVERGED, pre, sv / E, trajectory=traj)
        b = project_s(a + u, Es)
        u = u + a - b


METHODS = {"pocs": None, "dykstra": correct_dykstra, "dr": correct_douglas_rachford,
           "admm": correct_admm}


def correct_method(e0, E, D, method: str = "pocs", **kw) -> Result:
    """Alg. 1 (``pocs``) or one of the projection variants of Sec. III."""
    if method == "pocs":
        return correct(e0, E, D, **kw)
    return METHODS[method](e0, E, D, **kw)


# --------------------------------------------------------------------------
# Batched form (A15): every item runs its own loop
# --------------------------------------------------------------------------
def correct_batch(items, Es, Ds, **kw):
    """Run :func:`correct` on every item independently (A15)."""
    return [correct(x, float(E), float(D), **kw) for x, E, D in zip(items, Es, Ds)]
