"""Pins of the oracle's power-spectrum functions (Sec. III "Power spectrum";
the relative-bound mapping of reading A24), checked against values written out
here by hand or derived in closed form -- never against the functions
themselves.

Sec. III: x' = (x - mean) / mean, X' = FFT(x') with the zero frequency shifted
to the centre, and P(k) sums |X'|^2 over the bins whose distance from the
centre is k.  After the shift, bin index i of an axis of length n sits at the
signed frequency i for i <= (n - 1) // 2 and i - n above it; the distance is
rounded to the nearest integer shell (A12).
"""
import numpy as np
import pytest

from oracle import ffcz_oracle as O

# Shells of a 4 x 4 x 4 grid, enumerated by hand.  Axis index 0, 1, 2, 3 is
# the signed frequency 0, 1, -2, -1 (squares 0, 1, 4, 1); a bin's shell is the
# rounded root of the summed squares: 0 -> 0, 1 and 2 -> 1, 3 to 6 -> 2,
# 8, 9 and 12 -> 3.
SHELLS_444 = np.array([
    # i = 0
    [[0, 1, 2, 1], [1, 1, 2, 1], [2, 2, 3, 2], [1, 1, 2, 1]],
    # i = 1
    [[1, 1, 2, 1], [1, 2, 2, 2], [2, 2, 3, 2], [1, 2, 2, 2]],
    # i = 2
    [[2, 2, 3, 2], [2, 2, 3, 2], [3, 3, 3, 3], [2, 2, 3, 2]],
    # i = 3
    [[1, 1, 2, 1], [1, 2, 2, 2], [2, 2, 3, 2], [1, 2, 2, 2]],
])

# A 3 x 5 grid (odd lengths: signed frequencies 0, 1, -1 and 0, 1, 2, -2, -1;
# squares 0, 1, 1 and 0, 1, 4, 4, 1).
SHELLS_35 = np.array([
    [0, 1, 2, 2, 1],
    [1, 1, 2, 2, 1],
    [1, 1, 2, 2, 1],
])

# A 2 x 6 grid (signed frequencies 0, -1 and 0, 1, 2, -3, -2, -1): the
# Nyquist index of an even axis counts as -n/2, distance n/2 either way.
SHELLS_26 = np.array([
    [0, 1, 2, 3, 2, 1],
    [1, 1, 2, 3, 2, 1],
])


def test_shell_index_hand_enumerated():
    np.testing.assert_array_equal(O.shell_index((4, 4, 4)), SHELLS_444)
    np.testing.assert_array_equal(O.shell_index((3, 5)), SHELLS_35)
    np.testing.assert_array_equal(O.shell_index((2, 6)), SHELLS_26)
    np.testing.assert_array_equal(O.shell_index((8,)), [0, 1, 2, 3, 4, 3, 2, 1])


def _cosine_field(shape, k0, A, m):
    """m + A cos(2 pi k0 . n / N): mean exactly m for k0 != 0."""
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij", sparse=True)
    ph = sum(2.0 * np.pi * k * g / n for k, g, n in zip(k0, grids, shape))
    return m + A * np.cos(ph)


@pytest.mark.parametrize("shape,k0,shell", [((8, 8, 8), (1, 2, 3), 4),      # |k0| = sqrt 14 = 3.74
                                            ((16, 8), (5, -2), 5),           # sqrt 29 = 5.39
                                            ((6, 10, 4), (2, 3, 1), 4)])     # sqrt 14, non-cubic
def test_power_spectrum_single_cosine_closed_form(shape, k0, shell):
    """(x - m)/m = (A/m) cos(...) has the two real spikes N A / (2m) at +-k0
    and nothing else, so all of P sits in shell round(|k0|):
    P = 2 (N A / (2m))^2."""
    N = int(np.prod(shape))
    A, m = 0.75, 3.0
    P = O.power_spectrum(_cosine_field(shape, k0, A, m))
    want = np.zeros_like(P)
    want[shell] = 2.0 * (N * A / (2.0 * m)) ** 2
    np.testing.assert_allclose(P, want, rtol=1e-12, atol=1e-9 * want[shell])


def test_power_spectrum_self_conjugate_cosine():
    """k0 = (4, 0, 0) on 8^3 is its own mirror: cos(pi n) is one real spike
    N A / m, so P(4) = (N A / m)^2."""
    N, A, m = 512, 0.5, 2.0
    P = O.power_spectrum(_cosine_field((8, 8, 8), (4, 0, 0), A, m))
    want = np.zeros_like(P)
    want[4] = (N * A / m) ** 2
    np.testing.assert_allclose(P, want, rtol=1e-12, atol=1e-9 * want[4])


def test_power_spectrum_mean_normalisation():
    """P of x and of c x are equal (the mean normalisation makes P
    scale-free); P of x + c changes by the factor (m / (m + c))^2."""
    r = np.random.default_rng(3)
    x = r.standard_normal((6, 8, 4)) + 5.0
    m = float(np.mean(x))
    P = O.power_spectrum(x)
    tol = dict(rtol=1e-12, atol=1e-12 * float(P.max()))   # shell 0 holds only rounding
    np.testing.assert_allclose(O.power_spectrum(7.5 * x), P, **tol)
    np.testing.assert_allclose(O.power_spectrum(x + 2.0), P * (m / (m + 2.0)) ** 2, **tol)


def _signed_sq_radius(shape):
    """Squared distance of every bin from the shifted centre, written out
    per axis (used to pick bins of one shell without the oracle)."""
    r2 = np.zeros(shape)
    for ax, n in enumerate(shape):
        f = np.array([i if i <= (n - 1) // 2 else i - n for i in range(n)], dtype=np.float64)
        sh = [1] * len(shape)
        sh[ax] = n
        r2 = r2 + (f * f).reshape(sh)
    return r2


def _phase_pi4_field(shape, shell, mean, seed):
    """A real field of mean `mean` whose normalised spectrum X' has phase
    +-pi/4 or +-3pi/4 on every bin of `shell` (none of which is its own
    mirror) and random values elsewhere; returns (x, X', shell mask)."""
    r = np.random.default_rng(seed)
    Xp = np.fft.fftn(r.standard_normal(shape))
    Xp.flat[0] = 0.0
    r2 = _signed_sq_radius(shape)
    # rounded radius == shell  <=>  (shell - 1/2)^2 <= r2 < (shell + 1/2)^2
    # for integer r2 (no radius is a half integer)
    inshell = ((shell - 0.5) ** 2 <= r2) & (r2 < (shell + 0.5) ** 2)
    mirror = tuple(np.ix_(*[(-np.arange(n)) % n for n in shape]))
    idx = np.argwhere(inshell)
    done = np.zeros(shape, dtype=bool)
    for k in map(tuple, idx):
        if done[k]:
            continue
        km = tuple((-np.array(k)) % np.array(shape))
        assert km != k, "a self-conjugate bin in the chosen shell"
        sgn = r.choice([-1.0, 1.0], size=2)
        v = r.uniform(0.5, 2.0) * (sgn[0] + 1j * sgn[1])
        Xp[k], Xp[km] = v, np.conj(v)
        done[k] = done[km] = True
    xp = np.fft.ifftn(Xp)
    assert np.max(np.abs(xp.imag)) < 1e-12 * np.max(np.abs(xp.real))
    np.testing.assert_array_equal(inshell, inshell[mirror])
    return mean * (1.0 + xp.real), Xp, inshell


@pytest.mark.parametrize("shape,shell,rho", [((8, 8, 8), 3, 1e-2), ((16, 12), 5, 1e-3), ((10, 6, 8), 2, 0.3)])
def test_power_spectrum_bounds_are_tight_on_aligned_corners(shape, shell, rho):
    """Equality case of reading A24: when every bin of a shell has phase
    +-pi/4 (mod pi/2) and the error sits on the box corner aligned with it,
    |X' + d(+-1 +-i)|^2 - |X'|^2 = 2 sqrt2 d |X'| + 2 d^2 on every bin, so the
    shell's power changes by exactly 2 sqrt2 d A_s + 2 n_s d^2 = rho P(s)."""
    mean = 2.5
    x, Xp, inshell = _phase_pi4_field(shape, shell, mean, seed=sum(shape))
    D_re, D_im = O.power_spectrum_bounds(x, rho)
    np.testing.assert_array_equal(D_re, D_im)
    d = D_re[inshell] / mean                         # the per-bin d of the normalised error
    np.testing.assert_allclose(d, d[0], rtol=1e-12)  # one value per shell
    # the aligned corner error, on the shell's bins only
    delta = np.zeros(shape, dtype=np.complex128)
    delta[inshell] = D_re[inshell] * (np.sign(Xp[inshell].real) + 1j * np.sign(Xp[inshell].imag))
    e = np.fft.ifftn(delta)
    assert np.max(np.abs(e.imag)) < 1e-12 * np.max(np.abs(e.real))
    Xh = np.fft.fftn((x + e.real - mean) / mean)
    P_s = float(np.sum(np.abs(Xp[inshell]) ** 2))
    P_hat = float(np.sum(np.abs(Xh[inshell]) ** 2))
    np.testing.assert_allclose(P_hat - P_s, rho * P_s, rtol=1e-10)
    # the corner error at half the bound changes the shell by less than rho
    Xh2 = np.fft.fftn((x + 0.5 * e.real - mean) / mean)
    assert float(np.sum(np.abs(Xh2[inshell]) ** 2)) - P_s < 0.6 * rho * P_s


def test_power_spectrum_pins_catch_planted_mistakes(monkeypatch):
    """Each planted mistake in the shell or spectrum definition fails one of
    the pins above."""
    good_shell = O.shell_index

    def unsigned_shell(shape):          # radius of the raw index, no shift to the centre
        grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
        return np.rint(np.sqrt(sum(g * g for g in grids))).astype(np.int64)

    def floor_shell(shape):             # truncated instead of rounded radius
        grids = np.meshgrid(*[np.fft.fftfreq(n) * n for n in shape], indexing="ij")
        return np.floor(np.sqrt(sum(g * g for g in grids))).astype(np.int64)

    for bad in (unsigned_shell, floor_shell):
        monkeypatch.setattr(O, "shell_index", bad)
        with pytest.raises(AssertionError):
            test_shell_index_hand_enumerated()
        with pytest.raises(AssertionError):
            test_power_spectrum_single_cosine_closed_form((8, 8, 8), (1, 2, 3), 4)
    monkeypatch.setattr(O, "shell_index", good_shell)

    good_ps = O.power_spectrum

    def no_mean_division(x, mean=None):   # x - mean without the division by the mean
        x = np.asarray(x, dtype=np.float64)
        m = float(np.mean(x)) if mean is None else mean
        X = O.dft(x - m)
        return np.bincount(O.shell_index(x.shape).reshape(-1), weights=(np.abs(X) ** 2).reshape(-1))

    monkeypatch.setattr(O, "power_spectrum", no_mean_division)
    with pytest.raises(AssertionError):
        test_power_spectrum_single_cosine_closed_form((8, 8, 8), (1, 2, 3), 4)
    monkeypatch.setattr(O, "power_spectrum", good_ps)

    good_bounds = O.power_spectrum_bounds

    def half_root(x, rho):              # a root too small by 2x
        a, b = good_bounds(x, rho)
        return 0.5 * a, 0.5 * b

    def disc_root(x, rho):              # the disc reading |delta| <= d instead of the box corner
        x = np.asarray(x, dtype=np.float64)
        xbar = float(np.mean(x))
        Xp = O.dft((x - xbar) / xbar)
        s = O.shell_index(x.shape).reshape(-1)
        P = np.bincount(s, weights=(np.abs(Xp) ** 2).reshape(-1))
        A = np.bincount(s, weights=np.abs(Xp).reshape(-1))
        n = np.bincount(s).astype(np.float64)
        d = (-2.0 * A + np.sqrt(4.0 * A * A + 4.0 * n * rho * P)) / (2.0 * np.maximum(n, 1.0))
        d[0] = d[1:][n[1:] > 0].min()
        bnd = (abs(xbar) * d[s]).reshape(x.shape)
        return bnd, bnd.copy()

    for bad in (half_root, disc_root):
        monkeypatch.setattr(O, "power_spectrum_bounds", bad)
        with pytest.raises(AssertionError):
            test_power_spectrum_bounds_are_tight_on_aligned_corners((8, 8, 8), 3, 1e-2)
    monkeypatch.setattr(O, "power_spectrum_bounds", good_bounds)
