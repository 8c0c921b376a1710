"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each pin is independent of the oracle's own code: brute-force sums, dense
cos/sin bases built here, closed forms, invariants of the projections.  The
last tests plant mistakes in the oracle (on the CPU) and check that a pin
catches each of them.
"""
import itertools

import numpy as np
import pytest

from oracle import ffcz_oracle as O
from paper_2601_01596_b300 import workloads as W


# ---------------------------------------------------------------- transforms
def brute_dft(x):
    """O(N^2) DFT straight from Eq. 1 / its nD analogue (no FFT)."""
    x = np.asarray(x, dtype=np.float64)
    shape = x.shape
    out = np.zeros(shape, dtype=np.complex128)
    idx = list(itertools.product(*[range(n) for n in shape]))
    for k in idx:
        s = 0.0 + 0.0j
        for n in idx:
            ph = sum(kk * nn / N for kk, nn, N in zip(k, n, shape))
            s += x[n] * np.exp(-2j * np.pi * ph)
        out[k] = s
    return out


@pytest.mark.parametrize("n", list(range(1, 17)) + [61])
def test_dft_matches_bruteforce_1d(n):
    x = np.random.default_rng(n).standard_normal(n)
    np.testing.assert_allclose(O.dft(x), brute_dft(x), rtol=0, atol=1e-11 * n)


@pytest.mark.parametrize("shape", [(6, 10), (4, 6, 8), (3, 5, 7)])
def test_dft_matches_bruteforce_nd(shape):
    x = np.random.default_rng(1).standard_normal(shape)
    np.testing.assert_allclose(O.dft(x), brute_dft(x), rtol=0, atol=1e-10)


@pytest.mark.parametrize("shape", [(64,), (12, 20), (8, 6, 10)])
def test_parseval_and_inverse(shape):
    # Parseval (Sec. V-A): sum |delta|^2 = N sum |e|^2; idft inverts dft.
    e = np.random.default_rng(2).standard_normal(shape)
    d = O.dft(e)
    N = e.size
    assert np.isclose(np.sum(np.abs(d) ** 2), N * np.sum(e ** 2), rtol=1e-12)
    np.testing.assert_allclose(O.idft(d), e, atol=1e-13)


def test_impulse_and_cosine():
    N = 24
    imp = np.zeros(N); imp[0] = 1.0
    np.testing.assert_allclose(O.dft(imp), np.ones(N), atol=1e-14)
    k0 = 5
    c = np.cos(2 * np.pi * k0 * np.arange(N) / N)
    d = O.dft(c)
    want = np.zeros(N, complex); want[k0] = want[N - k0] = N / 2
    np.testing.assert_allclose(d, want, atol=1e-12)


def test_linearity():
    r = np.random.default_rng(3)
    a, b = r.standard_normal((2, 6, 8))
    np.testing.assert_allclose(O.dft(2.5 * a - b), 2.5 * O.dft(a) - O.dft(b), atol=1e-12)


# --------------------------------------------------------------- projections
def test_projections_are_projections():
    r = np.random.default_rng(4)
    d = r.standard_normal(50) + 1j * r.standard_normal(50)
    D = 0.7
    p = O.project_f(d, D)
    assert np.all(np.abs(p.real) <= D) and np.all(np.abs(p.imag) <= D)
    np.testing.assert_array_equal(O.project_f(p, D), p)           # idempotent
    inside = 0.5 * D * (np.tanh(d.real) + 1j * np.tanh(d.imag))
    np.testing.assert_array_equal(O.project_f(inside, D), inside)  # identity inside
    d2 = r.standard_normal(50) + 1j * r.standard_normal(50)
    assert np.linalg.norm(O.project_f(d, D) - O.project_f(d2, D)) <= np.linalg.norm(d - d2)
    e = r.standard_normal(40)
    q = O.project_s(e, 0.3)
    assert np.max(np.abs(q)) <= 0.3
    np.testing.assert_array_equal(O.project_s(q, 0.3), q)
    # Euclidean projection onto a box: no box point is closer.
    for _ in range(200):
        z = r.uniform(-0.3, 0.3, 40)
        assert np.linalg.norm(e - q) <= np.linalg.norm(e - z) + 1e-15


# -------------------------------------------------------------- closed forms
@pytest.mark.parametrize("shape,k0", [((64,), (5,)), ((16, 32), (3, 7)),
                                      ((8, 16, 16), (1, 2, 3))])
def test_single_mode_closed_form(shape, k0):
    """e0 = A cos(2 pi k0.n/N): one iteration, e* = (2 D'/N) cos(2 pi k0.n/N)."""
    N = int(np.prod(shape))
    E = 1.0
    A = 0.5
    D = 0.1 * A * N / 2
    e0 = W.single_mode(shape, k0, A)
    r = O.correct(e0, E, D)
    Es, Ds, _ = O.thresholds(E, D, O.ETA_DEFAULT)
    assert r.status == O.OK and r.iters == 1 and not r.preclipped
    np.testing.assert_allclose(r.e, W.single_mode(shape, k0, 2 * Ds / N), atol=1e-14)


def test_single_mode_self_conjugate():
    """k0 = N/2 is its own mirror: amplitude factor N instead of N/2."""
    N = 32
    e0 = W.single_mode((N,), (N // 2,), 0.5)
    D = 0.25 * 0.5 * N
    r = O.correct(e0, 1.0, D)
    Ds = D * (1 - O.ETA_DEFAULT)
    assert r.iters == 1
    np.testing.assert_allclose(r.e, W.single_mode((N,), (N // 2,), Ds / N), atol=1e-14)


@pytest.mark.parametrize("shape", [(17,), (6, 10), (4, 6, 8)])
def test_spike_closed_form(shape):
    """e0 = E' at n = 0: every delta_k = E' (real), clipped to D', e* = D' 1_{n=0}."""
    E, D = 1.0, 0.5
    Es, Ds, _ = O.thresholds(E, D, O.ETA_DEFAULT)
    e0 = np.zeros(shape); e0.flat[0] = Es
    r = O.correct(e0, E, D)
    want = np.zeros(shape); want.flat[0] = Ds
    assert r.iters == 1
    np.testing.assert_allclose(r.e, want, atol=1e-15)


def test_zero_iterations_bit_identical():
    e0 = np.zeros((8, 8, 8))
    r = O.correct(e0, 1.0, 1.0)
    assert r.iters == 0 and np.array_equal(r.e, e0)
    it = W.grf_field(n=16, seed=3)
    e0 = it["e0"].astype(np.float64)
    r = O.correct(e0, it["E"], it["D"])
    assert r.iters == 0 and np.array_equal(r.e, e0)


def test_preclip_reading_A3():
    e0 = np.array([0.5, -2.0, 0.1, 1.0])
    r = O.correct(e0, 1.0, 100.0)
    Es = 1.0 - O.ETA_DEFAULT
    assert r.preclipped and r.iters == 0
    np.testing.assert_array_equal(r.e, [0.5, -Es, 0.1, Es])


# ----------------------------------------- dense-basis POCS (no FFT anywhere)
def dense_basis(shape):
    """Distinct real cos/sin basis vectors of the DFT (Sec. IV-A)."""
    idx = list(itertools.product(*[range(n) for n in shape]))
    grid = np.array(idx, dtype=np.float64)
    seen, vecs = set(), []
    for k in idx:
        mk = tuple((-kk) % n for kk, n in zip(k, shape))
        if mk in seen:
            continue
        seen.add(k)
        ph = 2 * np.pi * sum(grid[:, i] * k[i] / shape[i] for i in range(len(shape)))
        vecs.append(np.cos(ph))
        if mk != k:
            vecs.append(np.sin(ph))
    B = np.array(vecs)
    return B, np.sum(B * B, axis=1)


def dense_pocs(e0, E, D, eta=O.ETA_DEFAULT, max_iters=1000):
    shape = e0.shape
    B, nrm = dense_basis(shape)
    Es, Ds, thr = E * (1 - eta), D * (1 - eta), D * (1 - eta / 2)
    e = e0.reshape(-1).astype(np.float64).copy()
    traj = []
    for t in range(max_iters + 1):
        c = B @ e
        if np.max(np.abs(c)) <= thr:
            return e.reshape(shape), t, traj
        cc = np.clip(c, -Ds, Ds)
        e = e + ((cc - c) / nrm) @ B
        e = np.clip(e, -Es, Es)
        traj.append(e.reshape(shape).copy())
    raise AssertionError("dense POCS did not converge")


@pytest.mark.parametrize("shape,seed", [((8,), 0), ((12,), 1), ((16,), 2),
                                        ((4, 4), 3), ((4, 6), 4), ((2, 4, 4), 5)])
def test_oracle_trajectory_matches_dense_pocs(shape, seed):
    r = np.random.default_rng(seed)
    E = 1.0
    e0 = r.uniform(-E, E, shape)
    D = 0.3 * O.f_violation(O.dft(e0))
    e_d, t_d, tr_d = dense_pocs(e0, E, D)
    res = O.correct(e0, E, D, record=True)
    assert t_d >= 1
    assert res.iters == t_d
    for a, b in zip(res.trajectory, tr_d):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)
    np.testing.assert_allclose(res.e, e_d, atol=1e-12)


# ---------------------------------------------------------------- invariants
def _stress(shape, seed, frac=0.5):
    e0 = W.bimodal_error(shape, seed)
    return e0, 1.0, frac * O.f_violation(O.dft(e0))


def test_fejer_monotone():
    e0, E, D = _stress((16, 16), 7)
    res = O.correct(e0, E, D, record=True)
    assert res.iters >= 3
    for z in (np.zeros_like(e0), res.e):
        prev = np.linalg.norm(e0 - z)
        for e in res.trajectory:
            cur = np.linalg.norm(e - z)
            assert cur <= prev + 1e-12
            prev = cur


def test_negation_and_pow2_scaling():
    e0, E, D = _stress((8, 12), 8)
    a = O.correct(e0, E, D, record=True)
    b = O.correct(-e0, E, D, record=True)
    assert a.iters == b.iters
    np.testing.assert_allclose(b.e, -a.e, atol=1e-13)
    c = O.correct(8.0 * e0, 8.0 * E, 8.0 * D)
    assert c.iters == a.iters
    np.testing.assert_array_equal(c.e, 8.0 * a.e)      # exact in binary FP


def test_index_reversal_and_axis_permutation():
    e0, E, D = _stress((8, 8, 8), 9)
    a = O.correct(e0, E, D)
    rev = e0[(-np.arange(8)) % 8][:, (-np.arange(8)) % 8][:, :, (-np.arange(8)) % 8]
    b = O.correct(rev, E, D)
    assert a.iters == b.iters
    back = b.e[(-np.arange(8)) % 8][:, (-np.arange(8)) % 8][:, :, (-np.arange(8)) % 8]
    np.testing.assert_allclose(back, a.e, atol=1e-13)
    c = O.correct(np.transpose(e0, (2, 0, 1)), E, D)
    assert c.iters == a.iters
    np.testing.assert_allclose(np.transpose(c.e, (1, 2, 0)), a.e, atol=1e-13)


def test_iteration_cap_and_nonfinite():
    e0, E, D = _stress((16,), 9, frac=0.6)
    assert O.correct(e0, E, D).iters > 2
    r = O.correct(e0, E, D, max_iters=2)
    assert r.status == O.NOT_CONVERGED and r.iters == 2
    bad = e0.copy(); bad[3] = np.nan
    assert O.correct(bad, E, D).status == O.NONFINITE


def test_min_iters_forces_iterations():
    e0 = np.zeros(16)
    r = O.correct(e0, 1.0, 1.0, min_iters=4)
    assert r.iters == 4 and np.array_equal(r.e, e0)


# ------------------------------------------------------------- certification
def test_certification_pass_fail():
    e0, E, D = _stress((8, 8), 11)
    r = O.correct(e0, E, D)
    ok, s, v = O.certify(r.e, E, D)
    assert ok and s <= E and v <= D
    ok0, _, v0 = O.certify(e0, E, 0.5 * O.f_violation(O.dft(e0)))
    assert not ok0


# ------------------------------------------------------------------- adjoint
def _fd_jvp(e0, v, E, D, K, h):
    fp, _, mp = O.forward_masks(e0 + h * v, E, D, K)
    fm, _, mm = O.forward_masks(e0 - h * v, E, D, K)
    same = all(np.array_equal(a, b) for x, y in zip(mp, mm) for a, b in zip(x, y))
    return (fp - fm) / (2 * h), same


@pytest.mark.parametrize("shape,K", [((16,), 4), ((6, 8), 3), ((4, 4, 4), 5)])
def test_adjoint_dot_product(shape, K):
    """<J v, w> = <v, J^T w>, J v by central differences (F is piecewise affine)."""
    e0, E, D = _stress(shape, 12)
    r = np.random.default_rng(13)
    v = r.standard_normal(shape)
    w = r.standard_normal(shape)
    jv, same = _fd_jvp(e0, v, E, D, K, 1e-7)
    assert same
    jtw = O.correct_backward(e0, w, E, D, K)
    assert np.isclose(np.sum(jv * w), np.sum(v * jtw), rtol=1e-6, atol=1e-9)


def test_adjoint_full_jacobian_tiny():
    shape, K = (8,), 3
    e0, E, D = _stress(shape, 14)
    N = 8
    J = np.zeros((N, N))
    for i in range(N):
        v = np.zeros(N); v[i] = 1.0
        J[:, i], same = _fd_jvp(e0, v, E, D, K, 1e-7)
        assert same
    w = np.random.default_rng(15).standard_normal(N)
    np.testing.assert_allclose(O.correct_backward(e0, w, E, D, K), J.T @ w, atol=1e-6)


def test_adjoint_with_preclip():
    e0 = np.array([0.2, -1.5, 0.7, 1.2, -0.1, 0.0, 0.4, -0.9])
    E = 1.0
    D = 0.3 * O.f_violation(O.dft(np.clip(e0, -1, 1)))
    w = np.random.default_rng(16).standard_normal(8)
    g = O.correct_backward(e0, w, E, D, 2)
    assert g[1] == 0.0 and g[3] == 0.0          # clipped inputs get no gradient


# ------------------------------------------------------ planted oracle errors
def test_pins_catch_planted_mistakes(monkeypatch):
    """A plausible slip anywhere in the oracle must fail one of the pins."""
    x = np.random.default_rng(17).standard_normal((4, 6))
    good = O.dft(x)
    # (1) wrong sign in the exponent -> brute-force pin fails
    monkeypatch.setattr(O, "dft", lambda e: np.conj(good) if e is x else None)
    assert not np.allclose(O.dft(x), brute_dft(x), atol=1e-10)
    monkeypatch.undo()
    # (2) disc projection instead of the Re/Im box -> dense POCS pin fails
    def disc(delta, D):
        m = np.abs(delta)
        s = np.where(m > D, D / np.maximum(m, 1e-300), 1.0)
        return delta * s
    e0 = np.random.default_rng(1).uniform(-1, 1, (12,))
    D = 0.3 * O.f_violation(O.dft(e0))
    want, t_d, _ = dense_pocs(e0, 1.0, D)
    monkeypatch.setattr(O, "project_f", disc)
    got = O.correct(e0, 1.0, D)
    assert got.iters != t_d or not np.allclose(got.e, want, atol=1e-12)
    monkeypatch.undo()
    # (3) missing 1/N in the inverse -> closed form 1 fails
    monkeypatch.setattr(O, "idft", lambda d: np.fft.ifftn(d).real * d.size)
    e1 = W.single_mode((64,), (5,), 0.5)
    got = O.correct(e1, 1.0, 0.1 * 0.5 * 32, max_iters=3)
    Ds = 0.1 * 0.5 * 32 * (1 - O.ETA_DEFAULT)
    assert not np.allclose(got.e, W.single_mode((64,), (5,), 2 * Ds / 64), atol=1e-12)


# --------------------------------------------- edits (Alg. 1, Sec. IV-B/C)
def _mirror(F):
    """F at -k for every k (index reversal modulo each axis length)."""
    idx = np.ix_(*[(-np.arange(n)) % n for n in F.shape])
    return F[idx]


@pytest.mark.parametrize("shape,seed", [((16, 16), 31), ((8, 16, 16), 32), ((61,), 33), ((6, 10), 34)])
def test_edits_sum_to_total_displacement(shape, seed):
    """eps* - eps0 = spatial edits + IDFT(frequency edits), and F Hermitian."""
    e0, E, D = _stress(shape, seed, 0.4)
    r = O.correct(e0, E, D, edits=True)
    assert r.iters >= 2
    idft_F = np.fft.ifftn(r.freq_edits)                    # numpy, not the oracle's scipy call
    np.testing.assert_allclose(r.e - e0, r.spat_edits + idft_F.real, rtol=0, atol=1e-12)
    assert np.max(np.abs(idft_F.imag)) < 1e-12
    np.testing.assert_allclose(_mirror(r.freq_edits), np.conj(r.freq_edits), rtol=0, atol=1e-12)
    assert np.count_nonzero(r.spat_edits) > 0 and np.count_nonzero(r.freq_edits) > 0


@pytest.mark.parametrize("shape,k0", [((64,), (5,)), ((8, 16, 16), (1, 2, 3))])
def test_edits_single_mode_closed_form(shape, k0):
    """One f-clip: delta(+-k0) = A N / 2 clipped to D' gives F(+-k0) = D' - A N/2,
    zero elsewhere, and no spatial edit."""
    N = int(np.prod(shape))
    A, E = 0.5, 1.0
    D = 0.1 * A * N / 2
    r = O.correct(W.single_mode(shape, k0, A), E, D, edits=True)
    Ds = D * (1 - O.ETA_DEFAULT)
    want = np.zeros(shape, dtype=complex)
    want[tuple(k0)] = Ds - A * N / 2
    want[tuple((-k) % n for k, n in zip(k0, shape))] = Ds - A * N / 2
    assert r.iters == 1
    np.testing.assert_allclose(r.freq_edits, want, rtol=0, atol=1e-10)
    assert not r.spat_edits.any()


@pytest.mark.parametrize("shape", [(17,), (4, 6, 8)])
def test_edits_spike_closed_form(shape):
    """e0 = E' at n = 0: every bin E' clipped to D', so F_k = D' - E' for all k."""
    E, D = 1.0, 0.5
    Es, Ds, _ = O.thresholds(E, D, O.ETA_DEFAULT)
    e0 = np.zeros(shape); e0.flat[0] = Es
    r = O.correct(e0, E, D, edits=True)
    np.testing.assert_allclose(r.freq_edits, np.full(shape, Ds - Es), rtol=0, atol=1e-14)
    assert not r.spat_edits.any()


def test_edits_preclip_is_a_spatial_edit():
    e0, E, D = _stress((8, 8), 35, 0.5)
    e0 = e0.copy(); e0[2, 3] = 1.5; e0[5, 1] = -3.0
    r = O.correct(e0, E, D, edits=True)
    assert r.preclipped
    np.testing.assert_allclose(r.e - e0, r.spat_edits + np.fft.ifftn(r.freq_edits).real, atol=1e-12)


def dense_pocs_edits(e0, E, D, eta=O.ETA_DEFAULT, max_iters=1000):
    """The dense cos/sin-coordinate POCS above, accumulating its own edits: a
    coordinate move dc of the cos row of bin k changes Re delta_k by dc and
    Re delta_-k by dc; of the sin row, Im delta_k by -dc and Im delta_-k by +dc
    (delta_k = sum e_n (cos - i sin))."""
    shape = e0.shape
    idx = list(itertools.product(*[range(n) for n in shape]))
    grid = np.array(idx, dtype=np.float64)
    rows, seen = [], set()
    for k in idx:
        mk = tuple((-kk) % n for kk, n in zip(k, shape))
        if mk in seen:
            continue
        seen.add(k)
        ph = 2 * np.pi * sum(grid[:, i] * k[i] / shape[i] for i in range(len(shape)))
        rows.append((np.cos(ph), k, mk, "c"))
        if mk != k:
            rows.append((np.sin(ph), k, mk, "s"))
    B = np.array([r[0] for r in rows])
    nrm = np.sum(B * B, axis=1)
    Es, Ds, thr = E * (1 - eta), D * (1 - eta), D * (1 - eta / 2)
    e = e0.reshape(-1).astype(np.float64).copy()
    S = np.zeros_like(e)
    F = np.zeros(shape, dtype=complex)
    for _ in range(max_iters + 1):
        c = B @ e
        if np.max(np.abs(c)) <= thr:
            return e.reshape(shape), S.reshape(shape), F
        cc = np.clip(c, -Ds, Ds)
        for (_, k, mk, kind), dc in zip(rows, cc - c):
            if dc == 0:
                continue
            if kind == "c":
                F[k] += dc
                if mk != k:
                    F[mk] += dc
            else:
                F[k] += -1j * dc
                F[mk] += 1j * dc
        ei = e + ((cc - c) / nrm) @ B
        e = np.clip(ei, -Es, Es)
        S += e - ei
    raise AssertionError("dense POCS did not converge")


@pytest.mark.parametrize("shape,seed", [((12,), 36), ((4, 6), 37), ((2, 4, 4), 38)])
def test_edits_match_dense_coordinate_pocs(shape, seed):
    r0 = np.random.default_rng(seed)
    E = 1.0
    e0 = r0.uniform(-E, E, shape)
    D = 0.3 * O.f_violation(O.dft(e0))
    e_d, S_d, F_d = dense_pocs_edits(e0, E, D)
    r = O.correct(e0, E, D, edits=True)
    np.testing.assert_allclose(r.e, e_d, atol=1e-12)
    np.testing.assert_allclose(r.spat_edits, S_d, atol=1e-12)
    np.testing.assert_allclose(r.freq_edits, F_d, atol=1e-12)


def test_compaction_quantization_and_application():
    """CompactEdits round trip, code error <= q/2, and the decompression side:
    x_hat + S + IFFT(F) from the stored half spectrum gives x + eps*."""
    shape = (8, 16, 16)
    e0, E, D = _stress(shape, 39, 0.4)
    r = O.correct(e0, E, D, edits=True)
    Fh = O.half_spectrum(r.freq_edits)
    assert Fh.shape == (8, 16, 9)
    for vals, bound in ((r.spat_edits, E), (Fh, D)):
        flags, comp = O.compact_edits(vals)
        n = vals.size
        assert flags.size == (n + 7) // 8
        assert int(np.unpackbits(flags, bitorder="little")[:n].sum()) == comp.size
        np.testing.assert_array_equal(O.expand_edits(flags, comp, n), vals.reshape(-1))
        codes = O.quantize_edits(comp, bound)
        back = O.dequantize_edits(codes, bound, complex_pairs=np.iscomplexobj(comp))
        q = 2 * bound / 2 ** 16
        err = back - comp
        assert max(np.max(np.abs(err.real)), np.max(np.abs(np.imag(err)))) <= q / 2 + 1e-18
    # bit order: component 0 in the least significant bit of byte 0
    f, _ = O.compact_edits(np.array([1.0, 0, 0, 0, 0, 0, 0, 0, 0, 2.0]))
    assert list(f) == [1, 2]
    # x_hat = x + e0; applying the exact edits reproduces x + eps*
    x = np.random.default_rng(40).standard_normal(shape)
    out = O.apply_edits(x + e0, r.spat_edits, Fh)
    np.testing.assert_allclose(out, x + r.e, rtol=0, atol=1e-12)
    # float32 decisions: the same codes from numpy float32 arithmetic
    v32 = r.spat_edits[r.spat_edits != 0].astype(np.float32)
    q32 = np.float32(E) * np.float32(2.0 ** -15)
    np.testing.assert_array_equal(O.quantize_edits(v32, E, dtype=np.float32),
                                  np.rint(v32 / q32).astype(np.int64))


def test_edit_pin_catches_recording_the_stopping_clip():
    """Planted mistake: also recording the f-clip of the check that stops the
    loop (Alg. 1 breaks before ProjectOntoFCube) breaks the displacement pin."""
    e0, E, D = _stress((16, 16), 41, 0.4)
    r = O.correct(e0, E, D, edits=True)
    Ds = D * (1 - O.ETA_DEFAULT)
    delta = O.dft(r.e)
    F_bad = r.freq_edits + (O.project_f(delta, Ds) - delta)
    assert np.max(np.abs(O.project_f(delta, Ds) - delta)) > 0
    bad = r.spat_edits + np.fft.ifftn(F_bad).real
    assert np.max(np.abs(r.e - e0 - bad)) > 1e-12


# ------------------------------------------ pointwise bounds (footnote, Sec. IV-A)
def test_pointwise_uniform_bounds_equal_scalar_bounds():
    for shape, seed in (((16, 16, 16), 42), ((32, 48), 43)):
        e0, E, D = _stress(shape, seed, 0.4)
        a = O.correct(e0, E, D)
        b = O.correct(e0, np.full(shape, E), (np.full(shape, D), np.full(shape, D)))
        assert a.iters == b.iters >= 2
        np.testing.assert_array_equal(a.e, b.e)


def dense_pocs_pw(e0, E_n, D_re, D_im, eta=O.ETA_DEFAULT, max_iters=2000):
    """The dense cos/sin-coordinate POCS with a bound per coordinate: the cos
    row of bin k carries Delta^Re_k, the sin row Delta^Im_k."""
    shape = e0.shape
    idx = list(itertools.product(*[range(n) for n in shape]))
    grid = np.array(idx, dtype=np.float64)
    rows, bnd, seen = [], [], set()
    for k in idx:
        mk = tuple((-kk) % n for kk, n in zip(k, shape))
        if mk in seen:
            continue
        seen.add(k)
        ph = 2 * np.pi * sum(grid[:, i] * k[i] / shape[i] for i in range(len(shape)))
        rows.append(np.cos(ph)); bnd.append(D_re[k])
        if mk != k:
            rows.append(np.sin(ph)); bnd.append(D_im[k])
    B, bnd = np.array(rows), np.array(bnd)
    nrm = np.sum(B * B, axis=1)
    Es = E_n.reshape(-1) * (1 - eta)
    e = e0.reshape(-1).astype(np.float64).copy()
    for t in range(max_iters + 1):
        c = B @ e
        if np.max(np.abs(c) / bnd) <= 1 - eta / 2:
            return e.reshape(shape), t
        cc = np.clip(c, -bnd * (1 - eta), bnd * (1 - eta))
        e = np.clip(e + ((cc - c) / nrm) @ B, -Es, Es)
    raise AssertionError("dense POCS did not converge")


@pytest.mark.parametrize("shape,seed", [((12,), 44), ((4, 6), 45), ((2, 4, 4), 46)])
def test_pointwise_trajectory_matches_dense_coordinate_pocs(shape, seed):
    r = np.random.default_rng(seed)
    e0 = r.uniform(-1, 1, shape)
    E_n = r.uniform(0.6, 1.4, shape)
    e0 = np.clip(e0, -E_n * 0.9, E_n * 0.9)
    v = np.abs(O.dft(e0))
    base = r.uniform(0.2, 0.5, shape)
    base = 0.5 * (base + base[np.ix_(*[(-np.arange(n)) % n for n in shape])])   # even in k
    D_re = base * np.max(v)
    D_im = base[::-1].copy() if len(shape) == 1 else base * np.max(v) * 1.1
    if len(shape) == 1:
        D_im = 0.5 * (D_im + D_im[(-np.arange(shape[0])) % shape[0]]) * np.max(v)
    e_d, t_d = dense_pocs_pw(e0, E_n, D_re, D_im)
    res = O.correct(e0, E_n, (D_re, D_im))
    assert t_d >= 1 and res.iters == t_d
    np.testing.assert_allclose(res.e, e_d, atol=1e-12)


def test_pointwise_single_mode_closed_form():
    """Only the bins +-k0 are bounded tightly: one iteration, the mode is
    scaled to the shrunk bin bound, every other bin is untouched."""
    shape, k0 = (16, 32), (3, 5)
    N = int(np.prod(shape))
    A = 0.5
    e0 = W.single_mode(shape, k0, A)
    D_re = np.full(shape, 10.0 * A * N)
    d = 0.1 * A * N / 2
    D_re[k0] = d
    D_re[tuple((-k) % n for k, n in zip(k0, shape))] = d
    r = O.correct(e0, np.full(shape, 1.0), (D_re, D_re.copy()))
    assert r.iters == 1
    np.testing.assert_allclose(r.e, W.single_mode(shape, k0, 2 * d * (1 - O.ETA_DEFAULT) / N), atol=1e-14)


def test_pointwise_certification():
    e0, E, D = _stress((16, 16), 47, 0.4)
    E_n = np.full(e0.shape, E)
    Db = (np.full(e0.shape, D), np.full(e0.shape, D))
    r = O.correct(e0, E_n, Db)
    ok, s, v = O.certify(r.e, E_n, Db)
    assert ok and s <= 1 and v <= 1
    E_n2 = E_n.copy(); E_n2[0, 0] = 0.5 * abs(r.e[0, 0]) + 1e-12
    assert not O.certify(r.e, E_n2, Db)[0]


def test_power_spectrum_bounds_guarantee():
    """Any error inside the pointwise f-cube built for relative bound rho keeps
    every power-spectrum shell (the zero-frequency one excepted) within rho,
    P measured with the original field's mean (reading A24)."""
    it = W.grf_field(16)
    x = it["x"].astype(np.float64) + 3.0          # positive mean
    rho = 1e-2
    D_re, D_im = O.power_spectrum_bounds(x, rho)
    np.testing.assert_array_equal(D_re, D_re[np.ix_(*[(-np.arange(n)) % n for n in x.shape])])
    P = O.power_spectrum(x)
    shells = O.shell_index(x.shape)
    r = np.random.default_rng(48)
    worst = 0.0
    for trial in range(20):
        # a real error whose spectrum sits on (or inside) the box: project hard
        e = r.standard_normal(x.shape) * 10
        delta = O.project_f_pw(O.dft(e), D_re, D_im)
        e = O.idft(delta)
        Ph = O.power_spectrum(x + e, mean=float(np.mean(x)))
        rel = np.abs(Ph[1:] - P[1:]) / P[1:]
        worst = max(worst, float(np.max(rel)))
        assert np.all(rel <= rho * (1 + 1e-9))
    assert worst > 0.1 * rho       # the bound is not vacuous
    assert shells[0, 0, 0] == 0 and D_re[0, 0, 0] == D_re[shells >= 1].min()
