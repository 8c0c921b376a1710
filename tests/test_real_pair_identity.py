"""The identity behind the certification of even-length 1D items (Sec. III
DFT, Eq. 1): for real x of even length N and z_n = x_2n + i x_2n+1,
Z = DFT_{N/2}(z), the spectrum of x is, for k <= N/2,

    X_k = (A - i W_N^k B) / 2,  A = Z_k + conj Z_{N/2-k},  B = Z_k - conj Z_{N/2-k}

(indices mod N/2, W_N = exp(-2 pi i / N)).  Checked against the plain DFT
by brute force and against the library FFT, with planted mistakes in the
formula that must fail.
"""
import numpy as np
import pytest


def via_pairs(x, sign=-1.0, conj_b=True):
    N = x.size
    H = N // 2
    z = x[0::2] + 1j * x[1::2]
    Z = np.fft.fft(z)
    k = np.arange(H + 1)
    zk, zm = Z[k % H], Z[(H - k) % H]
    A = zk + np.conj(zm)
    B = zk - (np.conj(zm) if conj_b else zm)
    W = np.exp(sign * 2j * np.pi * k / N)
    return (A - 1j * W * B) / 2


def brute(x):
    N = x.size
    n = np.arange(N)
    k = np.arange(N // 2 + 1)[:, None]
    return (x[None, :] * np.exp(-2j * np.pi * k * n / N)).sum(axis=1)


@pytest.mark.parametrize("N", [2, 4, 6, 10, 16, 64, 250])
def test_identity_matches_brute_force(N):
    x = np.random.default_rng(N).standard_normal(N)
    np.testing.assert_allclose(via_pairs(x), brute(x), rtol=0, atol=1e-10 * max(1.0, np.abs(x).sum()))


def test_identity_matches_library_fft_at_size():
    x = np.random.default_rng(1).standard_normal(31000)
    np.testing.assert_allclose(via_pairs(x), np.fft.rfft(x), rtol=0, atol=1e-9 * np.abs(x).sum())


@pytest.mark.parametrize("wrong", [{"sign": +1.0}, {"conj_b": False}])
def test_planted_mistakes_fail(wrong):
    x = np.random.default_rng(2).standard_normal(64)
    assert np.max(np.abs(via_pairs(x, **wrong) - brute(x))) > 1e-3
