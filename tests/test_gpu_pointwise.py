"""Pointwise bounds (E_n, Delta_k^Re, Delta_k^Im; ffcz_correct_pw) vs the oracle.

Bars as for scalar bounds: max|delta e| <= 1e-3 min(E_n) against the FP64
oracle run with the same pointwise bounds, iteration count within +-2, and
the FP64 certification on the GPU passes.
"""
import numpy as np
import pytest

from oracle import ffcz_oracle as O
from paper_2601_01596_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _even(a):
    return 0.5 * (a + a[np.ix_(*[(-np.arange(n)) % n for n in a.shape])])


def run_pw(e0, E_n, D_re, D_im, **opts):
    import torch
    import paper_2601_01596_b300 as ffcz
    shape = e0.shape
    plan = ffcz.Plan([shape], pointwise=1, **opts)
    half = O.half_spectrum(D_re + 1j * D_im).astype(np.complex64)
    t = torch.from_numpy(e0.reshape(-1).astype(np.float32).copy()).cuda()
    eb = torch.from_numpy(E_n.reshape(-1).astype(np.float32)).cuda()
    db = torch.from_numpy(half.reshape(-1)).cuda()
    st = plan.correct_pw(t, eb, db)
    return t.cpu().numpy().reshape(shape), st


@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 128), (16, 32, 64)])
def test_uniform_pointwise_bounds_behave_like_scalar(shape):
    import torch
    import paper_2601_01596_b300 as ffcz
    e0 = W.bimodal_error(shape, 90, E=1.0, dtype=np.float32)
    E, D = 1.0, 0.4 * O.f_violation(O.dft(e0.astype(np.float64)))
    e_pw, st = run_pw(e0, np.full(shape, E), np.full(shape, D), np.full(shape, D))
    plan = ffcz.Plan([shape])
    t = torch.from_numpy(e0.reshape(-1).copy()).cuda()
    st_s = plan.correct(t, [E], [D])
    assert abs(st[0]["iters"] - st_s[0]["iters"]) <= 1 and st[0]["certified"] == 1
    np.testing.assert_allclose(e_pw.reshape(-1), t.cpu().numpy(), rtol=0, atol=1e-4 * E)


@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 128), (16, 32, 64)])
def test_varying_pointwise_bounds_match_oracle(shape):
    r = np.random.default_rng(91)
    x = W.grf_field(shape[0], seed=3)["x"] if len(shape) == 3 and len(set(shape)) == 1 else \
        r.standard_normal(shape)
    x = x.astype(np.float64) + 4.0
    E_n = 0.01 * (0.6 + 0.8 * r.random(shape))
    e0 = (r.uniform(-1, 1, shape) * E_n * 0.999).astype(np.float32)
    D_re, D_im = O.power_spectrum_bounds(x, 2e-2)
    # keep the f-clip active: tighten toward the error's own spectrum
    scale = 0.3 * O.f_ratio_pw(O.dft(e0.astype(np.float64)), D_re, D_im)
    D_re, D_im = D_re * scale, D_im * scale
    ref = O.correct(e0, E_n, (D_re, D_im))
    e, st = run_pw(e0, E_n, D_re, D_im)
    assert ref.iters >= 2
    assert abs(st[0]["iters"] - ref.iters) <= 2
    assert st[0]["status"] == 0 and st[0]["certified"] == 1
    np.testing.assert_allclose(e, ref.e, rtol=0, atol=1e-3 * E_n.min())
    ok, s, v = O.certify(e.astype(np.float64), E_n, (D_re, D_im))
    assert ok


@pytest.mark.parametrize("k", [1, 3])
def test_pointwise_forced_iterations(k):
    shape = (32, 64)
    r = np.random.default_rng(92)
    E_n = 0.5 + r.random(shape)
    e0 = (r.uniform(-1, 1, shape) * E_n).astype(np.float32)
    base = _even(0.5 + r.random(shape))
    v = O.f_violation(O.dft(e0.astype(np.float64)))
    D_re, D_im = 0.3 * v * base, 0.3 * v * _even(0.5 + r.random(shape))
    ref = O.correct(e0, E_n, (D_re, D_im), min_iters=k, max_iters=k)
    e, st = run_pw(e0, E_n, D_re, D_im, min_iters=k, max_iters=k, certify=0)
    assert st[0]["iters"] == k
    np.testing.assert_allclose(e, ref.e, rtol=0, atol=1e-3 * E_n.min())


def test_invalid_bounds_and_scalar_calls_are_refused():
    import torch
    import paper_2601_01596_b300 as ffcz
    shape = (32, 32)
    e0 = np.zeros(shape, np.float32)
    E_n = np.ones(shape); E_n[3, 4] = 0.0
    with pytest.raises(ffcz.FFCzError):
        run_pw(e0, E_n, np.ones(shape), np.ones(shape))
    # subnormal bounds (below FLT_MIN) are refused too, spatial and frequency
    E_n[3, 4] = 1e-39
    with pytest.raises(ffcz.FFCzError):
        run_pw(e0, E_n, np.ones(shape), np.ones(shape))
    D_im = np.ones(shape); D_im[0, 5] = D_im[0, -5] = 1e-40
    with pytest.raises(ffcz.FFCzError):
        run_pw(e0, np.ones(shape), np.ones(shape), D_im)
    # the smallest and largest normal bounds are accepted
    e, st = run_pw(e0, np.full(shape, np.finfo(np.float32).tiny), np.ones(shape),
                   np.full(shape, np.finfo(np.float32).max))
    assert st[0]["status"] == 0 and st[0]["certified"] == 1 and np.array_equal(e, e0)
    plan = ffcz.Plan([shape], pointwise=1)
    with pytest.raises(ffcz.FFCzError):
        plan.correct(torch.zeros(32 * 32, device="cuda"), [1.0], [1.0])


@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 128), (16, 32, 64), (3000,), (1501,)])
def test_power_spectrum_bounds_match_oracle(shape):
    import torch
    import paper_2601_01596_b300 as ffcz
    r = np.random.default_rng(93)
    x = (r.standard_normal(shape) + 5.0).astype(np.float32)
    rho = 3e-3
    plan = ffcz.Plan([shape])
    got = plan.power_spectrum_bounds(torch.from_numpy(x.reshape(-1).copy()).cuda(), rho).cpu().numpy()
    D_re, D_im = O.power_spectrum_bounds(x.astype(np.float64), rho)
    want = O.half_spectrum(D_re + 1j * D_im).reshape(-1)
    # 1D shells are single bin pairs: the float32 transform's absolute error
    # on the smallest bins is not averaged over a shell
    atol = 0.0 if len(shape) > 1 else 1e-4 * float(np.median(want.real))
    np.testing.assert_allclose(got.real, want.real, rtol=1e-4, atol=atol)
    np.testing.assert_allclose(got.imag, want.imag, rtol=1e-4, atol=atol)


def test_power_spectrum_mode_end_to_end():
    """x_hat = x + e0; bounds from x for rho; after ffcz_correct_pw every
    shell but the zero-frequency one of x_hat' is within rho of x's."""
    import torch
    import paper_2601_01596_b300 as ffcz
    shape = (32, 32, 32)
    it = W.grf_field(32, seed=5)
    x = (it["x"].astype(np.float64) + 6.0).astype(np.float32)
    rng = np.random.default_rng(94)
    E_n = np.full(shape, 0.05)
    e0 = (rng.uniform(-1, 1, shape) * 0.05 * 0.999).astype(np.float32)
    rho = 1e-3
    plan = ffcz.Plan([shape], pointwise=1)
    db = plan.power_spectrum_bounds(torch.from_numpy(x.reshape(-1).copy()).cuda(), rho)
    t = torch.from_numpy(e0.reshape(-1).copy()).cuda()
    st = plan.correct_pw(t, torch.from_numpy(E_n.reshape(-1).astype(np.float32)).cuda(), db)
    assert st[0]["status"] == 0 and st[0]["certified"] == 1 and st[0]["iters"] >= 1
    e = t.cpu().numpy().reshape(shape).astype(np.float64)
    P = O.power_spectrum(x.astype(np.float64))
    P_hat = O.power_spectrum(x.astype(np.float64) + e, mean=float(np.mean(x.astype(np.float64))))
    rel = np.abs(P_hat[1:] - P[1:]) / P[1:]
    assert np.max(rel) <= rho * (1 + 1e-3)
    P_base = O.power_spectrum(x.astype(np.float64) + e0, mean=float(np.mean(x.astype(np.float64))))
    assert np.max(np.abs(P_base[1:] - P[1:]) / P[1:]) > rho     # the base error did violate it


def _pw_case(shape, seed, frac=0.3):
    """Varying E_n and (Delta^Re, Delta^Im) (even in k), the f-clip active."""
    r = np.random.default_rng(seed)
    E_n = 0.5 + r.random(shape)
    e0 = (r.uniform(-1, 1, shape) * E_n).astype(np.float32)
    D_re, D_im = _even(0.5 + r.random(shape)), _even(0.5 + r.random(shape))
    scale = frac * O.f_ratio_pw(O.dft(e0.astype(np.float64)), D_re, D_im)
    return e0, E_n, D_re * scale, D_im * scale


@pytest.mark.parametrize("shape", [(256, 32, 32), (256, 64), (512, 16, 32), (1024, 16, 32)])
def test_tma_fed_pointwise_check_equals_plain_and_matches_oracle(shape, monkeypatch):
    """The persistent check pass stages each tile's f-bounds in shared memory
    by the copy engine; the tiled pass reads them from global memory.  Same
    arithmetic: bit-identical results; and both match the FP64 oracle."""
    e0, E_n, D_re, D_im = _pw_case(shape, 93)
    monkeypatch.setenv("FFCZ_TUNE_FORCE", "axis=tma,px=tma,chk=tma")
    a, sa = run_pw(e0, E_n, D_re, D_im)
    monkeypatch.setenv("FFCZ_TUNE_FORCE", "axis=tma,px=tma,chk=8")
    b, sb = run_pw(e0, E_n, D_re, D_im)
    monkeypatch.delenv("FFCZ_TUNE_FORCE")
    assert sa[0]["iters"] == sb[0]["iters"] >= 2 and sa[0]["certified"] == 1
    assert np.array_equal(a, b)
    ref = O.correct(e0, E_n, (D_re, D_im))
    assert abs(sa[0]["iters"] - ref.iters) <= 2
    same = O.correct(e0, E_n, (D_re, D_im), min_iters=sa[0]["iters"], max_iters=sa[0]["iters"])
    np.testing.assert_allclose(a, same.e, rtol=0, atol=1e-3 * E_n.min())


def test_tma_fed_pointwise_batch_equals_singles(monkeypatch):
    """Every member of a batch has its own map of the packed f-bounds."""
    import torch
    import paper_2601_01596_b300 as ffcz
    monkeypatch.setenv("FFCZ_TUNE_FORCE", "axis=tma,px=tma,chk=tma")
    shapes = [(256, 16, 32), (256, 32, 16), (256, 16, 32)]
    cases = [_pw_case(sh, 100 + i, frac=0.25 + 0.1 * i) for i, sh in enumerate(shapes)]
    plan = ffcz.Plan(shapes, pointwise=1)
    t = torch.from_numpy(np.concatenate([c[0].reshape(-1) for c in cases])).cuda()
    eb = torch.from_numpy(np.concatenate([c[1].reshape(-1) for c in cases]).astype(np.float32)).cuda()
    half = np.concatenate([O.half_spectrum(c[2] + 1j * c[3]).reshape(-1) for c in cases]).astype(np.complex64)
    st = plan.correct_pw(t, eb, torch.from_numpy(half).cuda())
    out = t.cpu().numpy()
    off = 0
    for i, (sh, c) in enumerate(zip(shapes, cases)):
        n = int(np.prod(sh))
        single, s1 = run_pw(*c)
        assert st[i]["iters"] == s1[0]["iters"] >= 2 and st[i]["certified"] == 1, i
        assert np.array_equal(out[off:off + n], single.reshape(-1)), f"item {i}"
        off += n


# ------------------------------------------------------------- 1D items
def _pw1_batch(lengths, seed):
    """1D signals with pointwise bounds: E_n in [0.6, 1.4], Delta_k random on
    the half spectrum k <= N/2 (bin N - k takes the bounds of k), scaled so
    that the f-clip is active."""
    r = np.random.default_rng(seed)
    out = []
    for N in lengths:
        E_n = 0.6 + 0.8 * r.random(N)
        e0 = (r.uniform(-1, 1, N) * E_n * 0.999).astype(np.float32)
        v = O.f_violation(O.dft(e0.astype(np.float64)))
        half_re = 0.3 * v * (0.5 + r.random(N // 2 + 1))
        half_im = 0.3 * v * (0.5 + r.random(N // 2 + 1))
        k = np.arange(N)
        kk = np.minimum(k, N - k)
        out.append((e0, E_n, half_re, half_im, half_re[kk], half_im[kk]))
    return out


def _run_pw1(items, **opts):
    import torch
    import paper_2601_01596_b300 as ffcz
    plan = ffcz.Plan([(it[0].size,) for it in items], pointwise=1, **opts)
    assert plan.edit_layout(-1)[1] == sum(it[0].size // 2 + 1 for it in items)
    t = torch.from_numpy(np.concatenate([it[0] for it in items])).cuda()
    eb = torch.from_numpy(np.concatenate([it[1] for it in items]).astype(np.float32)).cuda()
    db = torch.from_numpy(np.concatenate([(it[2] + 1j * it[3]).astype(np.complex64) for it in items])).cuda()
    st = plan.correct_pw(t, eb, db)
    return t.cpu().numpy(), st


def test_1d_pointwise_bounds_match_oracle():
    """A batch of uneven 1D lengths (several Bluestein splits) with
    pointwise bounds, each item against the oracle run with the same
    bounds (full-spectrum arrays, even in k)."""
    lengths = [700, 1500, 3001, 1500, 9000]
    items = _pw1_batch(lengths, 95)
    out, st = _run_pw1(items)
    off = 0
    for i, (e0, E_n, _, _, D_re, D_im) in enumerate(items):
        N = e0.size
        ref = O.correct(e0, E_n, (D_re, D_im))
        assert ref.iters >= 1
        assert abs(st[i]["iters"] - ref.iters) <= 2 and st[i]["certified"] == 1, (i, st[i])
        np.testing.assert_allclose(out[off:off + N], ref.e, rtol=0, atol=1e-3 * E_n.min())
        assert O.certify(out[off:off + N].astype(np.float64), E_n, (D_re, D_im))[0]
        off += N


@pytest.mark.parametrize("k", [1, 2])
def test_1d_pointwise_forced_iterations(k):
    items = _pw1_batch([2000, 513], 96)
    out, st = _run_pw1(items, min_iters=k, max_iters=k, certify=0)
    off = 0
    for i, (e0, E_n, _, _, D_re, D_im) in enumerate(items):
        ref = O.correct(e0, E_n, (D_re, D_im), min_iters=k, max_iters=k)
        assert st[i]["iters"] == k
        np.testing.assert_allclose(out[off:off + e0.size], ref.e, rtol=0, atol=1e-3 * E_n.min())
        off += e0.size


@pytest.mark.parametrize("shape", [(32, 32, 32), (3000,)])
def test_certification_bound_of_uniform_pointwise_bounds_equals_scalar(shape):
    """Uniform pointwise bounds E_n = E = 100, Delta_k = D certify exactly
    like the scalar bounds: the FP64 rounding bound (and so f_margin64) must
    not depend on the spatial bounds' scale, whose ratio max|e_n|/E_n bounds
    no norm."""
    import torch
    import paper_2601_01596_b300 as ffcz
    N = int(np.prod(shape))
    e0 = W.bimodal_error(shape, 97, E=1.0, dtype=np.float32)
    # feasible as given; D a float32 value, so the complex64 bounds hold it exactly
    E, D = 100.0, float(np.float32(2.0 * O.f_violation(O.dft(e0.astype(np.float64)))))
    plan = ffcz.Plan([shape], pointwise=1, max_iters=0, certify=1)
    t = torch.from_numpy(e0.reshape(-1).copy()).cuda()
    nb = plan.edit_layout(-1)[1]
    eb = torch.full((N,), E, dtype=torch.float32, device="cuda")
    db = torch.full((nb,), D + 1j * D, dtype=torch.complex64, device="cuda")
    spw = plan.correct_pw(t, eb, db)[0]
    ps = ffcz.Plan([shape], max_iters=0, certify=1)
    ts = torch.from_numpy(e0.reshape(-1).copy()).cuda()
    ss = ps.correct(ts, [E], [D])[0]
    assert spw["certified"] == ss["certified"] == 1
    # the rounding bound is about 5e-13 D here; a norm bound taken from the
    # ratio max|e_n|/E_n would shrink it about 75-fold, and one left unscaled
    # by 1 / min Delta_k would be D times larger
    assert abs(spw["f_margin64"] - ss["f_margin64"]) <= 1e-14, (spw["f_margin64"], ss["f_margin64"])
