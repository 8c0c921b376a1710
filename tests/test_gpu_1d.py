"""1D items of any length (Bluestein path) vs the FP64 oracle."""
import numpy as np
import pytest

from oracle import ffcz_oracle as O
from paper_2601_01596_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-3


def run1d(items, Es, Ds, **opts):
    import torch
    import paper_2601_01596_b300 as ffcz
    plan = ffcz.Plan([(len(x),) for x in items], **opts)
    t = torch.from_numpy(np.concatenate([np.asarray(x, np.float32) for x in items])).cuda()
    st = plan.correct(t, Es, Ds)
    out = t.cpu().numpy()
    res, off = [], 0
    for x in items:
        res.append(out[off:off + len(x)])
        off += len(x)
    return res, st


@pytest.mark.parametrize("n", [32, 37, 61, 100, 128, 257, 1000, 4099, 40000])
def test_stress_1d_matches_oracle(n):
    e0 = W.bimodal_error((n,), 7 + n, dtype=np.float32)
    D = 0.5 * O.f_violation(O.dft(e0.astype(np.float64)))
    ref = O.correct(e0, 1.0, D)
    (got,), st = run1d([e0], [1.0], [D])
    assert st[0]["certified"] == 1, st[0]
    assert abs(st[0]["iters"] - ref.iters) <= 2
    np.testing.assert_allclose(got, ref.e, rtol=0, atol=TOL)


@pytest.mark.parametrize("n", [61, 1000])
def test_first_iterations_1d(n):
    e0 = W.bimodal_error((n,), 3, dtype=np.float32)
    D = 0.35 * O.f_violation(O.dft(e0.astype(np.float64)))
    for k in (1, 2, 5):
        ref = O.correct(e0, 1.0, D, min_iters=k, max_iters=k)
        (got,), st = run1d([e0], [1.0], [D], min_iters=k, max_iters=k, certify=0)
        assert st[0]["iters"] == k
        np.testing.assert_allclose(got, ref.e, rtol=0, atol=TOL, err_msg=f"iteration {k}")


def test_fp64_loop_1d_tight():
    n = 999
    e0 = W.bimodal_error((n,), 5, dtype=np.float32)
    D = 0.5 * O.f_violation(O.dft(e0.astype(np.float64)))
    ref = O.correct(e0, 1.0, D)
    (got,), st = run1d([e0], [1.0], [D], precision=64)
    assert st[0]["iters"] == ref.iters and st[0]["certified"] == 1
    np.testing.assert_allclose(got, ref.e, rtol=0, atol=1e-6)


def test_eeg_batch_as_written_and_batched_equals_singles():
    items = W.eeg_batch(count=8, seed=1, lo=1024, hi=20000)
    e0s = [it["e0"] for it in items]
    Es = [it["E"] for it in items]
    Ds = [it["D"] for it in items]
    got, st = run1d(e0s, Es, Ds)
    for i, it in enumerate(items):
        ref = O.correct(it["e0"], it["E"], it["D"])
        assert st[i]["iters"] == ref.iters and st[i]["certified"] == 1
        if not ref.preclipped:
            assert np.array_equal(got[i], it["e0"])
        single, s1 = run1d([it["e0"]], [it["E"]], [it["D"]])
        assert np.array_equal(single[0], got[i])


def test_batched_stress_1d_uneven_lengths():
    ns = [50, 333, 1024, 777, 2049]
    e0s = [W.bimodal_error((n,), 100 + n, dtype=np.float32) for n in ns]
    Ds = [0.4 * O.f_violation(O.dft(x.astype(np.float64))) for x in e0s]
    got, st = run1d(e0s, [1.0] * len(ns), Ds)
    for i, n in enumerate(ns):
        ref = O.correct(e0s[i], 1.0, Ds[i])
        assert abs(st[i]["iters"] - ref.iters) <= 2 and st[i]["certified"] == 1
        np.testing.assert_allclose(got[i], ref.e, rtol=0, atol=TOL)
        single, _ = run1d([e0s[i]], [1.0], [Ds[i]])
        assert np.array_equal(single[0], got[i])


def test_certification_1d_brackets_true_violation():
    import torch
    import paper_2601_01596_b300 as ffcz
    for n in (61, 5000):
        e0 = W.bimodal_error((n,), 11, dtype=np.float32)
        v = O.f_violation(O.dft(e0.astype(np.float64)))
        s = float(np.max(np.abs(e0)))
        plan = ffcz.Plan([(n,)])
        t = torch.from_numpy(e0.copy()).cuda()
        assert plan.check(t, [s], [v * (1 + 1e-7)])[0]["certified"] == 1
        assert plan.check(t, [s], [v * (1 - 1e-7)])[0]["certified"] == 0


@pytest.mark.parametrize("n", [64, 1500, 3000, 9000, 31000, 3001])
def test_certification_1d_even_lengths_through_half_transform(n):
    """Even N is certified through the N/2-point transform of x_2n + i x_2n+1
    and the real-input post-processing (odd N through the N-point one): the
    FP64 violation equals the oracle's to far below the certification's
    resolution, and the verdict brackets the true violation at 1e-8."""
    import torch
    import paper_2601_01596_b300 as ffcz
    e0 = W.bimodal_error((n,), 13, dtype=np.float32)
    v = O.f_violation(O.dft(e0.astype(np.float64)))
    s = float(np.max(np.abs(e0)))
    plan = ffcz.Plan([(n,)])
    t = torch.from_numpy(e0.copy()).cuda()
    D = v * (1 + 1e-8)
    ok = plan.check(t, [s], [D])[0]
    assert ok["certified"] == 1
    # f_margin64 = 1 - (v64 + b) / D: the shortfall against 1 - v / D is
    # (v64 - v) / D plus the stated rounding bound b / D (u = 2^-53, ||x||_2
    # from the sum of squares; log2 P of the N-point Bluestein length)
    u, x = 2.0 ** -53, e0.astype(np.float64)
    nrm = float(np.sqrt(np.sum(x * x)))
    lP = int(np.log2(max(64, 1 << int(np.ceil(np.log2(2 * n - 1))))))
    if n % 2 == 0 and n >= 64:
        b = 2 * 10 * (2 * (lP - 1) + 6) * u * n * nrm + 20 * u * np.sqrt(n) * nrm
    else:
        b = 10 * (2 * lP + 6) * u * 2 * n * nrm
    short = (1 - v / D) - ok["f_margin64"]
    assert abs(short - b / D) <= 1e-12 + 1e-3 * b / D, (short, b / D)
    assert plan.check(t, [s], [v * (1 - 1e-8)])[0]["certified"] == 0
    assert plan.check(t, [s * (1 - 1e-7)], [2 * v])[0]["certified"] == 0


def test_certification_1d_mixed_parities_in_one_batch():
    import torch
    import paper_2601_01596_b300 as ffcz
    ns = [1500, 1501, 3000, 2999, 64, 65]
    items = [W.bimodal_error((n,), 14 + i, dtype=np.float32) for i, n in enumerate(ns)]
    vs = [O.f_violation(O.dft(x.astype(np.float64))) for x in items]
    ss = [float(np.max(np.abs(x))) for x in items]
    plan = ffcz.Plan([(n,) for n in ns])
    t = torch.from_numpy(np.concatenate(items)).cuda()
    up = plan.check(t, ss, [v * (1 + 1e-8) for v in vs])
    down = plan.check(t, ss, [v * (1 - 1e-8) for v in vs])
    for i in range(len(ns)):
        assert up[i]["certified"] == 1 and down[i]["certified"] == 0, (ns[i], up[i], down[i])
