"""GPU projection variants (Dykstra, Douglas-Rachford, ADMM; Sec. III) against
the FP64 oracle's literal recurrences, through the C ABI.

Bars as for Alg. 1: max|e_gpu - e_oracle| <= 1e-3 eps_s after forced
iterations 1..10 and at the returned point, iteration count within +-2, and
every output passes the FP64 certification on the GPU.
"""
import numpy as np
import pytest

from oracle import ffcz_oracle as O
from paper_2601_01596_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-3
METHODS = ["dykstra", "dr", "admm"]


def run_gpu(e0, E, D, shapes=None, **opts):
    import torch
    import paper_2601_01596_b300 as ffcz
    if shapes is None:
        shapes, flat, Es, Ds = [e0.shape], e0.reshape(-1), [E], [D]
    else:
        flat, Es, Ds = e0, E, D
    plan = ffcz.Plan(shapes, **opts)
    t = torch.from_numpy(np.ascontiguousarray(flat, dtype=np.float32)).cuda()
    st = plan.correct(t, Es, Ds)
    torch.cuda.synchronize()
    return t.cpu().numpy(), st


def stress(shape, seed, frac=0.5):
    e0 = W.bimodal_error(shape, seed, E=1.0, dtype=np.float32)
    return e0, 1.0, frac * O.f_violation(O.dft(e0.astype(np.float64)))


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 32, 64), (64, 128), (3000,), (1500,)])
def test_forced_iterations_match_oracle(method, shape):
    e0, E, D = stress(shape, 3)
    for K in (1, 2, 3, 5, 10):
        ref = O.correct_method(e0, E, D, method, min_iters=K, max_iters=K)
        e, st = run_gpu(e0, E, D, method=method, min_iters=K, max_iters=K, certify=0)
        assert st[0]["iters"] == K
        np.testing.assert_allclose(e.reshape(shape), ref.e, rtol=0, atol=TOL * E,
                                   err_msg=f"{method} K={K}")


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 32, 64), (64, 128), (256, 32), (3000,), (9000,)])
def test_converged_matches_oracle_and_certifies(method, shape):
    e0, E, D = stress(shape, 5)
    ref = O.correct_method(e0, E, D, method)
    e, st = run_gpu(e0, E, D, method=method)
    assert ref.iters >= 1
    assert abs(st[0]["iters"] - ref.iters) <= 2
    assert st[0]["status"] == 0 and st[0]["certified"] == 1 and st[0]["repairs"] == 0
    same = O.correct_method(e0, E, D, method, min_iters=st[0]["iters"], max_iters=st[0]["iters"])
    np.testing.assert_allclose(e.reshape(shape), same.e, rtol=0, atol=TOL * E)


@pytest.mark.parametrize("method", METHODS)
def test_grf32_stress_workload(method):
    it = W.grf_field(32, stress=0.2)
    ref = O.correct_method(it["e0"], it["E"], it["D"], method)
    e, st = run_gpu(it["e0"], it["E"], it["D"], method=method)
    assert abs(st[0]["iters"] - ref.iters) <= 2 and st[0]["certified"] == 1
    same = O.correct_method(it["e0"], it["E"], it["D"], method,
                            min_iters=st[0]["iters"], max_iters=st[0]["iters"])
    np.testing.assert_allclose(e.reshape(it["shape"]), same.e, rtol=0, atol=TOL * it["E"])


@pytest.mark.parametrize("method", METHODS)
def test_zero_iterations_bit_identical(method):
    it = W.grf_field(32)
    e, st = run_gpu(it["e0"], it["E"], it["D"], method=method)
    assert st[0]["iters"] == 0 and st[0]["certified"] == 1
    ref = O.correct_method(it["e0"], it["E"], it["D"], method)
    if not ref.preclipped:
        assert np.array_equal(e.reshape(it["shape"]), it["e0"])


def test_single_mode_closed_forms_on_gpu():
    """The hand-derived one-iteration answers of the oracle pins, on the GPU."""
    shape = (8, 16, 16)
    N = int(np.prod(shape))
    z, y, x = np.indices(shape)
    c = np.cos(2 * np.pi * (1 * z / 8 + 2 * y / 16 + 3 * x / 16))
    E, A = 1.0, 0.5
    D = 0.4 * A * N / 2
    Ds = D * (1 - O.ETA_DEFAULT)
    want = {"dykstra": (2 * Ds / N) * c, "admm": (2 * Ds / N) * c, "dr": (4 * Ds / N - A) * c}
    for method, w in want.items():
        e, st = run_gpu((A * c).astype(np.float32), E, D, method=method)
        assert st[0]["iters"] == 1 and st[0]["certified"] == 1, method
        np.testing.assert_allclose(e.reshape(shape), w, rtol=0, atol=1e-6, err_msg=method)


@pytest.mark.parametrize("method", METHODS)
def test_batch_of_uneven_1d_items_equals_singles(method):
    shapes = [(3000,), (1500,), (3000,), (9000,)]
    items = [stress(s, 30 + i)[0] for i, s in enumerate(shapes)]
    Es = [1.0] * 4
    Ds = [0.5 * O.f_violation(O.dft(x.astype(np.float64))) for x in items]
    flat = np.concatenate([x.reshape(-1) for x in items])
    e, st = run_gpu(flat, Es, Ds, shapes=shapes, method=method)
    off = 0
    for i, (x, s) in enumerate(zip(items, shapes)):
        es, ss = run_gpu(x, Es[i], Ds[i], method=method)
        n = x.size
        assert st[i]["iters"] == ss[0]["iters"] and st[i]["certified"] == 1
        assert np.array_equal(e[off:off + n], es.reshape(-1))
        off += n


@pytest.mark.parametrize("method", METHODS)
def test_batch_of_uneven_items_equals_singles(method):
    shapes = [(32, 32, 32), (16, 32, 64), (32, 32, 32)]
    items = [stress(s, 20 + i)[0] for i, s in enumerate(shapes)]
    Es = [1.0] * 3
    Ds = [0.5 * O.f_violation(O.dft(x.astype(np.float64))) for x in items]
    # a plan holds one rank; group shapes of the same rank in one batch
    flat = np.concatenate([x.reshape(-1) for x in items])
    e, st = run_gpu(flat, Es, Ds, shapes=shapes, method=method)
    off = 0
    for i, (x, s) in enumerate(zip(items, shapes)):
        es, ss = run_gpu(x, Es[i], Ds[i], method=method)
        n = x.size
        assert st[i]["iters"] == ss[0]["iters"] and st[i]["certified"] == 1
        assert np.array_equal(e[off:off + n], es.reshape(-1))
        off += n


def test_variant_option_checks():
    import paper_2601_01596_b300 as ffcz
    with pytest.raises(ffcz.FFCzError):
        ffcz.Plan([(4096,)], method="dykstra", edits=1)   # 1D items: the same rules
    with pytest.raises(ffcz.FFCzError):
        ffcz.Plan([(32, 32, 32)], method="dr", edits=1)
    with pytest.raises(ffcz.FFCzError):
        ffcz.Plan([(32, 32, 32)], method="admm", pointwise=1)
    with pytest.raises(ffcz.FFCzError):
        ffcz.Plan([(32, 32, 32)], method="dykstra", precision=64)
    with pytest.raises(ffcz.FFCzError):
        ffcz.Plan([(32, 32, 32)], method=4)


@pytest.mark.parametrize("method", ["dykstra", "dr"])
@pytest.mark.parametrize("shape", [(256, 32, 32), (512, 16, 32), (256, 64)])
def test_tma_fed_residual_check_equals_plain_and_matches_oracle(method, shape, monkeypatch):
    """The persistent check pass stages the residual of Dykstra / Douglas-
    Rachford beside the spectrum; the tiled pass loads it with plain loads.
    Same arithmetic: bit-identical results, and both match the oracle."""
    e0, E, D = stress(shape, 7)
    monkeypatch.setenv("FFCZ_TUNE_FORCE", "axis=tma,px=tma,chk=tma")
    a, sa = run_gpu(e0, E, D, method=method)
    monkeypatch.setenv("FFCZ_TUNE_FORCE", "axis=tma,px=tma,chk=8")
    b, sb = run_gpu(e0, E, D, method=method)
    monkeypatch.delenv("FFCZ_TUNE_FORCE")
    assert sa[0]["iters"] == sb[0]["iters"] >= 2 and sa[0]["certified"] == 1
    assert np.array_equal(a, b)
    ref = O.correct_method(e0, E, D, method)
    assert abs(sa[0]["iters"] - ref.iters) <= 2
    same = O.correct_method(e0, E, D, method, min_iters=sa[0]["iters"], max_iters=sa[0]["iters"])
    np.testing.assert_allclose(a.reshape(shape), same.e, rtol=0, atol=TOL * E)
    for K in (1, 3):
        monkeypatch.setenv("FFCZ_TUNE_FORCE", "axis=tma,px=tma,chk=tma")
        f, _ = run_gpu(e0, E, D, method=method, min_iters=K, max_iters=K, certify=0)
        monkeypatch.delenv("FFCZ_TUNE_FORCE")
        refk = O.correct_method(e0, E, D, method, min_iters=K, max_iters=K)
        np.testing.assert_allclose(f.reshape(shape), refk.e, rtol=0, atol=TOL * E, err_msg=f"K={K}")
