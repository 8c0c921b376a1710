"""Edge cases of the GPU path against the FP64 oracle: the smallest and
largest supported extents (every pass at its shortest and longest pencil),
1D lengths at both ends of the Bluestein range, shapes the library must
refuse, and degenerate bounds."""
import numpy as np
import pytest

from oracle import ffcz_oracle as O
from paper_2601_01596_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-3


def run(e0, E, D, **opts):
    import torch
    import paper_2601_01596_b300 as ffcz
    plan = ffcz.Plan([e0.shape], **opts)
    t = torch.from_numpy(np.ascontiguousarray(e0, dtype=np.float32).reshape(-1)).cuda()
    st = plan.correct(t, [E], [D])
    return t.cpu().numpy().reshape(e0.shape), st[0]


def stress(shape, seed, frac=0.5):
    e0 = W.bimodal_error(shape, seed, E=1.0, dtype=np.float32)
    return e0, 1.0, frac * O.f_violation(O.dft(e0.astype(np.float64)))


@pytest.mark.parametrize("shape", [(8, 8, 16), (8, 16), (1024, 8, 16), (8, 1024, 16),
                                   (8, 8, 2048), (1024, 2048), (8, 1024, 2048)])
def test_extreme_extents_match_oracle(shape):
    """Shortest (8; 16 on x) and longest (1024; 2048 on x) pencils of every pass."""
    e0, E, D = stress(shape, 11)
    ref = O.correct(e0, E, D)
    e, st = run(e0, E, D)
    assert ref.iters >= 1 and abs(st["iters"] - ref.iters) <= 2
    assert st["status"] == 0 and st["certified"] == 1
    same = O.correct(e0, E, D, min_iters=st["iters"], max_iters=st["iters"])
    np.testing.assert_allclose(e, same.e, rtol=0, atol=TOL * E)


@pytest.mark.parametrize("n", [32, 33, 524287, 524288])
def test_1d_length_range_ends(n):
    e0, E, D = stress((n,), 5)
    ref = O.correct(e0, E, D)
    e, st = run(e0, E, D)
    assert abs(st["iters"] - ref.iters) <= 2 and st["certified"] == 1
    same = O.correct(e0, E, D, min_iters=st["iters"], max_iters=st["iters"])
    np.testing.assert_allclose(e, same.e, rtol=0, atol=TOL * E)


@pytest.mark.parametrize("shapes", [[(8, 8, 24)], [(4, 8, 16)], [(8, 8, 8)], [(2048, 8, 16)],
                                    [(8, 8, 4096)], [(31,)], [(524289,)], [(8, 12)],
                                    [(16, 16), (16, 16, 16)]])
def test_unsupported_shapes_are_refused(shapes):
    import paper_2601_01596_b300 as ffcz
    with pytest.raises((ffcz.FFCzError, ValueError)):
        ffcz.Plan(shapes)


def test_degenerate_bounds():
    shape = (16, 32, 32)
    e0, E, _ = stress(shape, 2)
    # the f-bound above every coefficient: zero iterations, e returned as given
    big = 2.0 * O.f_violation(O.dft(e0.astype(np.float64)))
    e, st = run(e0, E, big)
    assert st["iters"] == 0 and st["certified"] == 1 and np.array_equal(e, e0)
    # a tiny f-bound drives the field to (almost) zero; the result is certified
    tiny = 1e-4 * O.f_violation(O.dft(e0.astype(np.float64)))
    ref = O.correct(e0, E, tiny)
    e, st = run(e0, E, tiny)
    assert st["status"] == 0 and st["certified"] == 1 and abs(st["iters"] - ref.iters) <= 2
    # |e_n| <= (1/N) sum_k |delta_k| <= sqrt(2) Delta once every bin is in the box
    assert float(np.max(np.abs(e))) <= np.sqrt(2.0) * tiny
    # a field far outside the s-cube: pre-clip (A3), then the loop
    wide = (e0 * 3.0).astype(np.float32)
    ref = O.correct(wide, E, big)
    e, st = run(wide, E, big)
    assert ref.preclipped and st["preclipped"] == 1 and st["certified"] == 1
    np.testing.assert_allclose(e, ref.e, rtol=0, atol=TOL * E)


def test_certification_of_special_float_values():
    """The FP64 certification widens float32 on the integer pipe (subnormals,
    signed zeros and the largest exponents included): its violation must
    bracket the exact one computed from numpy's float64 upcast."""
    import torch
    import paper_2601_01596_b300 as ffcz
    shape = (16, 32, 64)
    r = np.random.default_rng(4)
    e0 = W.bimodal_error(shape, 9, dtype=np.float32)
    flat = e0.reshape(-1)
    idx = r.choice(flat.size, 400, replace=False)
    flat[idx[:100]] = np.float32(0.0)
    flat[idx[100:200]] = np.float32(-0.0)
    flat[idx[200:300]] = (r.uniform(-1, 1, 100) * 1e-40).astype(np.float32)   # subnormal
    flat[idx[300:]] = (r.uniform(-1, 1, 100) * 1e-30).astype(np.float32)
    for scale in (1.0, 2.0 ** 100, 2.0 ** -100):
        x = (e0 * np.float32(scale)).astype(np.float32)
        v = O.f_violation(O.dft(x.astype(np.float64)))
        s = float(np.max(np.abs(x.astype(np.float64))))
        plan = ffcz.Plan([shape])
        t = torch.from_numpy(x.reshape(-1).copy()).cuda()
        assert plan.check(t, [s], [v * (1 + 1e-8)])[0]["certified"] == 1, scale
        assert plan.check(t, [s], [v * (1 - 1e-8)])[0]["certified"] == 0, scale


@pytest.mark.parametrize("n", [4096, 4097])
def test_certification_1d_special_float_values_and_nonfinite(n):
    """1D items (even N through the N/2-point transform, odd N through the
    N-point one): signed zeros, subnormals and extreme scales keep the
    verdict bracketing the exact violation; a NaN or an Inf is never
    certified."""
    import torch
    import paper_2601_01596_b300 as ffcz
    r = np.random.default_rng(6)
    e0 = W.bimodal_error((n,), 10, dtype=np.float32)
    idx = r.choice(n, 200, replace=False)
    e0[idx[:50]] = np.float32(0.0)
    e0[idx[50:100]] = np.float32(-0.0)
    e0[idx[100:150]] = (r.uniform(-1, 1, 50) * 1e-40).astype(np.float32)
    e0[idx[150:]] = (r.uniform(-1, 1, 50) * 1e-30).astype(np.float32)
    plan = ffcz.Plan([(n,)])
    for scale in (1.0, 2.0 ** 100, 2.0 ** -100):
        x = (e0 * np.float32(scale)).astype(np.float32)
        v = O.f_violation(O.dft(x.astype(np.float64)))
        s = float(np.max(np.abs(x.astype(np.float64))))
        t = torch.from_numpy(x.copy()).cuda()
        assert plan.check(t, [s], [v * (1 + 1e-8)])[0]["certified"] == 1, scale
        assert plan.check(t, [s], [v * (1 - 1e-8)])[0]["certified"] == 0, scale
    for bad in (np.nan, np.inf):
        x = e0.copy()
        x[n // 3] = bad
        t = torch.from_numpy(x).cuda()
        st = plan.check(t, [1e30], [1e30])[0]
        assert st["certified"] == 0, (bad, st)


def test_fp64_repair_after_a_failed_certification():
    """A float32 loop stopped by its cap short of feasibility fails the FP64
    certification; the FP64 repair (Alg. 1 in float64 from the
    float32 result) brings the field inside.  The oracle's own check confirms
    the result, and the host-buffer entry point (which copies the field back
    early and again after a repair) returns the same bits."""
    import paper_2601_01596_b300 as ffcz
    e0, E, D = stress((32, 32, 32), 5, frac=0.2)
    ref = O.correct(e0, E, D)
    cap = ref.iters - 2                  # e_cap is outside the true f-cube (checked below)
    assert not O.certify(O.correct(e0, E, D, min_iters=cap, max_iters=cap).e, E, D)[0]
    e, st = run(e0, E, D, max_iters=cap)
    assert st["repairs"] >= 1 and st["certified"] == 1
    ok, s, v = O.certify(e.astype(np.float64), E, D)
    assert ok, (s, v)
    host = e0.reshape(-1).copy()
    plan = ffcz.Plan([e0.shape], max_iters=cap)
    sth = plan.correct_host(host, [E], [D])[0]
    assert sth["repairs"] == st["repairs"] and np.array_equal(host, e.reshape(-1))
    assert sth["host_copies"] >= 1


@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 128), (16, 16, 64), (64, 8, 16), (8, 256, 32)])
def test_host_entry_certification_from_the_upload_matches_device(shape):
    """At 0 iterations the host entry point certifies from the x pass (3D:
    and y pass, chunks of whole z-planes) it ran while uploading: same bits
    out, no copy back, certified, the same FP64 margins as the device entry
    point (up to the summation order of the norm)."""
    import torch
    import paper_2601_01596_b300 as ffcz
    r = np.random.default_rng(17)
    e0 = (r.uniform(-1, 1, shape) * 0.5).astype(np.float32)
    E = 1.0
    D = 2.0 * O.f_violation(O.dft(e0.astype(np.float64)))
    plan = ffcz.Plan([shape])
    t = torch.from_numpy(e0.reshape(-1).copy()).cuda()
    sd = plan.correct(t, [E], [D])[0]
    host = e0.reshape(-1).copy()
    sh = plan.correct_host(host, [E], [D])[0]
    assert sd["iters"] == 0 and sh["iters"] == 0
    assert sh["certified"] == 1 and np.array_equal(host, e0.reshape(-1))
    assert sh["host_copies"] == 0
    assert abs(sh["f_margin64"] - sd["f_margin64"]) < 1e-12
    assert sh["s_margin64"] == sd["s_margin64"]


@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 16, 64), (64, 128)])
def test_host_entry_iterating_field_is_copied_back(shape):
    """A field the loop edits comes back through the copy stream once, with
    the device entry point's bits and certification."""
    import torch
    import paper_2601_01596_b300 as ffcz
    e0, E, D = stress(shape, 8)
    plan = ffcz.Plan([shape])
    t = torch.from_numpy(e0.reshape(-1).copy()).cuda()
    sd = plan.correct(t, [E], [D])[0]
    host = e0.reshape(-1).copy()
    sh = plan.correct_host(host, [E], [D])[0]
    assert sd["iters"] >= 1 and sh["iters"] == sd["iters"] and sh["certified"] == 1
    assert sh["host_copies"] == 1 and np.array_equal(host, t.cpu().numpy())
    assert sh["f_margin64"] == sd["f_margin64"]
