"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Bars: max|e_gpu - e_oracle| <= 1e-3 * eps_s after every forced iteration
1..10 and at convergence; iteration count within +-2 of the oracle's; every
output passes the FP64 certification on the GPU.  The FP64 loop must match
to 1e-9 * eps_s with the same iteration count.
"""
import numpy as np
import pytest

from oracle import ffcz_oracle as O
from paper_2601_01596_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-3


def _torch():
    import torch
    return torch


def run_gpu(e0, E, D, shapes=None, **opts):
    """Correct packed items on the GPU; returns (e_out numpy, stats list)."""
    torch = _torch()
    import paper_2601_01596_b300 as ffcz
    if shapes is None:
        shapes = [e0.shape]
        flat = e0.reshape(-1)
        Es, Ds = [E], [D]
    else:
        flat = e0
        Es, Ds = E, D
    plan = ffcz.Plan(shapes, **opts)
    t = torch.from_numpy(np.ascontiguousarray(flat, dtype=np.float32)).cuda()
    st = plan.correct(t, Es, Ds)
    torch.cuda.synchronize()
    return t.cpu().numpy(), st


def stress(shape, seed, frac=0.5):
    e0 = W.bimodal_error(shape, seed, E=1.0, dtype=np.float32)
    D = frac * O.f_violation(O.dft(e0.astype(np.float64)))
    return e0, 1.0, D


# --------------------------------------------------------------- workloads
def test_grf32_as_written_zero_iterations_bit_identical():
    it = W.grf_field(32)
    e, st = run_gpu(it["e0"], it["E"], it["D"])
    ref = O.correct(it["e0"], it["E"], it["D"])
    assert ref.iters == 0 and st[0]["iters"] == 0
    assert st[0]["status"] == 0 and st[0]["certified"] == 1
    if not ref.preclipped:
        assert np.array_equal(e.reshape(it["shape"]), it["e0"])
    else:
        np.testing.assert_allclose(e.reshape(it["shape"]), ref.e, rtol=0, atol=TOL * it["E"])


@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 32, 64), (64, 128), (256, 32)])
def test_stress_converged_matches_oracle(shape):
    e0, E, D = stress(shape, 3)
    ref = O.correct(e0, E, D)
    e, st = run_gpu(e0, E, D)
    assert ref.iters >= 2
    assert abs(st[0]["iters"] - ref.iters) <= 2
    assert st[0]["status"] == 0 and st[0]["certified"] == 1
    np.testing.assert_allclose(e.reshape(shape), ref.e, rtol=0, atol=TOL * E)


def test_grf32_stress_variant():
    it = W.grf_field(32, stress=0.2)
    ref = O.correct(it["e0"], it["E"], it["D"])
    e, st = run_gpu(it["e0"], it["E"], it["D"])
    assert abs(st[0]["iters"] - ref.iters) <= 2 and st[0]["certified"] == 1
    np.testing.assert_allclose(e.reshape(it["shape"]), ref.e, rtol=0, atol=TOL * it["E"])


@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 128)])
def test_each_of_first_ten_iterations(shape):
    e0, E, D = stress(shape, 5, frac=0.35)
    for k in range(1, 11):
        ref = O.correct(e0, E, D, min_iters=k, max_iters=k)
        e, st = run_gpu(e0, E, D, min_iters=k, max_iters=k, certify=0)
        assert st[0]["iters"] == k
        np.testing.assert_allclose(e.reshape(shape), ref.e, rtol=0, atol=TOL * E,
                                   err_msg=f"iteration {k}")


@pytest.mark.parametrize("shape", [(16, 16, 32), (32, 64)])
def test_fp64_loop_matches_oracle_tightly(shape):
    e0, E, D = stress(shape, 7)
    ref = O.correct(e0, E, D)
    e, st = run_gpu(e0, E, D, precision=64)
    assert st[0]["iters"] == ref.iters and st[0]["certified"] == 1
    # float32 output of an FP64 loop: one rounding of each value
    np.testing.assert_allclose(e.reshape(shape), ref.e, rtol=0, atol=1e-6 * E)


# ------------------------------------------------------------ closed forms
def test_single_mode_closed_form_gpu():
    shape, k0 = (16, 16, 32), (1, 2, 3)
    N = int(np.prod(shape))
    A, E = 0.5, 1.0
    D = 0.1 * A * N / 2
    e0 = W.single_mode(shape, k0, A, dtype=np.float32)
    e, st = run_gpu(e0, E, D)
    Ds = D * (1 - 2.0 ** -16)
    assert st[0]["iters"] == 1
    np.testing.assert_allclose(e.reshape(shape), W.single_mode(shape, k0, 2 * Ds / N),
                               rtol=0, atol=1e-6 * A)


def test_spike_closed_form_gpu():
    shape = (8, 16, 16)
    E, D = 1.0, 0.5
    e0 = np.zeros(shape, np.float32)
    e0.flat[0] = np.float32(E * (1 - 2.0 ** -16))
    e, st = run_gpu(e0, E, D)
    want = np.zeros(shape); want.flat[0] = D * (1 - 2.0 ** -16)
    assert st[0]["iters"] == 1
    np.testing.assert_allclose(e.reshape(shape), want, rtol=0, atol=1e-6)


def test_zero_field_zero_iterations():
    e0 = np.zeros((32, 32), np.float32)
    e, st = run_gpu(e0, 1.0, 1.0)
    assert st[0]["iters"] == 0 and np.array_equal(e, e0.reshape(-1))


# -------------------------------------------------------------- invariants
def test_negation_and_pow2_scaling_exact_on_gpu():
    shape = (16, 32, 32)
    e0, E, D = stress(shape, 9)
    a, sa = run_gpu(e0, E, D, certify=0)
    b, sb = run_gpu(-e0, E, D, certify=0)
    c, sc = run_gpu(4.0 * e0, 4.0 * E, 4.0 * D, certify=0)
    assert sa[0]["iters"] == sb[0]["iters"] == sc[0]["iters"]
    assert np.array_equal(b, -a)          # both clips are odd maps
    assert np.array_equal(c, 4.0 * a)     # powers of two scale exactly


def test_preclip_reading_A3_gpu():
    e0, E, D = stress((32, 32), 11)
    e0 = e0.copy()
    e0[3, 5] = 1.7
    e0[10, 1] = -2.5
    ref = O.correct(e0, E, D)
    e, st = run_gpu(e0, E, D)
    assert ref.preclipped and st[0]["preclipped"] == 1
    assert abs(st[0]["iters"] - ref.iters) <= 2
    np.testing.assert_allclose(e.reshape(32, 32), ref.e, rtol=0, atol=TOL * E)


def test_nonfinite_and_cap_statuses():
    import paper_2601_01596_b300 as ffcz
    e0, E, D = stress((32, 32), 12, frac=0.3)
    bad = e0.copy(); bad[4, 4] = np.nan
    _, st = run_gpu(bad, E, D)
    assert st[0]["status"] == ffcz.ERR_NONFINITE
    ref = O.correct(e0, E, D)
    assert ref.iters > 2
    _, st = run_gpu(e0, E, D, max_iters=1)
    assert st[0]["status"] == ffcz.ERR_NOT_CONVERGED and st[0]["iters"] == 1


# ---------------------------------------------------------- certification
def test_certification_threshold_brackets_true_violation():
    torch = _torch()
    import paper_2601_01596_b300 as ffcz
    for shape in [(32, 32, 32), (64, 128)]:
        e0 = W.bimodal_error(shape, 21, dtype=np.float32)
        v = O.f_violation(O.dft(e0.astype(np.float64)))
        s = float(np.max(np.abs(e0.astype(np.float64))))
        plan = ffcz.Plan([shape])
        t = torch.from_numpy(e0.reshape(-1).copy()).cuda()
        ok = plan.check(t, [s], [v * (1 + 1e-8)])[0]
        assert ok["certified"] == 1
        assert abs(ok["s_margin64"]) < 1e-15
        bad = plan.check(t, [s], [v * (1 - 1e-8)])[0]
        assert bad["certified"] == 0
        bad_s = plan.check(t, [s * (1 - 1e-7)], [2 * v])[0]
        assert bad_s["certified"] == 0


# ----------------------------------------------------------------- batches
def test_batched_mixed_shapes_equal_singles():
    shapes = [(64, 64), (32, 128), (64, 64), (128, 32), (32, 128)]
    items, Es, Ds = [], [], []
    for i, sh in enumerate(shapes):
        e0, E, D = stress(sh, 30 + i, frac=0.3 + 0.1 * (i % 3))
        items.append(e0); Es.append(E); Ds.append(D)
    packed = np.concatenate([x.reshape(-1) for x in items])
    out, st = run_gpu(packed, Es, Ds, shapes=shapes)
    off = 0
    for i, sh in enumerate(shapes):
        n = int(np.prod(sh))
        single, s1 = run_gpu(items[i], Es[i], Ds[i])
        assert np.array_equal(out[off:off + n], single), f"item {i}"
        assert st[i]["iters"] == s1[0]["iters"]
        ref = O.correct(items[i], Es[i], Ds[i])
        assert abs(st[i]["iters"] - ref.iters) <= 2
        np.testing.assert_allclose(out[off:off + n].reshape(sh), ref.e, rtol=0, atol=TOL * Es[i])
        off += n


def test_host_buffer_entry_point_matches_device():
    import paper_2601_01596_b300 as ffcz
    e0, E, D = stress((32, 32, 32), 40)
    dev, _ = run_gpu(e0, E, D)
    host = e0.reshape(-1).copy()
    plan = ffcz.Plan([e0.shape])
    plan.correct_host(host, [E], [D])
    assert np.array_equal(host, dev)


@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 128)])
def test_device_loop_graph_chunk_graphs_and_direct_launch_agree(shape):
    e0, E, D = stress(shape, 41)
    a, sa = run_gpu(e0, E, D, use_graph=2)     # conditional WHILE node
    b, sb = run_gpu(e0, E, D, use_graph=1)     # chunk graphs, host checks
    c, sc = run_gpu(e0, E, D, use_graph=0)     # direct launches
    assert sa[0]["iters"] == sb[0]["iters"] == sc[0]["iters"] >= 2
    assert np.array_equal(a, b) and np.array_equal(a, c)
    # caps inside the device loop
    d, sd = run_gpu(e0, E, D, use_graph=2, max_iters=1)
    import paper_2601_01596_b300 as ffcz
    assert sd[0]["iters"] == 1 and sd[0]["status"] == ffcz.ERR_NOT_CONVERGED


# ------------------------------------------------- TMA-fed persistent passes
@pytest.mark.parametrize("shape", [(256, 256, 32), (512, 32, 16), (256, 64), (16, 32, 512), (8, 16, 16),
                                   (1024, 16, 32), (16, 1024, 32), (1024, 64)])
def test_tma_fed_passes_equal_plain_passes_and_match_oracle(shape, monkeypatch):
    e0, E, D = stress(shape, 43)
    monkeypatch.setenv("FFCZ_TUNE_FORCE", "axis=tma,chk=tma,px=tma,split=0")
    a, sa = run_gpu(e0, E, D)
    monkeypatch.delenv("FFCZ_TUNE_FORCE")
    monkeypatch.setenv("FFCZ_TUNE", "0")     # default plain variants
    b, sb = run_gpu(e0, E, D)
    assert sa[0]["iters"] == sb[0]["iters"] >= 2
    assert np.array_equal(a, b)          # same arithmetic, other load path
    ref = O.correct(e0, E, D)
    assert abs(sa[0]["iters"] - ref.iters) <= 2 and sa[0]["certified"] == 1
    np.testing.assert_allclose(a.reshape(shape), ref.e, rtol=0, atol=TOL * E)


def test_tma_fed_batch_equals_singles(monkeypatch):
    monkeypatch.setenv("FFCZ_TUNE_FORCE", "axis=tma,chk=tma,px=tma")
    shapes = [(256, 64), (256, 32), (256, 64), (512, 16)]
    items, Es, Ds = [], [], []
    for i, sh in enumerate(shapes):
        e0, E, D = stress(sh, 60 + i, frac=0.3 + 0.1 * (i % 3))
        items.append(e0); Es.append(E); Ds.append(D)
    packed = np.concatenate([x.reshape(-1) for x in items])
    out, st = run_gpu(packed, Es, Ds, shapes=shapes)
    off = 0
    for i, sh in enumerate(shapes):
        n = int(np.prod(sh))
        single, s1 = run_gpu(items[i], Es[i], Ds[i])
        assert np.array_equal(out[off:off + n], single), f"item {i}"
        assert st[i]["iters"] == s1[0]["iters"] and st[i]["certified"] == 1
        off += n


# ------------------------------------------------ radix split of the passes
def _split_force(shape):
    """FFCZ_TUNE_FORCE pinning the plain kernels in the swapped radix split
    (stage 1 of size V, stage 2 of size NT) for every pass whose length has
    an odd log2; returns (spec, the splits describe() must show)."""
    def lg(n):
        return int(n).bit_length() - 1
    M = shape[-1] // 2
    Lc = shape[0]
    parts, want = [], []
    if lg(M) % 2:
        parts.append(f"px={(32 >> (lg(M) // 2)) | 256}")
        want.append(f"px={32 >> (lg(M) // 2)} {M >> (lg(M) // 2)}x{1 << (lg(M) // 2)}")
    if len(shape) == 3 and lg(shape[1]) % 2:
        Ly = shape[1]
        parts.append(f"axis={8 | 256}")
        want.append(f"axis=8 {Ly >> (lg(Ly) // 2)}x{1 << (lg(Ly) // 2)}")
    if lg(Lc) % 2:
        parts.append(f"chk={8 | 256}")
        want.append(f"chk=8 {Lc >> (lg(Lc) // 2)}x{1 << (lg(Lc) // 2)}")
    return ",".join(parts), want


@pytest.mark.parametrize("shape", [(32, 32, 32), (128, 32, 512), (512, 32, 16), (128, 64), (512, 128)])
def test_swapped_radix_split_matches_oracle(shape, monkeypatch):
    """The tuner's radix-split candidates: the same passes with the stage
    sizes swapped (e.g. 512 = 32 x 16 instead of 16 x 32) after each forced
    iteration 1..3 and at convergence, against the oracle."""
    import paper_2601_01596_b300 as ffcz
    spec, want = _split_force(shape)
    assert want
    monkeypatch.setenv("FFCZ_TUNE_FORCE", spec)
    desc = ffcz.Plan([shape]).describe()
    for w in want:
        assert w in desc, (w, desc)
    e0, E, D = stress(shape, 44)
    for k in (1, 2, 3):
        ref = O.correct(e0, E, D, min_iters=k, max_iters=k)
        e, st = run_gpu(e0, E, D, min_iters=k, max_iters=k, certify=0)
        assert st[0]["iters"] == k
        np.testing.assert_allclose(e.reshape(shape), ref.e, rtol=0, atol=TOL * E, err_msg=f"iteration {k}")
    ref = O.correct(e0, E, D)
    e, st = run_gpu(e0, E, D)
    assert abs(st[0]["iters"] - ref.iters) <= 2 and st[0]["certified"] == 1
    np.testing.assert_allclose(e.reshape(shape), ref.e, rtol=0, atol=TOL * E)
