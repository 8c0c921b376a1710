"""Adjoint (ffcz_correct_backward) vs the oracle's vector-Jacobian product,
element by element.

The product depends on the clips' active-set masks, and a mask entry whose
pre-clip value lies within rounding of its bound may be decided either way by
a float32 trajectory.  One such decision moves EVERY coordinate of the
gradient (the DFT spreads it), so no coordinate can simply be excused.
Instead the oracle lists the near ties of its own FP64 trajectory (entries
within TAU of the bound, relative; far above the float32 drift of the GPU's
trajectory) and computes, coordinate by coordinate, how far its product moves
over other decisions of exactly those entries (``tie_spread``; zero where
there is none).  Every coordinate of the GPU's product must then lie within
GTOL * max|g| + 2 * spread of the oracle's.
"""
import numpy as np
import pytest

from oracle import ffcz_oracle as O
from paper_2601_01596_b300 import workloads as W

pytestmark = pytest.mark.gpu

TAU = 2e-5     # near-tie band of a clip decision, relative to its bound
GTOL = 1e-4    # element-wise tolerance, relative to max|g| (float32 steps)


def _assert_vjp_elementwise(got, e0, g, E, D, K, label, samples=8):
    ref = O.correct_backward(e0, g, E, D, K)
    spread, nnear = O.tie_spread(e0, g, E, D, K, TAU, samples=samples, seed=1)
    scale = float(np.max(np.abs(ref)))
    err = np.abs(got.astype(np.float64) - ref)
    allow = GTOL * scale + 2.0 * spread
    bad = err > allow
    print(f"{label}: max|dg|/max|g| = {err.max() / scale:.2e}, near ties {nnear}, "
          f"coordinates with spread > GTOL: {np.mean(spread > GTOL * scale):.4f}, "
          f"max|dg| where spread = 0: {err[spread == 0].max(initial=0.0) / scale:.2e}")
    assert not bad.any(), (label, int(bad.sum()), float((err - allow).max() / scale))
    return ref, spread


def _gpu_backward(shape, e0, g, E, D, K, m, ckpt=False):
    import torch
    import paper_2601_01596_b300 as ffcz
    te0 = torch.from_numpy(np.ascontiguousarray(e0).reshape(-1).copy()).cuda()
    tg = torch.from_numpy(np.ascontiguousarray(g, dtype=np.float32).reshape(-1).copy()).cuda()
    gi = torch.empty_like(te0)
    if ckpt:
        plan = ffcz.Plan([shape], K=K, ckpt_every=m, min_iters=K, max_iters=K, certify=0)
        ck = torch.empty(plan.ckpt_floats(), dtype=torch.float32, device="cuda")
        plan.correct_ckpt(te0.clone(), [E], [D], ck)
        plan.backward(te0, tg, gi, [E], [D], ckpt=ck)
    else:
        plan = ffcz.Plan([shape], K=K, ckpt_every=m)
        plan.backward(te0, tg, gi, [E], [D])
    return gi.cpu().numpy().reshape(shape)


@pytest.mark.parametrize("shape,K,m", [((16, 16, 32), 5, 2), ((32, 64), 6, 4), ((16, 16, 16), 3, 10)])
def test_backward_matches_oracle_vjp(shape, K, m):
    e0 = W.bimodal_error(shape, 50, dtype=np.float32)
    E = 1.0
    D = 0.4 * O.f_violation(O.dft(e0.astype(np.float64)))
    g = np.random.default_rng(51).standard_normal(shape).astype(np.float32)
    got = _gpu_backward(shape, e0, g, E, D, K, m)
    _assert_vjp_elementwise(got, e0, g, E, D, K, f"bimodal{shape} K={K}")


def _turbulence_like(shape, seed):
    """The differentiable workload's recipe on any shape: a GRF with E(k) ~
    k^-5/3, its quantisation error at eps_s = 1e-4 range, eps_f = 0.2 max box
    violation of e0 (A11)."""
    x = W.grf(shape, 5.0 / 3.0, seed).astype(np.float32)
    E = 1e-4 * (float(x.max()) - float(x.min()))
    e0 = W.quantization_error(x, E)
    return x, e0, E, 0.2 * W.max_box_fft(e0)


@pytest.mark.parametrize("shape", [(256, 8, 256), (8, 256, 256)])
def test_backward_K50_m10_on_256_point_passes(shape):
    """The differentiable workload's K = 50 forced iterations with a
    checkpoint every 10, on shapes whose z / y and x passes are the
    256-point kernels of the 256^3 form (checkpoints written by the forward,
    as the autograd function runs it)."""
    K, m = 50, 10
    x, e0, E, D = _turbulence_like(shape, 7)
    g = np.random.default_rng(52).standard_normal(shape).astype(np.float32)
    got = _gpu_backward(shape, e0, g, E, D, K, m, ckpt=True)
    _assert_vjp_elementwise(got, e0, g, E, D, K, f"turbulence{shape} K=50", samples=4)


def test_config5_crop_gradient_matches_fp64_finite_differences():
    """The differentiable workload's own check: the gradient on a 32^3 crop of
    the 256^3 turbulence field (an independent 32^3 problem: e0, the field's
    eps_s, eps_f by A11 on the crop), K = 50, checkpoint every 10, against
    central finite differences of the FP64 oracle's forward map (step 1e-6
    eps_s): for L(e0) = <g, e_K(e0)> along random directions and along
    single coordinates, and for the power-spectrum loss through the autograd
    function."""
    import torch
    from paper_2601_01596_b300.autograd import FFCzCorrect, power_spectrum_loss
    it = W.turbulence_field(256, seed=0)
    c = (slice(0, 32),) * 3
    x = np.ascontiguousarray(it["x"][c])
    e0 = np.ascontiguousarray(it["e0"][c])
    E = it["E"]
    D = 0.2 * W.max_box_fft(e0)
    del it
    K, m, shape = 50, 10, (32, 32, 32)
    e0d = e0.astype(np.float64)
    h = 1e-6 * E
    g = np.random.default_rng(53).standard_normal(shape).astype(np.float32).astype(np.float64)
    got = _gpu_backward(shape, e0, g, E, D, K, m, ckpt=True).astype(np.float64)
    ref, spread = _assert_vjp_elementwise(got, e0, g, E, D, K, "crop32 K=50")

    def L(e):
        return float(np.sum(g * O.forward_masks(e, E, D, K)[0]))
    rng = np.random.default_rng(54)
    for j in range(4):
        v = rng.standard_normal(shape)
        fd = (L(e0d + h * v) - L(e0d - h * v)) / (2 * h)
        # the oracle's product is the derivative of its own map ...
        assert abs(fd - np.sum(ref * v)) <= 1e-6 * np.linalg.norm(ref) * np.linalg.norm(v), j
        # ... and the GPU's is within its element-wise allowance of it
        slack = GTOL * np.max(np.abs(ref)) * np.sum(np.abs(v)) + 2.0 * np.sum(spread * np.abs(v))
        assert abs(fd - np.sum(got * v)) <= slack + 1e-6 * np.linalg.norm(ref) * np.linalg.norm(v), j
    for p in map(tuple, rng.integers(0, 32, size=(16, 3))):
        u = np.zeros(shape)
        u[p] = 1.0
        fd = (L(e0d + h * u) - L(e0d - h * u)) / (2 * h)
        assert abs(fd - ref[p]) <= 1e-6 * np.max(np.abs(ref)), p
        assert abs(fd - got[p]) <= GTOL * np.max(np.abs(ref)) + 2.0 * spread[p] + 1e-6 * np.max(np.abs(ref)), p

    # the power-spectrum loss of the workload, through torch.autograd
    xt = torch.from_numpy(x).cuda()
    e0t = torch.from_numpy(e0).cuda().requires_grad_(True)
    loss = power_spectrum_loss(xt, FFCzCorrect.apply(e0t, E, D, K, m))
    loss.backward()
    g_gpu = e0t.grad.cpu().numpy().astype(np.float64)
    xd = torch.from_numpy(x.astype(np.float64))

    def Ls(e):
        return float(power_spectrum_loss(xd, torch.from_numpy(O.forward_masks(e, E, D, K)[0])))
    eK = torch.from_numpy(O.forward_masks(e0d, E, D, K)[0]).requires_grad_(True)
    power_spectrum_loss(xd, eK).backward()
    gl = eK.grad.numpy()
    ref_l = O.correct_backward(e0, gl, E, D, K)
    spread_l, _ = O.tie_spread(e0, gl, E, D, K, TAU, samples=4, seed=2)
    scale = np.max(np.abs(ref_l))
    err = np.abs(g_gpu - ref_l)
    assert np.all(err <= 1e-3 * scale + 2.0 * spread_l), float(err.max() / scale)
    for j in range(2):
        v = rng.standard_normal(shape)
        fd = (Ls(e0d + h * v) - Ls(e0d - h * v)) / (2 * h)
        assert abs(fd - np.sum(ref_l * v)) <= 1e-5 * np.linalg.norm(ref_l) * np.linalg.norm(v), j


def test_autograd_function_matches_oracle_through_spectrum_loss():
    """d loss / d e0 for loss = log power-spectrum mismatch of x + e_K vs x,
    element by element against the oracle's product of the FP64 loss
    gradient (the loss gradient itself is taken at float32 e_K on the GPU:
    GTOL * 10)."""
    import torch
    from paper_2601_01596_b300.autograd import FFCzCorrect, power_spectrum_loss
    it = W.turbulence_field(16, seed=4)
    x = torch.from_numpy(it["x"].astype(np.float32)).cuda()
    e0 = torch.from_numpy(it["e0"]).cuda().requires_grad_(True)
    K, m = 6, 4
    eK = FFCzCorrect.apply(e0, it["E"], it["D"], K, m)
    loss = power_spectrum_loss(x, eK)
    loss.backward()
    g_gpu = e0.grad.cpu().numpy().astype(np.float64)
    # reference: same loss in float64 on the oracle's e_K, then the oracle VJP
    eK_ref, _, _ = O.forward_masks(it["e0"], it["E"], it["D"], K)
    et = torch.from_numpy(eK_ref).requires_grad_(True)
    lref = power_spectrum_loss(torch.from_numpy(it["x"].astype(np.float64)), et)
    lref.backward()
    gl = et.grad.numpy()
    g_ref = O.correct_backward(it["e0"], gl, it["E"], it["D"], K)
    spread, _ = O.tie_spread(it["e0"], gl, it["E"], it["D"], K, TAU, samples=8, seed=3)
    assert abs(loss.item() - lref.item()) <= 1e-3 * abs(lref.item()) + 1e-9
    scale = np.max(np.abs(g_ref))
    err = np.abs(g_gpu - g_ref)
    assert np.all(err <= 10 * GTOL * scale + 2.0 * spread), float(err.max() / scale)


def test_backward_with_copy_engine_fed_x_pass_equals_plain(monkeypatch):
    """The bulk-copy-fed x pass records and replays the same masks."""
    import torch
    import paper_2601_01596_b300 as ffcz
    shape, K, m = (16, 32, 512), 4, 2
    e0 = W.bimodal_error(shape, 52, dtype=np.float32)
    E = 1.0
    D = 0.4 * O.f_violation(O.dft(e0.astype(np.float64)))
    g = np.random.default_rng(53).standard_normal(shape).astype(np.float32)
    out = []
    for force in ("px=tma,split=0", None):
        if force:
            monkeypatch.setenv("FFCZ_TUNE_FORCE", force)
        else:
            monkeypatch.delenv("FFCZ_TUNE_FORCE")
            monkeypatch.setenv("FFCZ_TUNE", "0")
        plan = ffcz.Plan([shape], K=K, ckpt_every=m)
        te0 = torch.from_numpy(e0.reshape(-1).copy()).cuda()
        tg = torch.from_numpy(g.reshape(-1).copy()).cuda()
        gi = torch.empty_like(te0)
        plan.backward(te0, tg, gi, [E], [D])
        out.append(gi.cpu().numpy())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("shape,K,m,scale", [((16, 16, 32), 5, 2, 1.0), ((32, 64), 6, 4, 1.0),
                                             ((16, 16, 16), 3, 10, 1.0), ((16, 32, 32), 8, 4, 3.0)])
def test_checkpointed_forward_and_backward_equal_the_two_pass_form(shape, K, m, scale):
    """ffcz_correct_ckpt returns the same e_K as ffcz_correct and the
    checkpoints the backward would take itself; ffcz_correct_backward_ckpt
    gives the same gradient bits as ffcz_correct_backward.  scale = 3: e0
    outside the s-cube (pre-clip, checkpoint 0 is the clipped field); K = 8,
    m = 4: the loop's x pass at t = K is a multiple of m and writes nothing."""
    import torch
    import paper_2601_01596_b300 as ffcz
    e0 = (W.bimodal_error(shape, 54, dtype=np.float32) * np.float32(scale)).astype(np.float32)
    E = 1.0
    D = 0.4 * O.f_violation(O.dft(np.clip(e0, -E, E).astype(np.float64)))
    g = np.random.default_rng(55).standard_normal(shape).astype(np.float32)
    plan = ffcz.Plan([shape], K=K, ckpt_every=m, min_iters=K, max_iters=K, certify=0)
    n = e0.size
    nseg = (K + m - 1) // m
    assert plan.ckpt_floats() == nseg * n
    te0 = torch.from_numpy(e0.reshape(-1).copy()).cuda()
    ea = te0.clone()
    sa = plan.correct(ea, [E], [D])[0]
    eb = te0.clone()
    ck = torch.full((nseg * n,), float("nan"), dtype=torch.float32, device="cuda")
    sb = plan.correct_ckpt(eb, [E], [D], ck)[0]
    assert sa["iters"] == sb["iters"] == K and sa["preclipped"] == sb["preclipped"] == int(scale > 1)
    assert torch.equal(ea, eb)
    ckn = ck.cpu().numpy().reshape(nseg, n)
    assert np.isfinite(ckn).all()
    np.testing.assert_array_equal(ckn[0], np.clip(e0.reshape(-1), -E * (1 - 2.0 ** -16), E * (1 - 2.0 ** -16))
                                  if scale > 1 else e0.reshape(-1))
    # the last checkpoint is e_t of a run forced to t = (nseg - 1) m iterations
    t_last = (nseg - 1) * m
    if t_last > 0:
        p2 = ffcz.Plan([shape], min_iters=t_last, max_iters=t_last, certify=0)
        e2 = te0.clone()
        p2.correct(e2, [E], [D])
        np.testing.assert_allclose(ckn[-1], e2.cpu().numpy(), rtol=0, atol=1e-6 * E)
    # a plan that certifies (a repair could change e_K) is refused
    pc = ffcz.Plan([shape], K=K, ckpt_every=m, min_iters=K, max_iters=K, certify=1)
    with pytest.raises(ffcz.FFCzError):
        pc.correct_ckpt(te0.clone(), [E], [D], ck)
    tg = torch.from_numpy(g.reshape(-1).copy()).cuda()
    ga, gb = torch.empty_like(te0), torch.empty_like(te0)
    plan.backward(te0, tg, ga, [E], [D])
    plan.backward(te0, tg, gb, [E], [D], ckpt=ck)
    assert torch.equal(ga, gb)


def test_autograd_interleaved_forwards_keep_their_own_checkpoints():
    """Two forwards through the same cached plan before their backwards: each
    backward uses the checkpoints of its own forward."""
    import torch
    from paper_2601_01596_b300.autograd import FFCzCorrect
    shape, K, m = (16, 16, 32), 5, 2
    E = 1.0
    xs = [W.bimodal_error(shape, 60 + i, dtype=np.float32) for i in range(2)]
    D = 0.4 * O.f_violation(O.dft(xs[0].astype(np.float64)))
    gs = [torch.from_numpy(np.random.default_rng(70 + i).standard_normal(shape).astype(np.float32)).cuda()
          for i in range(2)]
    single = []
    for x, g in zip(xs, gs):
        e0 = torch.from_numpy(x).cuda().requires_grad_(True)
        (FFCzCorrect.apply(e0, E, D, K, m) * g).sum().backward()
        single.append(e0.grad.clone())
    e0s = [torch.from_numpy(x).cuda().requires_grad_(True) for x in xs]
    outs = [FFCzCorrect.apply(e, E, D, K, m) for e in e0s]
    for o, g in zip(reversed(outs), reversed(gs)):
        (o * g).sum().backward()
    for e, ref in zip(e0s, single):
        assert torch.equal(e.grad, ref)


@pytest.mark.parametrize("shapes,K,m", [([(16, 16, 32), (16, 32, 16), (16, 16, 32)], 5, 2),
                                        ([(32, 64), (64, 32), (32, 32), (32, 64)], 6, 4)])
@pytest.mark.parametrize("ckpt", [False, True])
def test_batched_backward_equals_single_items_and_oracle(shapes, K, m, ckpt, monkeypatch):
    """A batch of items of several shapes: each item's product is that of its
    own single-item plan, bit for bit, and matches the oracle's VJP element
    by element."""
    import torch
    import paper_2601_01596_b300 as ffcz
    monkeypatch.setenv("FFCZ_TUNE_FORCE", "split=0")
    items, gs, Es, Ds = [], [], [], []
    for i, sh in enumerate(shapes):
        e0 = W.bimodal_error(sh, 60 + i, dtype=np.float32)
        items.append(e0)
        gs.append(np.random.default_rng(61 + i).standard_normal(sh).astype(np.float32))
        Es.append(1.0 + 0.25 * i)
        Ds.append((0.3 + 0.05 * i) * O.f_violation(O.dft(e0.astype(np.float64))))
        items[-1] = (items[-1] * Es[-1]).astype(np.float32)
    te0 = torch.from_numpy(np.concatenate([x.reshape(-1) for x in items])).cuda()
    tg = torch.from_numpy(np.concatenate([x.reshape(-1) for x in gs])).cuda()
    gi = torch.empty_like(te0)
    if ckpt:
        plan = ffcz.Plan(shapes, K=K, ckpt_every=m, min_iters=K, max_iters=K, certify=0)
        ck = torch.empty(plan.ckpt_floats(), dtype=torch.float32, device="cuda")
        plan.correct_ckpt(te0.clone(), Es, Ds, ck)
        plan.backward(te0, tg, gi, Es, Ds, ckpt=ck)
    else:
        plan = ffcz.Plan(shapes, K=K, ckpt_every=m)
        plan.backward(te0, tg, gi, Es, Ds)
    got = gi.cpu().numpy()
    off = 0
    for i, sh in enumerate(shapes):
        n = int(np.prod(sh))
        one = _gpu_backward(sh, items[i], gs[i], Es[i], Ds[i], K, m, ckpt=ckpt)
        assert np.array_equal(got[off:off + n].reshape(sh), one), (i, sh)
        off += n
    # the oracle once per distinct item (the repeated shape has its own data)
    off = 0
    for i, sh in enumerate(shapes):
        n = int(np.prod(sh))
        _assert_vjp_elementwise(got[off:off + n].reshape(sh), items[i], gs[i], Es[i], Ds[i], K,
                                f"batch item {i} {sh}", samples=4)
        off += n


def test_batched_autograd_function_runs_and_matches_backward():
    import torch
    from paper_2601_01596_b300.autograd import correct_differentiable_batch
    import paper_2601_01596_b300 as ffcz
    shapes = [(16, 16, 32), (32, 16, 16)]
    items = [W.bimodal_error(sh, 70 + i, dtype=np.float32) for i, sh in enumerate(shapes)]
    Es = [1.0, 1.0]
    Ds = [0.4 * O.f_violation(O.dft(x.astype(np.float64))) for x in items]
    e0 = torch.from_numpy(np.concatenate([x.reshape(-1) for x in items])).cuda().requires_grad_(True)
    e = correct_differentiable_batch(e0, shapes, Es, Ds, K=4, ckpt_every=2)
    w = torch.from_numpy(np.random.default_rng(71).standard_normal(e.numel()).astype(np.float32)).cuda()
    (e * w).sum().backward()
    plan = ffcz.Plan(shapes, K=4, ckpt_every=2)
    gi = torch.empty_like(e0)
    plan.backward(e0.detach(), w, gi, Es, Ds)
    assert torch.equal(e0.grad, gi)


@pytest.mark.parametrize("shape,K,m", [((3000,), 5, 2), ((1500,), 6, 4), ((9000,), 3, 10)])
@pytest.mark.parametrize("ckpt", [False, True])
def test_1d_backward_matches_oracle_vjp(shape, K, m, ckpt):
    """1D items: the transposed step on the Bluestein passes, element by
    element against the oracle's VJP (near ties excused as above)."""
    e0 = W.bimodal_error(shape, 55, dtype=np.float32)
    E = 1.0
    D = 0.4 * O.f_violation(O.dft(e0.astype(np.float64)))
    g = np.random.default_rng(56).standard_normal(shape).astype(np.float32)
    got = _gpu_backward(shape, e0, g, E, D, K, m, ckpt=ckpt)
    _assert_vjp_elementwise(got, e0, g, E, D, K, f"1d{shape} K={K} ckpt={ckpt}")


def test_1d_batched_backward_equals_single_items():
    import torch
    import paper_2601_01596_b300 as ffcz
    shapes = [(3000,), (1500,), (3000,)]
    K, m = 4, 2
    items = [W.bimodal_error(sh, 57 + i, dtype=np.float32) for i, sh in enumerate(shapes)]
    gs = [np.random.default_rng(58 + i).standard_normal(sh).astype(np.float32) for i, sh in enumerate(shapes)]
    Es = [1.0] * 3
    Ds = [0.4 * O.f_violation(O.dft(x.astype(np.float64))) for x in items]
    te0 = torch.from_numpy(np.concatenate(items)).cuda()
    tg = torch.from_numpy(np.concatenate(gs)).cuda()
    gi = torch.empty_like(te0)
    plan = ffcz.Plan(shapes, K=K, ckpt_every=m)
    plan.backward(te0, tg, gi, Es, Ds)
    got = gi.cpu().numpy()
    off = 0
    for i, sh in enumerate(shapes):
        one = _gpu_backward(sh, items[i], gs[i], Es[i], Ds[i], K, m)
        assert np.array_equal(got[off:off + sh[0]], one), i
        off += sh[0]


@pytest.mark.parametrize("shapes,K,m", [([(16, 16, 32)], 6, 2), ([(32, 64), (64, 32), (32, 64)], 5, 10),
                                        ([(256, 8, 256)], 12, 4), ([(3000,), (1500,), (3001,)], 6, 4)])
def test_kept_masks_backward_equals_replay(shapes, K, m):
    """opts.keep_masks: the forward keeps every step's masks and the backward
    skips the segment replays; the product is the replayed one, bit for bit."""
    import torch
    import paper_2601_01596_b300 as ffcz
    items = [W.bimodal_error(sh, 80 + i, dtype=np.float32) for i, sh in enumerate(shapes)]
    gs = [np.random.default_rng(81 + i).standard_normal(sh).astype(np.float32) for i, sh in enumerate(shapes)]
    Es = [1.0] * len(shapes)
    Ds = [0.4 * O.f_violation(O.dft(x.astype(np.float64))) for x in items]
    te0 = torch.from_numpy(np.concatenate([x.reshape(-1) for x in items])).cuda()
    tg = torch.from_numpy(np.concatenate([x.reshape(-1) for x in gs])).cuda()
    out = {}
    for keep in (0, 1):
        plan = ffcz.Plan(shapes, K=K, ckpt_every=m, min_iters=K, max_iters=K, certify=0, keep_masks=keep)
        ck = torch.empty(plan.ckpt_floats(), dtype=torch.float32, device="cuda")
        e = te0.clone()
        plan.correct_ckpt(e, Es, Ds, ck)
        gi = torch.empty_like(te0)
        plan.backward(te0, tg, gi, Es, Ds, ckpt=ck)
        out[keep] = (e.cpu().numpy(), gi.cpu().numpy())
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert np.abs(out[1][1]).max() > 0
