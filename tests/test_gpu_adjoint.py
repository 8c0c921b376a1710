"""Adjoint (ffcz_correct_backward) vs the oracle's vector-Jacobian product."""
import numpy as np
import pytest

from oracle import ffcz_oracle as O
from paper_2601_01596_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,K,m", [((16, 16, 32), 5, 2), ((32, 64), 6, 4), ((16, 16, 16), 3, 10)])
def test_backward_matches_oracle_vjp(shape, K, m):
    import torch
    import paper_2601_01596_b300 as ffcz
    e0 = W.bimodal_error(shape, 50, dtype=np.float32)
    E = 1.0
    D = 0.4 * O.f_violation(O.dft(e0.astype(np.float64)))
    g = np.random.default_rng(51).standard_normal(shape).astype(np.float32)
    ref = O.correct_backward(e0, g, E, D, K)
    plan = ffcz.Plan([shape], K=K, ckpt_every=m)
    te0 = torch.from_numpy(e0.reshape(-1).copy()).cuda()
    tg = torch.from_numpy(g.reshape(-1).copy()).cuda()
    gi = torch.empty_like(te0)
    plan.backward(te0, tg, gi, [E], [D])
    got = gi.cpu().numpy().reshape(shape)
    scale = np.max(np.abs(ref))
    # masks can flip for values within FP32 rounding of a bound; allow a tiny
    # fraction of outliers, require the rest to agree to FP32 accuracy
    err = np.abs(got - ref)
    assert np.mean(err > 1e-4 * scale) < 1e-3
    assert np.linalg.norm(got - ref) <= 1e-3 * np.linalg.norm(ref)


def test_autograd_function_matches_oracle_through_spectrum_loss():
    """d loss / d e0 for loss = log power-spectrum mismatch of x + e_K vs x."""
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
    g_ref = O.correct_backward(it["e0"], et.grad.numpy(), it["E"], it["D"], K)
    assert abs(loss.item() - lref.item()) <= 1e-3 * abs(lref.item()) + 1e-9
    assert np.linalg.norm(g_gpu - g_ref) <= 2e-3 * np.linalg.norm(g_ref)


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
    for force in ("px=tma", None):
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
