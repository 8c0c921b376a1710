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
