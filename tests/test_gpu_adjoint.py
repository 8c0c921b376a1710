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
