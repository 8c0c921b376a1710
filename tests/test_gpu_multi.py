"""Multi-group form of the loop passes: one persistent launch per pass kind
walks a work list over the members of every shape group (Alg. 1 per item).

Batches of uneven items must give the same bits with the multi-group form as
with one launch per group, match the oracle, and launch a fixed number of
kernels per iteration whatever the number of distinct shapes.
"""
import numpy as np
import pytest

from oracle import ffcz_oracle as O
from paper_2601_01596_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _batch(shapes, seed):
    items, Es, Ds = [], [], []
    for i, sh in enumerate(shapes):
        e0 = W.bimodal_error(sh, seed + i, E=1.0, dtype=np.float32)
        D = (0.3 + 0.1 * (i % 3)) * O.f_violation(O.dft(e0.astype(np.float64)))
        items.append(e0)
        Es.append(1.0)
        Ds.append(D)
    return items, Es, Ds


def _run(shapes, items, Es, Ds, monkeypatch, multi, **opts):
    import torch
    import paper_2601_01596_b300 as ffcz
    monkeypatch.setenv("FFCZ_TUNE_FORCE", f"multi={multi},split=0")
    plan = ffcz.Plan(shapes, **opts)
    desc = plan.describe()
    packed = np.concatenate([x.reshape(-1) for x in items])
    t = torch.from_numpy(packed).cuda()
    st = plan.correct(t, Es, Ds)
    torch.cuda.synchronize()
    return t.cpu().numpy(), [dict(x) for x in st], desc


CASES = {
    "2d": [(64, 64), (32, 128), (128, 256), (64, 64), (256, 32), (32, 128), (1024, 16)],
    "3d": [(16, 32, 64), (32, 16, 64), (8, 64, 32), (16, 32, 64), (32, 32, 32)],
    "1d": [(1500,), (3000,), (1500,), (9000,), (700,), (40000,)],
}


@pytest.mark.parametrize("kind", sorted(CASES))
def test_multi_group_form_equals_separate_launches_and_oracle(kind, monkeypatch):
    shapes = CASES[kind]
    items, Es, Ds = _batch(shapes, 70)
    a, sa, da = _run(shapes, items, Es, Ds, monkeypatch, 1)
    b, sb, db = _run(shapes, items, Es, Ds, monkeypatch, 0)
    assert "=multi" in da and "=multi" not in db, (da, db)
    assert np.array_equal(a, b)
    off = 0
    for i, sh in enumerate(shapes):
        n = int(np.prod(sh))
        assert sa[i]["iters"] == sb[i]["iters"] and sa[i]["certified"] == 1
        assert sa[i]["active_s"] == sb[i]["active_s"] and sa[i]["active_f"] == sb[i]["active_f"]
        ref = O.correct(items[i], Es[i], Ds[i])
        assert abs(sa[i]["iters"] - ref.iters) <= 2
        np.testing.assert_allclose(a[off:off + n].reshape(sh), ref.e, rtol=0, atol=1e-3 * Es[i])
        off += n


@pytest.mark.parametrize("kind", sorted(CASES))
def test_multi_group_launches_per_iteration_do_not_grow_with_shapes(kind, monkeypatch):
    """Direct launches (no graph), K forced iterations: the loop body of the
    multi-group form launches one kernel per pass kind plus the per-item stop
    decision, for any number of shape groups."""
    import torch
    import paper_2601_01596_b300 as ffcz
    shapes = CASES[kind]
    items, Es, Ds = _batch(shapes, 80)
    packed = np.concatenate([x.reshape(-1) for x in items])
    ngroups = len(set(shapes))
    per = {}
    for multi in (1, 0):
        monkeypatch.setenv("FFCZ_TUNE_FORCE", f"multi={multi},split=0")
        counts = []
        for K in (2, 6):
            plan = ffcz.Plan(shapes, min_iters=K, max_iters=K, certify=0, use_graph=0, chunk=1)
            t = torch.from_numpy(packed).cuda()
            plan.correct(t, Es, Ds)          # warm-up (module loads)
            t = torch.from_numpy(packed).cuda()
            l0 = ffcz.launch_count()
            plan.correct(t, Es, Ds)
            torch.cuda.synchronize()
            counts.append(ffcz.launch_count() - l0)
        per[multi] = (counts[1] - counts[0]) / 4
    kinds = {"2d": 2, "3d": 4, "1d": 4}[kind]
    extra = per[1] - kinds            # the stop decision (and any loop bookkeeping)
    assert 1 <= extra <= 2, per
    # separate launches: one per pass kind and group, the same bookkeeping
    assert per[0] == kinds * ngroups + extra, per
