"""Full-size parity (512^3 lognormal, the workload and launch configuration
the benchmark times).

As written the field converges in 0 iterations: the output must equal the
input (apart from the A3 pre-clip of points the float32 cast put outside the
s-cube), pass the FP64 certification, and randomly sampled DFT bins computed
here by direct FP64 sums must lie within the bound.  The labelled stress
variant (eps_f = 0.2 max box violation of e0) iterates; it is compared with
the FP64 oracle run on the whole field: max|delta e| <= 1e-3 eps_s and the
iteration count within +-2.
"""
import numpy as np
import pytest

from oracle import ffcz_oracle as O
from paper_2601_01596_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _gpu(e0, E, D):
    import torch
    import paper_2601_01596_b300 as ffcz
    plan = ffcz.Plan([e0.shape])          # tuned variants, as the benchmark runs them
    t = torch.from_numpy(e0.reshape(-1).copy()).cuda()
    st = plan.correct(t, [E], [D])[0]
    return t.cpu().numpy().reshape(e0.shape), st


def _bin(e, k):
    """delta_k = sum_n e_n exp(-2 pi i k.n / N) by separable direct sums (FP64)."""
    n = e.shape[0]
    w = [np.exp(-2j * np.pi * kk * np.arange(n) / n) for kk in k]
    return np.einsum("zyx,x->zy", e, w[2], optimize=True) @ w[1] @ w[0]


def test_lognormal512_as_written_full_size():
    it = W.lognormal_field(512)
    e0, E, D = it["e0"], it["E"], it["D"]
    e, st = _gpu(e0, E, D)
    assert st["status"] == 0 and st["iters"] == 0 and st["certified"] == 1
    if st["preclipped"]:
        moved = e != e0
        assert np.all(np.abs(e0[moved]) > E) and np.all(np.abs(e[moved]) <= E)
        assert np.array_equal(e[~moved], e0[~moved])
    else:
        assert np.array_equal(e, e0)
    assert float(np.max(np.abs(e))) <= E
    ed = e.astype(np.float64)
    rng = np.random.default_rng(100)
    ks = [(0, 0, 0), (1, 0, 0), (0, 0, 256), (256, 256, 256)] + \
         [tuple(int(v) for v in rng.integers(0, 512, 3)) for _ in range(8)]
    for k in ks:
        d = _bin(ed, k)
        assert abs(d.real) <= D and abs(d.imag) <= D, k


def test_lognormal512_stress_matches_oracle_full_size():
    it = W.lognormal_field(512, stress=0.2)
    e0, E, D = it["e0"], it["E"], it["D"]
    e, st = _gpu(e0, E, D)
    ref = O.correct(e0, E, D)
    assert ref.iters >= 2 and abs(st["iters"] - ref.iters) <= 2
    assert st["status"] == 0 and st["certified"] == 1
    assert float(np.max(np.abs(e.astype(np.float64) - ref.e))) <= 1e-3 * E


@pytest.mark.parametrize("shape", [(512, 64, 512), (64, 512, 512)])
def test_each_of_first_ten_iterations_on_the_bench_kernels(shape, monkeypatch):
    """After each forced iteration k = 1..10, element by element against the
    oracle, on the kernels that produce the 512^3 numbers: the variants the
    tuner picks there are pinned (the copy-engine-fed persistent passes, in
    their lean forward forms), and these shapes run them at the same template
    sizes -- (512, 64, 512): the 512-point z check pass and the 512-real x
    pass; (64, 512, 512): the 512-point y passes and the x pass.  Input: the
    512^3 workload's recipe on this shape (lognormal of a P(k) ~ k^-2.5 GRF,
    quantisation error at eps_s = 1e-4 range) with the stress bound eps_f =
    0.2 max box violation so that every clip is active."""
    import torch
    import paper_2601_01596_b300 as ffcz
    monkeypatch.setenv("FFCZ_TUNE_FORCE", "px=tma,axis=tma,chk=tma")
    g = W.grf(shape, 2.5, 0)
    x = np.exp(g).astype(np.float32)
    del g
    E = 1e-4 * (float(x.max()) - float(x.min()))
    e0 = W.quantization_error(x, E)
    D = 0.2 * W.max_box_fft(e0)
    del x
    t0 = torch.from_numpy(e0.reshape(-1).copy()).cuda()
    ref = e0
    worst = 0.0
    for k in range(1, 11):
        ref = O.correct(ref, E, D, min_iters=1, max_iters=1).e     # one more oracle iteration
        plan = ffcz.Plan([shape], min_iters=k, max_iters=k, certify=0)
        if k == 1:
            desc = plan.describe()
            assert "px=tma" in desc, desc
            assert ("chk=tma" in desc) == (shape[0] == 512) and ("axis=tma" in desc) == (shape[1] == 512), desc
        t = t0.clone()
        st = plan.correct(t, [E], [D])[0]
        assert st["iters"] == k
        err = float(np.max(np.abs(t.cpu().numpy().reshape(shape).astype(np.float64) - ref)))
        worst = max(worst, err / E)
        assert err <= 1e-3 * E, (k, err / E)
    print(f"{shape}: max|de|/eps_s over iterations 1..10 = {worst:.2e}")
