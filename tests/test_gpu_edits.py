"""Alg. 1 edits recorded by the GPU loop (opts.edits) vs the FP64 oracle.

Bars: after k forced iterations the dense spatial edits match the oracle's
to 1e-3 eps_s and the frequency edits to 1e-3 eps_f (plus float32 rounding of
the spectrum); the GPU's own output satisfies e_out - e_in = S + IFFT(F) to
1e-4 eps_s (in converged runs too, where the stopping check's clip must not be
recorded); flags and codes are bit-exact against the oracle's CompactEdits /
QuantizeEdits applied to the GPU's float32 edits in float32.
"""
import numpy as np
import pytest

from oracle import ffcz_oracle as O
from paper_2601_01596_b300 import workloads as W

pytestmark = pytest.mark.gpu


def stress(shape, seed, frac=0.4):
    e0 = W.bimodal_error(shape, seed, E=1.0, dtype=np.float32)
    return e0, 1.0, frac * O.f_violation(O.dft(e0.astype(np.float64)))


def run(items, Es, Ds, **opts):
    import torch
    import paper_2601_01596_b300 as ffcz
    shapes = [x.shape for x in items]
    plan = ffcz.Plan(shapes, edits=1, **opts)
    t = torch.from_numpy(np.concatenate([x.reshape(-1) for x in items]).astype(np.float32)).cuda()
    st = plan.correct(t, Es, Ds)
    S, F = plan.edits_dense()
    torch.cuda.synchronize()
    return plan, t.cpu().numpy(), st, S.cpu().numpy(), F.cpu().numpy()


def split(plan, S, F, shapes):
    out = []
    for i, sh in enumerate(shapes):
        npt, nb, *_ = plan.edit_layout(i)
        s0 = sum(plan.edit_layout(j)[0] for j in range(i))
        f0 = sum(plan.edit_layout(j)[1] for j in range(i))
        half = tuple(sh[:-1]) + (sh[-1] // 2 + 1,)
        out.append((S[s0:s0 + npt].reshape(sh), F[f0:f0 + nb].reshape(half)))
    return out


@pytest.mark.parametrize("shape,k", [((32, 32, 32), 3), ((64, 128), 4), ((16, 32, 64), 2), ((3000,), 3),
                                     ((1500,), 4)])
def test_forced_iterations_edits_match_oracle(shape, k):
    e0, E, D = stress(shape, 70)
    ref = O.correct(e0, E, D, min_iters=k, max_iters=k, edits=True)
    plan, e, st, S, F = run([e0], [E], [D], min_iters=k, max_iters=k, certify=0)
    assert st[0]["iters"] == k
    (Sg, Fg), = split(plan, S, F, [shape])
    np.testing.assert_allclose(Sg, ref.spat_edits, rtol=0, atol=1e-3 * E)
    Fh = O.half_spectrum(ref.freq_edits)
    np.testing.assert_allclose(Fg, Fh, rtol=0, atol=1e-3 * D + 1e-5 * np.max(np.abs(Fh)))
    assert np.count_nonzero(Sg) > 0 and np.count_nonzero(Fg) > 0
    # the GPU's own trajectory: e_k - e_0 = S + IFFT(F)
    disp = Sg.astype(np.float64) + np.fft.irfftn(Fg.astype(np.complex128), s=shape, axes=tuple(range(len(shape))))
    np.testing.assert_allclose(e.reshape(shape) - e0, disp, rtol=0, atol=1e-4 * E)


@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 128), (256, 64), (3000,), (9000,)])
def test_converged_run_drops_the_stopping_clip(shape):
    e0, E, D = stress(shape, 71)
    plan, e, st, S, F = run([e0], [E], [D])
    assert st[0]["status"] == 0 and st[0]["iters"] >= 2 and st[0]["certified"] == 1
    (Sg, Fg), = split(plan, S, F, [shape])
    disp = Sg.astype(np.float64) + np.fft.irfftn(Fg.astype(np.complex128), s=shape, axes=tuple(range(len(shape))))
    np.testing.assert_allclose(e.reshape(shape) - e0, disp, rtol=0, atol=1e-4 * E)


def test_preclip_recorded_as_spatial_edit():
    e0, E, D = stress((32, 64), 72)
    e0 = e0.copy(); e0[3, 5] = 1.75; e0[20, 7] = -2.5
    plan, e, st, S, F = run([e0], [E], [D])
    assert st[0]["preclipped"] == 1
    (Sg, Fg), = split(plan, S, F, [(32, 64)])
    disp = Sg.astype(np.float64) + np.fft.irfftn(Fg.astype(np.complex128), s=(32, 64), axes=(0, 1))
    np.testing.assert_allclose(e.reshape(32, 64) - e0, disp, rtol=0, atol=1e-4 * E)


def test_compaction_bit_exact_against_oracle_quantizer():
    shapes = [(32, 32, 32), (16, 32, 64), (32, 32, 32)]
    items, Es, Ds = [], [], []
    for i, sh in enumerate(shapes):
        e0, E, D = stress(sh, 73 + i)
        items.append(e0); Es.append(E * (1 + 0.5 * i)); Ds.append(D * (1 + 0.25 * i))
        items[-1] = (items[-1] * (1 + 0.5 * i)).astype(np.float32)
    plan, e, st, S, F = run(items, Es, Ds)
    for m in (16, 12):
        c = plan.edits_compact(m)
        sf, sc = c["s_flags"].cpu().numpy(), c["s_codes"].cpu().numpy()
        ff, fc = c["f_flags"].cpu().numpy(), c["f_codes"].cpu().numpy()
        for i, (Sg, Fg) in enumerate(split(plan, S, F, shapes)):
            npt, nb, so, sco, fo, fco = plan.edit_layout(i)
            flags, comp = O.compact_edits(Sg)
            np.testing.assert_array_equal(sf[so:so + flags.size], flags)
            assert c["counts"][i, 0] == comp.size
            want = O.quantize_edits(comp.astype(np.float32), Es[i], m, dtype=np.float32)
            np.testing.assert_array_equal(sc[sco:sco + comp.size], want)
            flags, comp = O.compact_edits(Fg)
            np.testing.assert_array_equal(ff[fo:fo + flags.size], flags)
            assert c["counts"][i, 1] == comp.size
            want = O.quantize_edits(comp.astype(np.complex64), Ds[i], m, dtype=np.float32)
            np.testing.assert_array_equal(fc[fco:fco + 2 * comp.size].reshape(-1, 2), want)


def test_preclip_recorded_as_spatial_edit_1d():
    e0, E, D = stress((3000,), 74)
    e0 = e0.copy(); e0[17] = 1.75; e0[2900] = -2.5
    plan, e, st, S, F = run([e0], [E], [D])
    assert st[0]["preclipped"] == 1
    (Sg, Fg), = split(plan, S, F, [(3000,)])
    assert Sg[17] != 0 and Sg[2900] != 0
    disp = Sg.astype(np.float64) + np.fft.irfft(Fg.astype(np.complex128), n=3000)
    np.testing.assert_allclose(e - e0, disp, rtol=0, atol=1e-4 * E)


def test_compaction_bit_exact_against_oracle_quantizer_1d():
    shapes = [(3000,), (1500,), (9000,)]
    items, Es, Ds = [], [], []
    for i, sh in enumerate(shapes):
        e0, E, D = stress(sh, 75 + i)
        items.append(e0); Es.append(E); Ds.append(D)
    plan, e, st, S, F = run(items, Es, Ds)
    c = plan.edits_compact(16)
    sf, sc = c["s_flags"].cpu().numpy(), c["s_codes"].cpu().numpy()
    ff, fc = c["f_flags"].cpu().numpy(), c["f_codes"].cpu().numpy()
    for i, (Sg, Fg) in enumerate(split(plan, S, F, shapes)):
        npt, nb, so, sco, fo, fco = plan.edit_layout(i)
        assert (npt, nb) == (shapes[i][0], shapes[i][0] // 2 + 1)
        flags, comp = O.compact_edits(Sg)
        np.testing.assert_array_equal(sf[so:so + flags.size], flags)
        np.testing.assert_array_equal(sc[sco:sco + comp.size],
                                      O.quantize_edits(comp.astype(np.float32), Es[i], 16, dtype=np.float32))
        flags, comp = O.compact_edits(Fg)
        np.testing.assert_array_equal(ff[fo:fo + flags.size], flags)
        np.testing.assert_array_equal(fc[fco:fco + 2 * comp.size].reshape(-1, 2),
                                      O.quantize_edits(comp.astype(np.complex64), Ds[i], 16, dtype=np.float32))


def test_edits_off_by_default_and_plan_without_edits_refuses():
    import paper_2601_01596_b300 as ffcz
    plan = ffcz.Plan([(32, 32)])
    assert plan.edit_layout(-1)[:2] == (32 * 32, 32 * 17)     # layout exists for application
    with pytest.raises(ffcz.FFCzError):
        plan.edits_dense()
    with pytest.raises(ffcz.FFCzError):
        plan.edits_compact()


@pytest.mark.parametrize("shapes", [[(32, 32, 32)], [(64, 128), (32, 256)], [(16, 32, 64), (16, 32, 64)],
                                    [(3000,), (1500,), (9000,)]])
def test_apply_edits_matches_oracle_application(shapes):
    """Decompression side: x_hat + S~ + IFFT(F~) from the stored codes, GPU vs
    the oracle's apply_edits on the same dequantized edits."""
    import torch
    items, Es, Ds = [], [], []
    for i, sh in enumerate(shapes):
        e0, E, D = stress(sh, 80 + i)
        items.append(e0); Es.append(E); Ds.append(D)
    plan, e, st, S, F = run(items, Es, Ds)
    stored = plan.edits_compact(16)
    rng = np.random.default_rng(81)
    xs = [rng.standard_normal(sh) for sh in shapes]
    xhat = np.concatenate([(x + e0).reshape(-1) for x, e0 in zip(xs, items)]).astype(np.float32)
    t = torch.from_numpy(xhat.copy()).cuda()
    plan.apply_edits(t, Es, Ds, stored, 16)
    got = t.cpu().numpy()
    sf, sc = stored["s_flags"].cpu().numpy(), stored["s_codes"].cpu().numpy()
    ff, fc = stored["f_flags"].cpu().numpy(), stored["f_codes"].cpu().numpy()
    off = 0
    for i, sh in enumerate(shapes):
        npt, nb, so, sco, fo, fco = plan.edit_layout(i)
        ns, nf = stored["counts"][i]
        half = tuple(sh[:-1]) + (sh[-1] // 2 + 1,)
        Sq = O.expand_edits(sf[so:so + (npt + 7) // 8],
                            O.dequantize_edits(sc[sco:sco + ns], Es[i], 16), npt).reshape(sh)
        Fq = O.expand_edits(ff[fo:fo + (nb + 7) // 8],
                            O.dequantize_edits(fc[fco:fco + 2 * nf].reshape(-1, 2), Ds[i], 16, complex_pairs=True),
                            nb).reshape(half)
        want = O.apply_edits(xhat[off:off + npt].reshape(sh).astype(np.float64), Sq, Fq)
        scale = np.max(np.abs(want))
        np.testing.assert_allclose(got[off:off + npt].reshape(sh), want, rtol=0, atol=2e-6 * scale)
        # and the round trip lands within quantization error of x + e_out
        np.testing.assert_allclose(got[off:off + npt].reshape(sh), xs[i] + e[off:off + npt].reshape(sh),
                                   rtol=0, atol=1e-3 * Es[i] + 2e-6 * scale)
        off += npt


@pytest.mark.parametrize("shape,seed,frac", [((32, 32, 32), 3, 0.4), ((64, 128), 5, 0.4), ((16, 32, 64), 7, 0.2),
                                            ((3000,), 9, 0.3)])
def test_decompressed_field_certifies_with_the_doubled_shrink(shape, seed, frac):
    """Reading A21 on the library: corrected with shrink 2^(1-m), the field
    rebuilt from the stored m-bit edits (x_hat + S~ + IFFT(F~), here with
    x = 0 so that x_hat is e0) passes the FP64 certification against the
    true bounds."""
    import torch
    import paper_2601_01596_b300 as ffcz
    e0 = W.bimodal_error(shape, seed, E=1.0, dtype=np.float32)
    E, D, m = 1.0, frac * O.f_violation(O.dft(e0.astype(np.float64))), 16
    plan = ffcz.Plan([shape], edits=1, shrink=2.0 ** (1 - m))
    t = torch.from_numpy(e0.reshape(-1).copy()).cuda()
    st = plan.correct(t, [E], [D])[0]
    assert st["certified"] == 1 and st["iters"] >= 2
    stored = plan.edits_compact(m)
    xhat = torch.from_numpy(e0.reshape(-1).copy()).cuda()
    plan.apply_edits(xhat, [E], [D], stored, m)
    chk = plan.check(xhat, [E], [D])[0]
    assert chk["certified"] == 1, chk


@pytest.mark.parametrize("shapes", [[(32, 32, 32), (16, 32, 64)], [(64, 128), (32, 256)], [(3000,), (1500,)]])
def test_16bit_codes_bit_exact_against_oracle_and_apply_equals_int32_form(shapes):
    """Codes stored in 16 bits with escapes (Sec. IV-B, m = 16; reading A27):
    int16 codes and escape lists equal the oracle's narrowing of the oracle
    quantiser's codes, and applying the 16-bit form gives the same bits as
    applying the int32 form."""
    import torch
    items, Es, Ds = [], [], []
    for i, sh in enumerate(shapes):
        e0, E, D = stress(sh, 90 + i, frac=0.2)
        items.append(e0); Es.append(E); Ds.append(D)
    plan, e, st, S, F = run(items, Es, Ds)
    c16 = plan.edits_compact16(16)
    c32 = plan.edits_compact(16)
    sc, sw = c16["s_codes"].cpu().numpy(), c16["s_wide"].cpu().numpy()
    fc, fw = c16["f_codes"].cpu().numpy(), c16["f_wide"].cpu().numpy()
    np.testing.assert_array_equal(c16["s_flags"].cpu().numpy(), c32["s_flags"].cpu().numpy())
    np.testing.assert_array_equal(c16["f_flags"].cpu().numpy(), c32["f_flags"].cpu().numpy())
    n_esc = 0
    for i, (Sg, Fg) in enumerate(split(plan, S, F, shapes)):
        npt, nb, so, sco, fo, fco = plan.edit_layout(i)
        _, comp = O.compact_edits(Sg)
        want16, wantw = O.narrow_codes(O.quantize_edits(comp.astype(np.float32), Es[i], 16, dtype=np.float32))
        assert tuple(c16["counts"][i, [0, 2]]) == (comp.size, wantw.size)
        np.testing.assert_array_equal(sc[sco:sco + comp.size], want16)
        np.testing.assert_array_equal(sw[sco:sco + wantw.size], wantw)
        _, comp = O.compact_edits(Fg)
        codes = O.quantize_edits(comp.astype(np.complex64), Ds[i], 16, dtype=np.float32).reshape(-1)
        want16, wantw = O.narrow_codes(codes)
        assert tuple(c16["counts"][i, [1, 3]]) == (comp.size, wantw.size)
        np.testing.assert_array_equal(fc[fco:fco + codes.size], want16)
        np.testing.assert_array_equal(fw[fco:fco + wantw.size], wantw)
        n_esc += wantw.size
    assert n_esc > 0   # the stress bounds make frequency edits larger than the bound
    rng = np.random.default_rng(91)
    xhat = np.concatenate([(rng.standard_normal(sh) + x).reshape(-1) for sh, x in zip(shapes, items)])
    t16 = torch.from_numpy(xhat.astype(np.float32)).cuda()
    t32 = t16.clone()
    plan.apply_edits16(t16, Es, Ds, c16, 16)
    plan.apply_edits(t32, Es, Ds, c32, 16)
    assert torch.equal(t16, t32)


def test_16bit_codes_refuse_bad_counts_and_m_bits():
    import torch
    import paper_2601_01596_b300 as ffcz
    e0, E, D = stress((32, 32), 95, frac=0.2)
    plan, e, st, S, F = run([e0], [E], [D])
    with pytest.raises(ffcz.FFCzError):
        plan.edits_compact16(17)
    c16 = plan.edits_compact16(16)
    x = torch.zeros(32 * 32, dtype=torch.float32, device="cuda")
    bad = dict(c16)
    bad["counts"] = c16["counts"].copy()
    bad["counts"][0, 3] += 1          # one escape more than the codes hold
    with pytest.raises(ffcz.FFCzError):
        plan.apply_edits16(x, [E], [D], bad, 16)
    assert float(x.abs().max()) == 0.0   # nothing applied
    bad["counts"] = c16["counts"].copy()
    bad["counts"][0, 0] = 32 * 32 + 1   # more nonzero points than the item has
    with pytest.raises(ffcz.FFCzError):
        plan.apply_edits16(x, [E], [D], bad, 16)
