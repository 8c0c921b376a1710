"""The bound shrink and the quantised edits (Sec. IV-B, "Compaction,
quantization ..."; reading A21), on the oracle.

The paper shrinks E and Delta by 2^-m so that the QUANTISED edits still move
the error into the feasible region.  The decompressed error is e0 + S~ +
IFFT(F~) with S~, F~ the dequantised edits.  Its rounding against the exact
edits is up to q/2 = bound 2^-m per component, plus the inverse transform of
the frequency codes' rounding, so the margin 2^-m that the paper's shrink
leaves is used up by the spatial rounding alone.  With the shrink doubled to
2^(1-m) the decompressed field is feasible on every stress case here, while
at 2^-m it lands just outside (by a few 1e-6 relative).
"""
import numpy as np
import pytest

from oracle import ffcz_oracle as O
from paper_2601_01596_b300 import workloads as W


def decompressed(e0, E, D, eta, m=16):
    """Correct with shrink eta, store the edits (flags + m-bit codes),
    apply them to the base error: the decompressed error x_hat' - x."""
    r = O.correct(e0, E, D, eta=eta, edits=True)
    fS, cS = O.compact_edits(r.spat_edits)
    Fh = O.half_spectrum(r.freq_edits)
    fF, cF = O.compact_edits(Fh)
    S = O.expand_edits(fS, O.dequantize_edits(O.quantize_edits(cS, E, m), E, m), r.spat_edits.size)
    F = O.expand_edits(fF, O.dequantize_edits(O.quantize_edits(cF, D, m), D, m, complex_pairs=True), Fh.size)
    return O.apply_edits(np.asarray(e0, np.float64), S.reshape(e0.shape), F.reshape(Fh.shape)), r


CASES = {
    "bimodal32^3": lambda: (W.bimodal_error((32, 32, 32), 3, E=1.0, dtype=np.float32), 1.0, 0.4),
    "bimodal64x128": lambda: (W.bimodal_error((64, 128), 5, E=1.0, dtype=np.float32), 1.0, 0.4),
    "bimodal16x32x64": lambda: (W.bimodal_error((16, 32, 64), 7, E=1.0, dtype=np.float32), 1.0, 0.2),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_doubled_shrink_makes_the_decompressed_field_feasible(name):
    e0, E, frac = CASES[name]()
    D = frac * O.f_violation(O.dft(e0.astype(np.float64)))
    m = 16
    # the paper's shrink 2^-m: the exact edits are feasible, the quantised
    # ones land just outside (A21)
    e_dec, r = decompressed(e0, E, D, 2.0 ** -m, m)
    assert r.iters >= 2 and O.certify(r.e, E, D)[0]
    ok, s, v = O.certify(e_dec, E, D)
    assert not ok and max(s / E, v / D) < 1 + 2e-5
    # shrink 2^(1-m): feasible after quantisation
    e_dec, r = decompressed(e0, E, D, 2.0 ** (1 - m), m)
    ok, s, v = O.certify(e_dec, E, D)
    assert ok, (s / E, v / D)
