"""16-bit storage of the quantised edits (Sec. IV-B: codes of m bits,
m = 16), on the oracle.  Reading A27: a code in [-32767, 32767] is stored as
itself, any other as the escape -32768 with its value appended to an int32
list in order of appearance.
"""
import numpy as np

from oracle import ffcz_oracle as O
from paper_2601_01596_b300 import workloads as W


def test_hand_written_example():
    codes = [0, 1, -1, 32767, -32767, 32768, -32768, 100000, -5, -70000]
    c16, wide = O.narrow_codes(codes)
    assert c16.dtype == np.int16 and wide.dtype == np.int32
    assert c16.tolist() == [0, 1, -1, 32767, -32767, -32768, -32768, -32768, -5, -32768]
    assert wide.tolist() == [32768, -32768, 100000, -70000]
    assert O.widen_codes(c16, wide).tolist() == codes


def test_end_points_of_the_cube_escape_at_m16():
    """q = 2E/2^16: an edit equal to +-E is the code +-2^15, outside int16's
    symmetric range, and escapes; one step inside does not."""
    E = np.float32(0.75)
    q = O.quant_step(E, 16, np.float32)
    edits = np.array([E, -E, E - q, -(E - q), np.float32(3) * E], dtype=np.float32)
    codes = O.quantize_edits(edits, E, 16, dtype=np.float32)
    assert codes.tolist() == [32768, -32768, 32767, -32767, 98304]
    c16, wide = O.narrow_codes(codes)
    assert c16.tolist() == [-32768, -32768, 32767, -32767, -32768]
    assert wide.tolist() == [32768, -32768, 98304]


def test_round_trip_and_escape_count_on_random_codes():
    rng = np.random.default_rng(5)
    codes = rng.integers(-40000, 40001, size=5000)
    c16, wide = O.narrow_codes(codes)
    assert len(wide) == int(np.sum(np.abs(codes) >= 32768))
    np.testing.assert_array_equal(O.widen_codes(c16, wide), codes)


def test_planted_mistakes_are_caught():
    """Storing -32768 directly (a limit of 32768) makes it indistinguishable
    from the escape; dropping the order of the list scrambles the values."""
    codes = np.array([5, -32768, 40000, 32768])

    def narrow_wrong_limit(c):
        out, wide = [], []
        for v in c:
            if -32768 <= v <= 32767:
                out.append(v)
            else:
                out.append(-32768)
                wide.append(v)
        return np.array(out, np.int16), np.array(wide, np.int32)

    c16, wide = narrow_wrong_limit(codes)
    try:
        back = O.widen_codes(c16, wide)
    except (ValueError, IndexError):
        back = None
    assert back is None or back.tolist() != codes.tolist()
    c16, wide = O.narrow_codes(codes)
    assert not np.array_equal(O.widen_codes(c16, wide[::-1]), codes)


def test_stored_size_of_a_corrected_field():
    """The codes of a real correction: 2 bytes per code plus 4 per escape,
    below the 4 bytes per code of int32 storage, and the widened codes equal
    the quantiser's."""
    e0 = W.bimodal_error((32, 32, 32), 3, E=1.0, dtype=np.float32)
    D = 0.4 * O.f_violation(O.dft(e0.astype(np.float64)))
    r = O.correct(e0, 1.0, D, edits=True)
    for edits, bound in ((r.spat_edits, 1.0), (O.half_spectrum(r.freq_edits), D)):
        _, comp = O.compact_edits(edits)
        if np.iscomplexobj(comp):
            codes = O.quantize_edits(comp.astype(np.complex64), bound, 16, dtype=np.float32).reshape(-1)
        else:
            codes = O.quantize_edits(comp.astype(np.float32), bound, 16, dtype=np.float32)
        c16, wide = O.narrow_codes(codes)
        np.testing.assert_array_equal(O.widen_codes(c16, wide), codes)
        assert 2 * c16.size + 4 * wide.size < 4 * codes.size
