"""The path kernels form their FP32 uniform u = ((w >> 9) + 1/2) 2^-23 from a
Philox word without an int-to-float conversion: the float with mantissa bits
w >> 9 and exponent 0 is 1 + (w >> 9) 2^-23, and subtracting 1 - 2^-24 is
exact (Sterbenz), so both forms give the same float.  Checked here for every
one of the 2^23 mantissas with IEEE single-precision arithmetic (numpy), so
the kernels' uniforms are those of the oracle's closed form bit for bit."""
import numpy as np


def test_bit_built_uniform_equals_closed_form_for_every_mantissa():
    m = np.arange(1 << 23, dtype=np.uint32)
    one_plus = (m | np.uint32(0x3F800000)).view(np.float32)
    u_bits = one_plus - np.float32(1.0 - 2.0**-24)
    u_ref = (m.astype(np.float64) + 0.5) * 2.0**-23  # exact in FP64
    assert u_bits.dtype == np.float32
    assert np.array_equal(u_bits.astype(np.float64), u_ref)
    assert u_bits.min() > 0 and u_bits.max() < 1
