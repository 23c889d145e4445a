"""The deposit's quantised charges are rint(x) for 0 <= x < 2^41 (x = beta 2^40 or
beta offset 2^40), formed on the GPU as two 32-bit words, value = hi 2^32 + lo, from FP32
operations: hf = floor(x 2^-32); hi from the bits of hf + 2^23; lo the conversion of
x - hf 2^32 to an unsigned integer with ties to even.  Written out here step for step in
float32 numpy and held to rint in float64 (exact for these values) over every float of the
binades where the rule could go wrong -- [1/2, 2) (rint's ties around 1/2 and 3/2),
[2^22, 2^24) (the last binades where rint rounds), [2^31, 2^33) (hi begins) and
[2^40, 2^41) (the top) -- and over every 61st float of the rest of [0, 2^41)."""
import numpy as np

TOP = np.float32(2.0 ** 41)


def split(x):
    """hi, lo of the rule, from float32 x >= 0."""
    hf = np.floor(x * np.float32(2.0 ** -32))  # exact scaling, then floor: an integer < 2^9
    hi = (hf + np.float32(2.0 ** 23)).view(np.uint32) - np.uint32(0x4B000000)
    lf = x - hf * np.float32(2.0 ** 32)  # both steps exact, as the fused multiply-add
    assert (lf >= 0).all() and (lf < np.float32(2.0 ** 32)).all()
    lo = np.rint(lf)  # ties to even
    return hi.astype(np.uint64), lo.astype(np.uint64), hf


def check_bits(bits):
    x = bits.view(np.float32)
    hi, lo, hf = split(x)
    assert (hi == hf.astype(np.uint64)).all()
    got = (hi << np.uint64(32)) | lo
    want = np.rint(x.astype(np.float64)).astype(np.uint64)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, (x[bad[:5]], got[bad[:5]], want[bad[:5]])


def f32_bits(v):
    return int(np.float32(v).view(np.uint32))


def binade_range(lo_val, hi_val, step=1):
    a, b = f32_bits(lo_val), f32_bits(hi_val)
    for s in range(a, b, 1 << 22):
        yield np.arange(s, min(b, s + (1 << 22)), step, dtype=np.uint32)


def test_every_float_of_the_critical_binades():
    for lo_val, hi_val in ((0.5, 2.0), (2.0 ** 22, 2.0 ** 24), (2.0 ** 31, 2.0 ** 33),
                           (2.0 ** 40, 2.0 ** 41)):
        for bits in binade_range(lo_val, hi_val):
            check_bits(bits)


def test_a_strided_sample_of_all_of_0_to_2_pow_41():
    for bits in binade_range(0.0, TOP, step=61):
        check_bits(bits)
    check_bits(np.array([0, 1, f32_bits(0.5), f32_bits(1.5), f32_bits(2.5),
                         f32_bits(8388607.5), f32_bits(2.0 ** 32 - 256), f32_bits(2.0 ** 32),
                         f32_bits(TOP) - 1], dtype=np.uint32))
