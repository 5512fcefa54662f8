"""The Ozaki digit cut of ozaki.cu, restated on the CPU: adding 128 in each of the six low
byte positions of the 56-bit integer F and reading the bytes gives the balanced base-256
digits of F (every low digit in [-128, 127], the top one in [-128, 128]) that a carry loop
produces, and a byte permuted into the bits of 2^23 minus (2^23 + 128) is the digit's exact
FP32 value.  CPU only."""
import struct

import numpy as np
import pytest


def f_of(x, E):
    """F = round(x 2^(56 - (E - 1021))) with E >= the biased exponent of x (the row's)."""
    u = struct.unpack("<Q", struct.pack("<d", x))[0]
    hi = u >> 32
    ea = (hi >> 20) & 0x7FF
    m = u & ((1 << 52) - 1)
    if ea:
        m |= 1 << 52
    sh = max(ea, 1) - E + 2
    if sh >= 0:
        F = m << sh
    elif sh > -60:
        F = (m + (1 << (-sh - 1))) >> (-sh)
    else:
        F = 0
    return -F if hi & 0x80000000 else F


def digits_carry_loop(F):
    d = [0] * 7
    for s in range(6, -1, -1):
        v = F & 0xFF
        if v >= 128:
            v -= 256
        d[s] = v
        F = (F - v) >> 8
    d[0] += F * 256
    return d


def digits_byte_add(F):
    G = (F + 0x808080808080) & ((1 << 64) - 1)
    g0, g1 = G & 0xFFFFFFFF, G >> 32
    bias = np.float32(8388736.0)  # 2^23 + 128

    def fbyte(word, k):
        bits = 0x4B000000 | ((word >> (8 * k)) & 0xFF)
        return float(np.float32(struct.unpack("<f", struct.pack("<I", bits))[0]) - bias)

    top = (g1 - (1 << 32) if g1 >= 1 << 31 else g1) >> 16
    d0 = float(np.float32(struct.unpack("<f", struct.pack("<I", (top + 0x4B000000 + 128) & 0xFFFFFFFF))[0]) - bias)
    return [d0, fbyte(g1, 1), fbyte(g1, 0), fbyte(g0, 3), fbyte(g0, 2), fbyte(g0, 1), fbyte(g0, 0)]


def biased_exp(x):
    return (struct.unpack("<Q", struct.pack("<d", x))[0] >> 52) & 0x7FF


@pytest.mark.parametrize("seed", range(4))
def test_byte_add_gives_the_balanced_digits(seed):
    rng = np.random.default_rng(seed)
    cases = [0.0, -0.0, 1.0, -1.0, 0.5, np.nextafter(2.0, 0.0), -np.nextafter(2.0, 0.0), 5e-324, -5e-324]
    xs = cases + list(rng.standard_normal(3000) * 2.0 ** rng.integers(-40, 40, 3000))
    for x in xs:
        e = biased_exp(x)
        for E in {max(e, 1), max(e, 1) + 1, max(e, 1) + 9, max(e, 1) + 57, max(e, 1) + 70}:
            if E > 2046:
                continue
            F = f_of(float(x), E)
            assert abs(F) < 2 ** 55
            ref = digits_carry_loop(F)
            got = digits_byte_add(F)
            assert got == [float(v) for v in ref], (x, E)
            assert all(-128 <= v <= 127 for v in got[1:]) and -128 <= got[0] <= 128
            assert sum(int(v) * 256 ** (6 - s) for s, v in enumerate(got)) == F


def test_a_carry_slip_is_caught():
    F = f_of(0.7071, biased_exp(0.7071))
    wrong = digits_byte_add(F + 0x80)  # one digit position off
    assert sum(int(v) * 256 ** (6 - s) for s, v in enumerate(wrong)) != F
