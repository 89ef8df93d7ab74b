"""Pins of the oracle's random stream (Philox4x32-10 and the uniform maps).

The paper names no generator; the stream is Philox4x32-10 as defined by
Salmon et al. (SC'11).  The oracle's block function is pinned against an
independent implementation -- the host-side Philox4_32_10 generator of the
cuRAND library, which runs on the CPU -- for several keys and for counters
that exercise words c0, c1 and c2.  The uniform maps are pinned by exact
rational arithmetic.
"""
import ctypes
import ctypes.util
import math
import os
from fractions import Fraction

import numpy as np
import pytest

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so",
                 ctypes.util.find_library("curand")):
        if path and (os.path.exists(path) or not path.startswith("/")):
            try:
                return ctypes.CDLL(path)
            except OSError:
                pass
    return None


def _curand_words(lib, seed, offset_words, count):
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(
        ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(
            gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(
            gen, ctypes.c_ulonglong(offset_words)) == 0
        buf = (ctypes.c_uint32 * count)()
        assert lib.curandGenerate(gen, buf, ctypes.c_size_t(count)) == 0
        return np.array(list(buf), dtype=np.uint32)
    finally:
        lib.curandDestroyGenerator(gen)


# cuRAND's host Philox generator emits block B of its output from counter
# (c0 | c1 << 32) = B >> 16, c2 = B & 0xFFFF, c3 = 0 under key = seed words;
# the mapping was established empirically and is asserted block by block.
@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 2**64 - 1,
                                  0xDEADBEEF00000000])
@pytest.mark.parametrize("block0", [0, 65535, 3 * 65536 + 5,
                                    (1 << 48) + (7 << 16) + 11])
def test_philox_matches_curand_host_generator(oracle, seed, block0):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    nblk = 24
    ref = _curand_words(lib, seed, 4 * block0, 4 * nblk)
    key = oracle.seed_key(seed)
    for j in range(nblk):
        B = block0 + j
        hi = B >> 16
        ctr = (hi & 0xFFFFFFFF, hi >> 32, B & 0xFFFF, 0)
        got = oracle.philox4x32_10(ctr, key)
        assert np.array_equal(got, ref[4 * j:4 * j + 4]), (seed, B)


def test_weyl_increments_are_the_published_irrationals():
    # The key schedule adds floor(2^32 (phi - 1)) and floor(2^32 (sqrt3 - 1));
    # a wrong increment would already fail the cuRAND comparison, this pins
    # where those numbers come from.
    phi = (1 + 5 ** 0.5) / 2
    assert math.floor((phi - 1) * 2**32) == 0x9E3779B9
    assert math.floor((3 ** 0.5 - 1) * 2**32) == 0xBB67AE85


def test_stream_layout(oracle):
    # sample s, dimension i of (level, slot, trial) is lane s % 4 of the
    # block with counter ((s // 4) * d + i, trial, slot, level).
    seed, level, slot, trial, d = 0xABCDEF12345, 3, 77, 4, 5
    words = oracle.stream_words(seed, level, slot, trial, d, 6, 11)
    key = oracle.seed_key(seed)
    for r, s in enumerate(range(6, 17)):
        for i in range(d):
            blk = oracle.philox4x32_10(((s // 4) * d + i, trial, slot, level), key)
            assert words[r, i] == blk[s % 4]


@pytest.mark.parametrize("w", [0, 1, 2**31, 2**32 - 2, 2**32 - 1, 0x12345678])
def test_uniform64_exact_and_open(oracle, w):
    u = oracle.uniform64(w)
    assert Fraction(u) == Fraction(2 * w + 1, 2**33)
    assert 0.0 < u < 1.0


@pytest.mark.parametrize("block", [(0, 0, 0, 0), (0xFFFFFFFF,) * 4,
                                   (0x12345678, 0x9ABCDEF0, 0x0F1E2D3C, 0x4B5A6978),
                                   (1, 1 << 31, 0x80000001, 0x7FFFFFFF)])
def test_field23_is_the_128_bit_slice(oracle, block):
    # the block read as one little-endian 128-bit integer, sliced 23 bits at a time
    B = sum(int(w) << (32 * j) for j, w in enumerate(block))
    for f in range(5):
        assert oracle.field23(block, f) == (B >> (23 * f)) & ((1 << 23) - 1)


@pytest.mark.parametrize("field", [0, 1, 2**22, 2**23 - 2, 2**23 - 1, 0x5A5A5A])
def test_field_uniform_exact_and_open(oracle, field):
    u = oracle.field_uniform(field)
    assert Fraction(u) == Fraction(2 * field + 1, 2**24)
    assert 0.0 < u < 1.0
    assert float(np.float32(u)) == u          # exactly representable in binary32


@pytest.mark.parametrize("a,b", [((0, 0, 0, 0), (0xFFFFFFFF,) * 4),
                                 ((0xFFFFFFFF,) * 4, (0, 0, 0, 0)),
                                 ((0x12345678, 0x9ABCDEF0, 0x0F1E2D3C, 0x4B5A6978),
                                  (0xDEADBEEF, 0x01234567, 0x89ABCDEF, 0xFEDCBA98))])
def test_pair_field_is_the_two_blocks_slices(oracle, a, b):
    # fields 0..4 from the first block's 128-bit integer, 5..9 from the
    # second's, 10 = bits 115..127 of the first + 2^13 * bits 115..124 of the
    # second: 253 of the pair's 256 bits, each used once
    A = sum(int(w) << (32 * j) for j, w in enumerate(a))
    B = sum(int(w) << (32 * j) for j, w in enumerate(b))
    m23 = (1 << 23) - 1
    want = [(A >> (23 * f)) & m23 for f in range(5)] + [(B >> (23 * f)) & m23 for f in range(5)]
    want.append((A >> 115) + (((B >> 115) & 0x3FF) << 13))
    assert [oracle.pair_field(a, b, f) for f in range(11)] == want


def test_fp32_stream_layout(oracle):
    # point s, dimension i of the FP32 stream is field s % 11 of the pair of
    # blocks with counters (2 ((s // 11) * d + i) + {0, 1}, trial, slot, level)
    seed, level, slot, trial, d = 0x5EED, 2, 41, 3, 3
    u = oracle.stream_uniforms(seed, level, slot, trial, d, True, 7, 30)
    key = oracle.seed_key(seed)
    for r, s in enumerate(range(7, 37)):
        for i in range(d):
            c0 = 2 * ((s // 11) * d + i)
            a = oracle.philox4x32_10((c0, trial, slot, level), key)
            b = oracle.philox4x32_10((c0 + 1, trial, slot, level), key)
            assert u[r, i] == oracle.field_uniform(oracle.pair_field(a, b, s % 11))
    # and the FP64 stream reads whole words, four points per block
    u64 = oracle.stream_uniforms(seed, level, slot, trial, d, False, 7, 12)
    w = oracle.stream_words(seed, level, slot, trial, d, 7, 12)
    assert np.array_equal(u64, (w.astype(np.float64) + 0.5) / 2**32)


def test_fp32_stream_statistics(oracle):
    u = oracle.stream_uniforms(77, 1, 5, 0, 4, True, 0, 50000).ravel()
    N = u.size
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / N)
    assert abs(u.var() - 1 / 12) < 5 * math.sqrt(1 / 180 / N)
    c = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(c) < 5 / math.sqrt(N)


def test_uniform_statistics(oracle):
    # 2^18 uniforms of one stream: mean, variance, lag-1 correlation and a
    # 64-bin chi-square, all at the 5-sigma level.
    d, count = 4, 2**16
    w = oracle.stream_words(2024, 1, 9, 2, d, 0, count).ravel()
    u = (w.astype(np.float64) + 0.5) / 2**32
    N = u.size
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / N)
    assert abs(u.var() - 1 / 12) < 5 * math.sqrt(1 / 180 / N)
    c = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(c) < 5 / math.sqrt(N)
    hist = np.bincount((u * 64).astype(int), minlength=64)
    chi2 = ((hist - N / 64) ** 2 / (N / 64)).sum()
    assert chi2 < 63 + 5 * math.sqrt(2 * 63)


def test_distinct_streams_differ(oracle):
    a = oracle.stream_words(5, 1, 0, 0, 3, 0, 64)
    for args in [(5, 2, 0, 0), (5, 1, 1, 0), (5, 1, 0, 1), (6, 1, 0, 0)]:
        b = oracle.stream_words(*args, 3, 0, 64)
        assert not np.array_equal(a, b)
