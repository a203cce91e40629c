"""The seeded input generator (synth/) against its published definition and
its own stated properties.  Pure host code; no GPU and no oracle."""

import numpy as np

import synth

# SplitMix64's reference sequence from state 0 (the first four outputs of the
# generator of Steele, Lea and Flood, as published with it).  With stream 0
# the counter-based stream here walks the same states (i * gamma), so its
# first elements must be exactly these.
SPLITMIX64_FROM_ZERO = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_stream_zero_is_the_splitmix64_reference_sequence():
    assert [int(x) for x in synth.raw64(0, 4)] == SPLITMIX64_FROM_ZERO


def test_offsets_and_chunks_are_consistent():
    seed = 1234567
    full = synth.raw64(seed, 5000)
    np.testing.assert_array_equal(synth.raw64(seed, 1000, start=4000), full[4000:])
    u = synth.uniform01(seed, 5000)
    np.testing.assert_array_equal(synth.uniform01(seed, 5000, chunk=333), u)
    np.testing.assert_array_equal(synth.uniform01(seed, 1000, start=4000), u[4000:])


def test_uniform01_and_u16_take_the_stated_bits():
    seed = 99
    raw = synth.raw64(seed, 20000)
    u = synth.uniform01(seed, 20000)
    np.testing.assert_array_equal(u, (raw >> np.uint64(11)).astype(np.float64) * 2.0 ** -53)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1.0 / 12.0) < 0.005
    v = synth.uniform_u16(seed, 20000)
    np.testing.assert_array_equal(v, (raw >> np.uint64(48)).astype(np.int32))
    assert v.min() >= 0 and v.max() <= 65535


def test_streams_differ_and_repeat():
    a = synth.uniform01(1001, 1000)
    np.testing.assert_array_equal(a, synth.uniform01(1001, 1000))
    assert not np.array_equal(a, synth.uniform01(1002, 1000))
