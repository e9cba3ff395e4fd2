"""Philox4x32-10 against the known-answer vectors published with the Random123 library
(Salmon et al., SC'11)."""
from oracle.philox import philox4x32_10, uniform53


def test_kat_zero():
    assert philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]


def test_kat_ones():
    assert philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]


def test_kat_pi():
    ctr = [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]
    key = [0xA4093822, 0x299F31D0]
    assert philox4x32_10(ctr, key) == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_uniform_range_and_mean():
    us = [uniform53((i, 0, 0, 0), (7, 0)) for i in range(4000)]
    assert all(0.0 <= u < 1.0 for u in us)
    assert abs(sum(us) / len(us) - 0.5) < 0.02
