"""The split search's child index for full lower nodes, without a 64-bit
remainder (the digit-sum identity of the search kernel), checked on the host;
also in the form the kernel evaluates it, with the digits of the hash read
from the remix's value before its last xor-shift.

A full lower node of MM keys has parts of U = 2^a b keys; the search needs
p >> a for p = h mod MM.  As 2^a divides MM, p >> a = (h >> a) mod D with
D = MM >> a.  With D = 2^t D' (D' odd) and k a multiple of the order of 2
modulo D', (h >> (a + t)) mod D' is the sum of its k-bit digits mod D', and
the low t bits are copied.  This file restates those steps, with the same
digit positions and widths as the kernel, in Python integers and compares
them with the definition for every compiled leaf size (8, 12, 16) and both
lower levels, on random hashes and on hashes at the edges (all ones, top
bits set, digit boundaries)."""
import numpy as np
import pytest

COMPILED_LEAVES = (8, 12, 16)


def fanouts(leaf):
    return max(2, (35 * leaf + 154) // 100), max(2, (21 * leaf + 189) // 100)


def ctz(x):
    return (x & -x).bit_length() - 1


def order_of_two(d):
    if d <= 1:
        return 1
    e, p = 1, 2 % d
    while p != 1:
        p, e = (2 * p) % d, e + 1
    return e


def bits(h, pos, width):
    return (h >> pos) & ((1 << width) - 1)


def hbits_from_pre(y, pos, width):
    """Bits [pos, pos + width) of h = y ^ (y >> 31) (the remix's last
    xor-shift) read from y as the kernel does: the field of y xor the field
    31 bits higher, zero past bit 63."""
    v = (y >> pos) & 0xFFFFFFFF
    if pos + 31 < 64:
        v ^= (y >> (pos + 31)) & 0xFFFFFFFF
    return v & ((1 << width) - 1)


def child_index(h, mm, a, field=bits):
    """The kernel's steps: digits of h >> z (z = a + t) of k bits, their sum
    (with the carry of two 32-bit digits added back), its remainder mod D',
    and the low t bits of h >> a below it."""
    d = mm >> a
    t = ctz(d)
    dp = d >> t
    z = a + t
    e = order_of_two(dp)
    k = (32 // e) * e
    r = 0
    if dp > 1:
        if k == 32:
            d0 = field(h, z, min(64 - z, 32))
            if z + 32 < 64:
                s = d0 + field(h, z + 32, 32 - z)
                if s >= 1 << 32:  # 2^32 = 1 (mod D'): the carry adds one
                    s = s - (1 << 32) + 1
            else:
                s = d0
        else:
            assert 64 - z <= 3 * k and k <= 30
            s = field(h, z, k)
            if z + k < 64:
                s += field(h, z + k, min(64 - z - k, k))
            if z + 2 * k < 64:
                s += field(h, z + 2 * k, 64 - z - 2 * k)
        assert s < 1 << 32  # the kernel sums in 32-bit registers
        r = s % dp
    if t:
        return (r << t) | field(h, a, t)
    return r


def full_lower_nodes():
    for leaf in COMPILED_LEAVES:
        f1, f2 = fanouts(leaf)
        l1 = f1 * leaf
        yield leaf, l1, leaf          # lower-1: parts of l keys
        yield leaf, f2 * l1, l1       # lower-2: parts of l1 keys


def edge_hashes():
    out = [0, 1, (1 << 64) - 1, 1 << 63, (1 << 32) - 1, 1 << 32, ((1 << 32) - 1) << 32]
    for p in range(64):
        out += [(1 << p) - 1, ((1 << 64) - 1) ^ ((1 << p) - 1), 1 << p]
    return out


@pytest.mark.parametrize("leaf,mm,unit", list(full_lower_nodes()))
def test_digit_sum_child_index_equals_the_remainder(leaf, mm, unit):
    a = ctz(unit)
    assert mm % (1 << a) == 0
    rng = np.random.default_rng(7000 + mm)
    hs = [int(x) for x in rng.integers(0, 2**64, 100_000, dtype=np.uint64)] + edge_hashes()
    for h in hs:
        assert child_index(h, mm, a) == (h % mm) >> a, (leaf, mm, h)


@pytest.mark.parametrize("leaf,mm,unit", list(full_lower_nodes()))
def test_the_index_read_before_the_last_xor_shift(leaf, mm, unit):
    """The kernel reads the digits of h = y ^ (y >> 31) from y directly."""
    a = ctz(unit)
    rng = np.random.default_rng(7100 + mm)
    ys = [int(x) for x in rng.integers(0, 2**64, 100_000, dtype=np.uint64)] + edge_hashes()
    for y in ys:
        h = y ^ (y >> 31)
        assert child_index(y, mm, a, field=hbits_from_pre) == (h % mm) >> a, (leaf, mm, y)


@pytest.mark.parametrize("leaf,mm,unit", list(full_lower_nodes()))
def test_the_index_gives_the_child(leaf, mm, unit):
    """The increment tables hold child q // b at index q = p >> a: the same
    child as p // unit for every position p of the node."""
    a = ctz(unit)
    b = unit >> a
    for p in range(mm):
        assert (p >> a) // b == p // unit


def test_digit_widths_of_the_compiled_sizes():
    """The cases the kernel comments name: at l = 16, D = 7 with two 30-bit
    digits and D = 35 with three 24-bit digits; at l = 12, D = 15 and 60 with
    32-bit digits; at l = 8, D = 4 (bits only) and 3."""
    got = {}
    for leaf, mm, unit in full_lower_nodes():
        a = ctz(unit)
        d = mm >> a
        dp = d >> ctz(d)
        got[(leaf, mm)] = (d, (32 // order_of_two(dp)) * order_of_two(dp) if dp > 1 else None)
    assert got[(16, 112)] == (7, 30) and got[(16, 560)] == (35, 24)
    assert got[(12, 60)] == (15, 32) and got[(12, 240)] == (60, 32)
    assert got[(8, 32)] == (4, None) and got[(8, 96)] == (3, 32)
